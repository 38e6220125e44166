"""Host side of multi-GPU runs: every rank builds and solves its own replica of the workload
(the rows of one toolbox are independent, but every run here has one GPU per process and no
data-path exchange), and the timing is combined across ranks: the job's time is the slowest
rank's, its work the sum of the ranks' work."""
from __future__ import annotations


def combine(ms_total: float, work: float, device=None):
    """(max of ms_total, sum of work) over the ranks of the default process group (identity
    without one).  device: where the reduction tensors live (CUDA for NCCL, CPU for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms_total, work
    t = torch.tensor([float(ms_total)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())
