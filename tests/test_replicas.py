"""Multi-rank combination of the benchmark's timing (world size 2, gloo on CPU): the job time is
the slowest rank's and the work is summed, as bench.py does for --gpus N."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2608_07017_b300.replicas import combine
    ms, work = combine(10.0 + 5.0 * rank, 100.0 * (rank + 1))
    out[rank] = (ms, work)
    dist.barrier()
    dist.destroy_process_group()


def test_combine_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == (15.0, 300.0) and out[1] == (15.0, 300.0)


def test_combine_single_process_is_identity():
    from paper_2608_07017_b300.replicas import combine
    assert combine(3.5, 7.0) == (3.5, 7.0)
