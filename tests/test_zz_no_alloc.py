"""The allocation-free toolbox build (ewos_toolbox_build_noalloc) against the ordinary build.

Callers that cannot call cudaMalloc (code under an allocator that owns all device memory, or
that must not allocate while other work is in flight) use the no-allocation entry point: they
pass the output matrices and the library keeps its temporaries in a static device array.  The
test calls it twice in a row through the C ABI and compares both results with
ewos_toolbox_build on the same inputs: exit counts bit-exact, G, grad G and grad H within the
1e-4 relative rule of the parity tests (shared-memory atomics add in a different order).
This file is collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from paper_2608_07017_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _close(a, b, rel=1e-4):
    scale = np.maximum(np.abs(b), np.abs(b).mean(axis=-1, keepdims=True))
    return bool(np.all(np.abs(a - b) <= rel * scale + 1e-30))


def test_noalloc_build_matches_ordinary_build_twice():
    import torch
    from paper_2608_07017_b300 import build, ewos
    build.build()
    w = W.square(32, 32, walks=2000, eps=1e-4, problem=False)
    n, p, d = w.x.shape[0], w.z.shape[0], 2
    tb = ewos.build_toolbox("box", d, w.domain.params, w.x, w.z, w.walks, w.eps, seed=w.seed, precision=32,
                            cell_samples=1000)
    ref = dict(G=tb.get("G"), gradG=tb.get("gradG"), Hc=tb.get("Hc"), gradH=tb.get("gradH"))
    ref_steps = tb.report()["steps"]
    tb.close()
    dev = torch.device("cuda", 0)
    xd = torch.from_numpy(w.x).to(dev)
    zd = torch.from_numpy(w.z).to(dev)
    for call in range(2):
        P = torch.full(((d + 1), n, n), float("nan"), dtype=torch.float32, device=dev)
        KH = torch.full(((d + 1), n, p), float("nan"), dtype=torch.float32, device=dev)
        Hc = torch.full((n, p), -1, dtype=torch.int32, device=dev)
        st, rep = ewos.build_toolbox_noalloc("box", d, w.domain.params, xd, zd, w.walks, w.eps, P, KH, Hc,
                                             seed=w.seed)
        torch.cuda.synchronize()
        assert st == ewos.OK, call
        assert rep["steps"] == ref_steps and rep["capped"] == 0, call
        Pn, KHn = P.double().cpu().numpy(), KH.double().cpu().numpy()
        Hn = Hc.cpu().numpy().view(np.uint32)
        assert np.array_equal(Hn, ref["Hc"]), call
        assert _close(Pn[d], ref["G"]), call
        for c in range(d):
            assert _close(Pn[c], ref["gradG"][c]), call
            assert _close(KHn[c], ref["gradH"][c]), call
        assert np.allclose(KHn[d], ref["Hc"] / w.walks, rtol=0, atol=1e-7), call
