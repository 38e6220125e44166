"""Failure paths, made on purpose without faulting, trapping or hanging the GPU.

* A bounded device wait that runs out: the flag waits of the dataflow triangular solves get a
  limit of 0 polls (a test hook), so every wait that does not find its flag already set gives
  up; the kernels return, the call reports EWOS_ETIMEOUT, and with the default limit restored
  the same toolbox solves again to the same result.  These waits poll plain flags: no copy is in
  flight when they give up.
* A device allocation that fails: a host-side hook makes the library's next allocations fail
  as if the device were out of memory; builds and solves report EWOS_ENOMEM and the next call
  succeeds.
"""
import numpy as np
import pytest

from paper_2608_07017_b300 import ewos
from paper_2608_07017_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2608_07017_b300 import build
    build.build()


@pytest.fixture(scope="module")
def square():
    w = W.square(16, 16, walks=400, eps=1e-4)
    tb = ewos.build_workload(w, cell_samples=100000)
    yield w, tb
    tb.close()


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_flow_wait_timeout_is_reported_and_the_device_stays_usable(square, mode):
    w, tb = square
    pb = w.problem
    u0, _, _ = tb.solve(pb.A, pb.f, pb.g, b=pb.b, mode=mode)
    ewos.debug_set_flow_wait_limit(0)
    try:
        with pytest.raises(ewos.EwosError) as ei:
            tb.solve(pb.A, pb.f, pb.g, b=pb.b, mode=mode)
        assert ei.value.status == ewos.ETIMEOUT
    finally:
        ewos.debug_set_flow_wait_limit(-1)
    u1, _, rep = tb.solve(pb.A, pb.f, pb.g, b=pb.b, mode=mode)
    assert rep["converged"]
    assert np.max(np.abs(u1 - u0)) <= 1e-12 * np.max(np.abs(u0))


def test_allocation_failure_reports_enomem_and_the_next_call_succeeds(square):
    w, tb = square
    pb = w.problem
    ref = tb.get("Hc")
    for after in (0, 2, 7):
        ewos.debug_fail_allocations(after)
        try:
            with pytest.raises(ewos.EwosError) as ei:
                ewos.build_workload(w, cell_samples=100000)
            assert ei.value.status == ewos.ENOMEM
        finally:
            ewos.debug_fail_allocations(-1)
    again = ewos.build_workload(w, cell_samples=100000)
    assert np.array_equal(again.get("Hc"), ref)
    # a solve on a new toolbox whose workspace allocation fails, then the same solve again
    # (compared with the solve of a third, identical build: the FP32 accumulation order of the
    # builds differs, so the toolboxes agree to rounding, not bit for bit)
    third = ewos.build_workload(w, cell_samples=100000)
    u_ref, _, _ = third.solve(pb.A, pb.f, pb.g, b=pb.b, mode="mixed")
    third.close()
    ewos.debug_fail_allocations(0)
    try:
        with pytest.raises(ewos.EwosError) as ei:
            again.solve(pb.A, pb.f, pb.g, b=pb.b, mode="mixed")
        assert ei.value.status == ewos.ENOMEM
    finally:
        ewos.debug_fail_allocations(-1)
    u, _, rep = again.solve(pb.A, pb.f, pb.g, b=pb.b, mode="mixed")
    assert rep["converged"] and np.max(np.abs(u - u_ref)) <= 1e-5 * np.max(np.abs(u_ref))
    u2, _, _ = again.solve(pb.A, pb.f, pb.g, b=pb.b, mode="mixed")
    assert np.max(np.abs(u2 - u)) <= 1e-12 * np.max(np.abs(u))
    again.close()
