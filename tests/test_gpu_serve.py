"""Batched right-hand sides (CUDA-graph sweeps, chord iteration) and the request server.

* batched mixed solves agree with the oracle's solves on the same toolbox and the same alpha
  (1e-9 linear, 1e-8 semilinear: the chord iteration and Newton stop at the same zero of
  R(s) + alpha s to the 1e-10 residual tolerance);
* a semilinear request too strong for the chord iteration falls back to Newton and still
  agrees;
* each request's result is the same alone (one slot) and inside a mix of concurrent requests
  on several slots (1e-10: only the order of floating-point atomics differs);
* admission by memory: a budget that holds one workspace serialises the requests, a budget
  below one workspace rejects them with EWOS_ENOMEM.
"""
import numpy as np
import pytest

import oracle
from oracle import solve as S
from paper_2608_07017_b300 import ewos
from paper_2608_07017_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def disk():
    from paper_2608_07017_b300 import build
    build.build()
    w = W.disk400()
    r = oracle.walk_rows(2, "ball", w.domain.params, w.x, w.z, 1000, 1e-3, 0)
    lam = np.full(400, 1.0 / 400)
    # FP32 toolbox (as the server's toolboxes are); the oracle solves with the same FP32-rounded
    # entries, so both sides solve the same system
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    tb = dict(G=f32(r["G"]), gradG=f32(r["gradG"]), H=f32(r["Hc"] / 1000.0), gradH=f32(r["gradH"]))
    gtb = ewos.toolbox_from_host(2, w.x, w.z, tb["G"], tb["gradG"], tb["H"], tb["gradH"], lam, precision=32)
    yield w, tb, lam, gtb
    gtb.close()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_batched_linear_matches_oracle(disk):
    w, tb, lam, gtb = disk
    rq = W.serving_requests(w.x, w.z, 1, seed=5, nrhs=5, p_semilinear=0.0)[0]
    U, _, rep = gtb.solve(rq["A"], rq["f"], rq["g"], b=rq["b"], mode="mixed", batched=True)
    assert rep["converged"] and rep["factorizations"] == 1
    Ue, _, _ = gtb.solve(rq["A"], rq["f"], rq["g"], b=rq["b"], mode="mixed", batched=False)
    for r in range(5):
        ref = S.solve_linear(tb, lam, rq["A"], rq["b"], None, rq["f"][r], rq["g"][r], alpha=rep["alpha"])
        assert _rel(U[r], ref["u"]) < 1e-9
        assert _rel(U[r], Ue[r]) < 1e-9


def test_batched_semilinear_chord_matches_newton(disk):
    w, tb, lam, gtb = disk
    rq = W.serving_requests(w.x, w.z, 1, seed=6, nrhs=3, p_semilinear=1.0)[0]
    U, _, rep = gtb.solve(rq["A"], rq["f"], rq["g"], b=rq["b"], kind="semilinear", coef=rq["coef"], mode="mixed",
                          batched=True)
    assert rep["converged"] and rep["factorizations"] == 1      # chord: one factorisation
    for r in range(3):
        ref = S.newton(tb, lam, rq["A"], rq["b"], None, rq["f"][r], rq["g"][r], rq["coef"], alpha=rep["alpha"])
        assert ref["converged"]
        assert _rel(U[r], ref["u"]) < 1e-8


def test_batched_semilinear_falls_back_to_newton(disk):
    # u* three times larger: N'(u) = 3u^2 ~ 30 makes the chord iteration diverge
    w, tb, lam, gtb = disk
    pb = w.problem
    us = 3.0 * pb.u_star
    f3 = 3.0 * pb.f + us ** 3
    F = np.stack([f3, f3])
    G = np.stack([3.0 * pb.g, 3.0 * pb.g])
    U, _, rep = gtb.solve(pb.A, F, G, kind="semilinear", coef=[0, 0, 0, 1], mode="mixed", batched=True)
    assert rep["converged"] and rep["factorizations"] > 1       # Newton refactorises
    ref = S.newton(tb, lam, pb.A, None, None, f3, 3.0 * pb.g, [0, 0, 0, 1], alpha=rep["alpha"])
    assert _rel(U[0], ref["u"]) < 1e-8 and _rel(U[1], ref["u"]) < 1e-8


def _submit_all(sv, gtb, reqs, mode="mixed"):
    return [sv.submit(gtb, q["A"], q["f"], q["g"], b=q["b"], kind=q["kind"], coef=q["coef"], mode=mode)
            for q in reqs]


def test_server_result_same_alone_and_in_the_mix(disk):
    w, tb, lam, gtb = disk
    reqs = W.serving_requests(w.x, w.z, 8, seed=7, nrhs_max=16)
    probe = 5
    sv1 = ewos.Server(max_slots=1)
    t = _submit_all(sv1, gtb, [reqs[probe]])[0]
    u_alone, _, rep_alone, _ = sv1.wait(t)
    sv1.close()
    sv = ewos.Server(max_slots=4)
    tickets = _submit_all(sv, gtb, reqs)
    outs = [sv.wait(t) for t in tickets]
    st = sv.stats()
    sv.close()
    assert st["completed"] == 8 and st["failed"] == 0
    assert st["peak_active"] >= 2                                # requests overlapped
    assert {o[3]["slot"] for o in outs} != {0} or st["slots"] == 1
    u_mix = outs[probe][0]
    assert _rel(u_mix, u_alone) < 1e-10
    # every request against the oracle on the same toolbox and alpha
    for q, (u, _, rep, tm) in zip(reqs, outs):
        assert rep["converged"] and tm["total_ms"] >= tm["run_ms"] >= 0
        U = u.reshape(q["f"].shape[0], -1)
        r = 0
        if q["kind"] == "linear":
            ref = S.solve_linear(tb, lam, q["A"], q["b"], None, q["f"][r], q["g"][r], alpha=rep["alpha"])
        else:
            ref = S.newton(tb, lam, q["A"], q["b"], None, q["f"][r], q["g"][r], q["coef"], alpha=rep["alpha"])
        assert _rel(U[r], ref["u"]) < 1e-8


def test_server_fp64_requests(disk):
    w, tb, lam, gtb = disk
    reqs = W.serving_requests(w.x, w.z, 2, seed=8, nrhs=2, p_semilinear=0.0)
    sv = ewos.Server(max_slots=2)
    tickets = _submit_all(sv, gtb, reqs, mode="fp64")
    for q, t in zip(reqs, tickets):
        u, _, rep, _ = sv.wait(t)
        ref = S.solve_linear(tb, lam, q["A"], q["b"], None, q["f"][1], q["g"][1])
        assert _rel(u[1], ref["u"]) < 1e-9
    sv.close()


def test_server_admission_by_memory(disk):
    w, tb, lam, gtb = disk
    reqs = W.serving_requests(w.x, w.z, 3, seed=9, nrhs=4, p_semilinear=0.0)
    # the estimate of one workspace, from a server that ran one request
    sv = ewos.Server(max_slots=1)
    sv.wait(_submit_all(sv, gtb, reqs[:1])[0])
    one = sv.stats()["charged_bytes"]
    sv.close()
    assert one > 0
    # room for one workspace: the requests run one at a time
    sv = ewos.Server(max_slots=3, budget_bytes=int(1.5 * one))
    tickets = _submit_all(sv, gtb, reqs)
    for t in tickets:
        sv.wait(t)
    st = sv.stats()
    sv.close()
    assert st["completed"] == 3 and st["peak_active"] == 1 and st["charged_bytes"] <= 1.5 * one
    # below one workspace: rejected, nothing runs
    sv = ewos.Server(max_slots=2, budget_bytes=1 << 20)
    t = _submit_all(sv, gtb, reqs[:1])[0]
    with pytest.raises(ewos.EwosError) as e:
        sv.wait(t)
    assert e.value.status == ewos.ENOMEM
    sv.close()


def test_server_slot_reused_by_a_new_toolbox_of_the_same_shape(disk):
    # One slot: its workspace (and the sweep graph cached in it) outlives the first toolbox.  A
    # second toolbox of the same shape, made after the first is destroyed (often at the same host
    # address), must be solved with its own operators, not with a graph of the destroyed one.
    w, tb, lam, gtb = disk
    q = W.serving_requests(w.x, w.z, 1, seed=11, nrhs=3, p_semilinear=0.0)[0]

    def scaled(scale):      # FP32-rounded, as the toolbox stores it, so the oracle solves the same system
        return {k: (np.asarray(scale * v, np.float32).astype(np.float64) if k in ("G", "gradG") else v)
                for k, v in tb.items()}

    def make(scale):
        t = scaled(scale)
        return ewos.toolbox_from_host(2, w.x, w.z, t["G"], t["gradG"], t["H"], t["gradH"], lam, precision=32)

    sv = ewos.Server(max_slots=1)
    a = make(1.0)
    sv.wait(_submit_all(sv, a, [q])[0])
    a.close()
    b = make(0.8)
    u_reused, _, rep, _ = sv.wait(_submit_all(sv, b, [q])[0])
    sv.close()
    fresh = ewos.Server(max_slots=1)
    u_fresh, _, _, _ = fresh.wait(_submit_all(fresh, b, [q])[0])
    fresh.close()
    b.close()
    assert rep["converged"]
    assert _rel(u_reused, u_fresh) < 1e-10
    ref = S.solve_linear(scaled(0.8), lam, q["A"], q["b"], None, q["f"][0], q["g"][0], alpha=rep["alpha"])
    assert _rel(u_reused.reshape(3, -1)[0], ref["u"]) < 1e-8
