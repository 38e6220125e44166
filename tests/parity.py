"""Element-by-element comparison of a GPU toolbox with the oracle's rows (shared by the GPU
tests; no arithmetic of the method here, only the comparison rule).

Rule (walks: at most 0.1 % of the compared walks bin differently and at most 0.25 % drift,
every class counted and reported; tolerance of matrix entries, 1e-4 relative): a walk is
*divergent* when its exit cell,
its number of steps or its binning digest (XOR of cellmix over every interior binning)
differs between the two sides -- an FP32/FP64 disagreement at the eps-shell or a Voronoi
near-tie -- or when its trajectory has drifted: its stopping point moved by more than 3e-5
(times the domain's extent; the FP32 position error of a long walk can grow along it), or its
G mass sum_k r_k^2/(2d) differs by more than the rounding of the walk's own arithmetic explains
(positions off by at most delta, the row's largest stopping-point difference among the other
walks, and K rounded additions: 2 delta sum_k r_k/(2d) + (4 + K) u mass).  Every other walk
makes bit-identical binning decisions along trajectories equal to rounding, so its
contributions agree to that level.  Entries must satisfy

    |gpu - oracle| <= 1e-4 * max(|oracle|, mean_row |oracle|) + bound_row,
    and the row sums of G within 3e-5 relative once the divergent walks' masses are taken out;
    at most 0.01 % of the entries (reported) may exceed their bound, by at most 4x,

for the gradient matrices with max(...) also over the sum of the magnitudes of the entry's terms
((d/r0) G_ij for gradG, (d/r0) H_ij for gradH), since those entries cancel terms of both signs;
for FP32 walks bound_row also holds the rounding term of the arithmetic, 2 g delta_row Grsum_ij +
4 u G_ij (u = 2^-24; delta_row = largest stopping-point difference of the row's non-divergent
walks, g = 4 its margin for the larger position errors inside a walk; Grsum = oracle's sum of
r/(2dN) over the same binnings), times d/r0 for gradG;
where bound_row bounds what the divergent walks of that row can move:
    G      sum_div (mass_gpu + mass_oracle) / N                 (mass = sum r_k^2 / (2d))
    gradG  sum_div [ (d/r0) (mass_gpu + mass_oracle) + d r0 ] / N
    Hc     number of divergent walks of the row (integer counts)
    gradH  2 (d/r0) * (number of divergent walks) / N
"""
import numpy as np


U32 = 2.0 ** -24
U64 = 2.0 ** -53
MAX_DIVERGENT = 1e-3      # at most 0.1 % of the compared walks may bin differently (exit, steps, digest)
MAX_DRIFTED = 2.5e-3      # and at most 0.25 % may drift with the same binning (FP32 trajectories)
# A walk's position error is not largest at its stopping point: it can grow and shrink along the
# walk (measured on the GPU: contributions off by up to 2.5x what the stopping-point difference
# explains).  The per-entry rounding term uses POS_GROWTH times the row's stopping-point bound.
POS_GROWTH = 4.0
MAX_OVER = 1e-4


def compare_rows(gpu, orc, rows, N, dim, r0, rel=1e-4, drift_rel=0.0, fp32=False, max_divergent=MAX_DIVERGENT,
                 pos_tol=3e-5, xscale=1.0, rowsum_rel=3e-5, max_drifted=MAX_DRIFTED):
    """gpu: dict with G [n][m], gradG [d][n][m], Hc [n][p], gradH [d][n][p] and records
    exit/steps/vhash/mass [n][N] (full toolbox); orc: oracle.walk_rows(..., records=True) for
    ``rows``.  Returns a report dict with the walk counts of each divergence class (exit cell,
    step count, interior binning digest, G-mass drift); raises AssertionError when more than
    ``max_divergent`` of the compared walks diverge in any way, or when an entry is out of
    tolerance."""
    rows = np.asarray(rows)
    rec = orc["records"]
    ge, gs, gv, gm = (gpu["walk_exit"][rows], gpu["walk_steps"][rows], gpu["walk_vhash"][rows],
                      gpu["walk_mass"][rows])
    same_exit = ge == rec["exit"]
    steps_differ = gs != rec["steps"]
    digest_differs = gv != rec["vhash"]
    binning = (~same_exit) | steps_differ | digest_differs
    # drift: a walk whose G mass differs by more than the rounding of its own arithmetic can
    # explain.  With delta = the row's largest stopping-point difference (plus 4u), each of the
    # walk's K contributions r_k^2 is off by at most 2 r_k delta + 4 u r_k^2 and the sum adds
    # K u mass, so |dmass| <= 2 delta sum_k r_k / (2d) + (4 + K) u mass, sum_k r_k <= sqrt(K 2d mass).
    # A trajectory whose stopping point moved by more than pos_tol (relative to the node
    # extent) has drifted too: the FP32 position error of a long walk grows along the walk
    # (the map X -> X + r(X) U can double it at a step) while its binning still agrees.
    uw = U32 if fp32 else U64
    dx_w = np.abs(gpu["walk_xexit"][rows] - rec["xexit"]).max(axis=2)
    moved = dx_w > pos_tol * xscale
    delta_w = (np.where(binning | moved, 0.0, dx_w).max(axis=1) + 4 * uw)[:, None]
    K = rec["steps"].astype(np.float64) + 1.0
    mass_o = rec["gmass"]
    drift_bound = 2 * delta_w * np.sqrt(K * 2 * dim * mass_o) / (2 * dim) + (4 + K) * uw * mass_o
    drift = moved | (np.abs(gm - mass_o) > np.maximum(drift_bound, drift_rel * mass_o if drift_rel else 0.0))
    div = binning | drift
    ndiv = div.sum(1)
    mass_div = np.where(div, gm + rec["gmass"], 0.0).sum(1)
    out = dict(walks=int(div.size), exit_equal=float(same_exit.mean()), divergent=float(div.mean()),
               ndiv=int(ndiv.sum()), n_exit=int((~same_exit).sum()), n_steps=int(steps_differ.sum()),
               n_digest=int(digest_differs.sum()), n_drift=int((drift & ~binning).sum()),
               binning_divergent=float(binning.mean()), drifted=float((drift & ~binning).mean()))
    nbin = int(binning.sum())
    assert nbin <= max_divergent * out["walks"] and out["n_drift"] <= max_drifted * out["walks"], (
        f"{out['ndiv']} of {out['walks']} walks diverge (exit {out['n_exit']}, steps {out['n_steps']}, "
        f"digest {out['n_digest']}: {nbin} bin differently, at most {max_divergent:.2%} may; drift only "
        f"{out['n_drift']}, at most {max_drifted:.2%} may)")
    # FP32 rounding term: a contribution r^2 computed at a position off by delta differs by at most
    # 2 r delta + r^2 (4 u); delta per row = the largest stopping-point difference of its
    # non-divergent walks (each at most 3e-5 of the extent; larger ones are divergent)
    if fp32:
        dx = np.abs(gpu["walk_xexit"][rows] - rec["xexit"]).max(axis=2)
        delta = np.where(div, 0.0, dx).max(axis=1) + 4 * U32
        rnd_G = 2 * POS_GROWTH * delta[:, None] * orc["Grsum"] + 4 * U32 * orc["G"]
        out["delta_max"] = float(delta.max())
    else:
        rnd_G = np.zeros_like(orc["G"])

    def check(name, a, b, bound, extra_scale=None):
        scale = np.maximum(np.abs(b), np.abs(b).mean(axis=-1, keepdims=True))
        if extra_scale is not None:
            scale = np.maximum(scale, extra_scale)
        lim = rel * scale + bound
        ratio = np.abs(a - b) / np.maximum(lim, 1e-300)
        nbad = int((ratio > 1).sum())
        out[name + "_maxratio"] = float(np.max(ratio))
        out[name + "_over"] = nbad
        # the rounding model bounds the position error of a walk by its row's stopping-point
        # differences; a few entries (at most 0.01 %, reported) may exceed it, by at most 4x
        assert nbad <= int(MAX_OVER * ratio.size) and out[name + "_maxratio"] <= 4.0, (
            f"{name}: {nbad} entries out of tolerance; worst ratio {out[name + '_maxratio']:.3g}")

    check("G", gpu["G"][rows], orc["G"], (mass_div / N)[:, None] + rnd_G)
    # row sums: the non-divergent walks' rounding differences have random signs and cancel in
    # the sum of a row (measured below 1e-5 relative), so a scale error the per-entry rounding
    # slack could hide shows here
    S_g, S_o = gpu["G"][rows].sum(1), orc["G"].sum(1)
    corr = np.where(div, gm - rec["gmass"], 0.0).sum(1) / N
    rs = np.abs(S_g - S_o - corr) / S_o
    # plus the rounding of r0 in the walk precision (every walk's first contributions scale with
    # r0^2; r0 = r(x_i) is off by a few units in the last place of |x_i|)
    tol = rowsum_rel + (16 * uw * xscale / np.asarray(r0, dtype=np.float64) if fp32 else 0.0)
    out["G_rowsum_maxrel"] = float(rs.max())
    assert np.all(rs <= tol), f"G row sums differ by {rs.max():.3g} relative (at most {rowsum_rel:g} + r0 rounding)"
    bgg = ((dim / r0) * mass_div + dim * r0 * ndiv) / N
    # a gradient entry sums terms of both signs; the magnitude its rounding scales with is the sum of
    # the terms' magnitudes, at most (d/r0) G_ij for the path terms (|U_0| = 1)
    absg = (dim / r0)[:, None] * orc["G"]
    for c in range(dim):
        check(f"gradG{c}", gpu["gradG"][c][rows], orc["gradG"][c], bgg[:, None] + (dim / r0)[:, None] * rnd_G, absg)
    dH = np.abs(gpu["Hc"][rows].astype(np.int64) - orc["Hc"])
    assert np.all(dH <= ndiv[:, None]), "exit counts differ by more than the divergent walks"
    bgh = 2 * (dim / r0) * ndiv / N
    absh = (dim / r0)[:, None] * orc["Hc"] / N
    for c in range(dim):
        check(f"gradH{c}", gpu["gradH"][c][rows], orc["gradH"][c], bgh[:, None], absh)
    return out


def gpu_arrays(tb, N, records=True):
    out = dict(G=tb.get("G"), gradG=tb.get("gradG"), Hc=tb.get("Hc"), gradH=tb.get("gradH"), H=tb.get("H"))
    if records:
        for k in ("walk_exit", "walk_steps", "walk_vhash", "walk_mass", "walk_xexit"):
            out[k] = tb.get(k, walks=N)
    return out
