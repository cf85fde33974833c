"""Shared helpers of the GPU-vs-oracle parity tests.

Element-wise comparison of one GPU half-step with the oracle's from the same
state and the same Philox draws. The GPU computes in FP32 with the hardware
sin/cos/exp approximations, the oracle in FP64, so a site may legitimately take
the other branch of a decision when the oracle sees that decision within
rounding of its threshold:
  * Metropolis accepts iff dE < theta = -T ln u1 (equivalent to the paper's
    rule); a flip needs |dE - theta| below TIE_E;
  * the over-relaxed candidate is kept iff it lies in [0, 2pi]; a flip needs
    it within TIE_PHI of an end.
Every other site must agree within ATOL + RTOL_PSI / R, where R = |C + iS| is
the length of the neighbour field (the reflection angle psi = atan2(S, C) is
ill-conditioned as R -> 0).
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2 * np.pi
ATOL = 2e-5
RTOL_PSI = 2e-5
TIE_E = 1e-4
TIE_PHI = 1e-4


def checkerboard(H, W):
    yy, xx = np.mgrid[0:H, 0:W]
    return (yy + xx) & 1


def compare_site_updates(gpu, ora, pre, diag, may_move, storage=0):
    """Returns (n_sites_checked, n_explained_flips, n_bad, message).

    storage (1 BF16, 2 FP16): both sides round the reflected angle to the
    stored type; a site whose reflected angle lies within rounding of the
    midpoint between two stored values may round either way (the GPU takes
    it from FP32 arithmetic, the oracle from FP64)."""
    gpu = np.asarray(gpu, np.float64)
    ora = np.asarray(ora, np.float64)
    pre = np.asarray(pre, np.float64)
    # Sites that must not move: bitwise unchanged.
    still = ~may_move
    bad_still = int(np.count_nonzero(gpu[still] != pre[still]))
    d = np.abs(gpu - ora)
    R = np.maximum(diag["R"], 1e-6)
    tol = ATOL + RTOL_PSI / R
    ok = d <= tol
    por = diag["phi_or"]
    fin = np.isfinite(por)
    or_tie = np.zeros_like(ok)
    or_tie[fin] = (np.abs(por[fin]) < TIE_PHI + tol[fin]) | \
                  (np.abs(por[fin] - TWO_PI) < TIE_PHI + tol[fin])
    acc_tie = np.abs(diag["dE"] - diag["theta"]) < TIE_E
    round_tie = np.zeros_like(ok)
    if storage:
        import oracle
        for idx in np.argwhere(may_move & ~ok & fin):
            v, e = float(por[tuple(idx)]), float(tol[tuple(idx)])
            round_tie[tuple(idx)] = oracle.round_store(v - e, storage) != oracle.round_store(v + e, storage)
    explained = may_move & ~ok & (or_tie | acc_tie | round_tie)
    bad = may_move & ~ok & ~(or_tie | acc_tie | round_tie)
    msg = ""
    if bad.any():
        idx = np.argwhere(bad)[:5]
        msg = "; ".join(
            f"site {tuple(i)} gpu={gpu[tuple(i)]:.7f} ora={ora[tuple(i)]:.7f} "
            f"pre={pre[tuple(i)]:.7f} dE={diag['dE'][tuple(i)]:.3e} th={diag['theta'][tuple(i)]:.3e} "
            f"R={diag['R'][tuple(i)]:.3e} acc={diag['accepted'][tuple(i)]} or={diag['or_applied'][tuple(i)]}"
            for i in idx)
    if bad_still:
        msg += f" | {bad_still} sites moved that must not"
    return int(may_move.sum()), int(explained.sum()), int(bad.sum()) + bad_still, msg


def sampled_sweep_parity(o, mask, T_of_site, pre, post, r, rng, n_sample, storage=0, t=1, tag=0):
    """One sweep of realization r (colour 0 from `pre`, colour 1 from the
    GPU's colour-0 result), recomputed by the oracle site by site at
    n_sample sampled gap sites per colour and compared with the GPU's `post`.
    Returns (checked, explained, bad, message); a mismatch is explained by a
    decision within rounding of its threshold, as in compare_site_updates."""
    import oracle
    H, W = mask.shape
    cb = checkerboard(H, W)
    gaps = np.flatnonzero(mask.ravel())
    checked = explained = bad = 0
    msgs = []
    post_f = post.ravel()
    for colour in (0, 1):
        cand = gaps[cb.ravel()[gaps] == colour]
        if cand.size == 0:
            continue
        sample = rng.choice(cand, size=min(n_sample, cand.size), replace=False)
        base = pre if colour == 0 else np.where(cb == 0, post, pre)
        ph = base.astype(np.float64).ravel()
        for i in sample:
            d = o.update_site(ph, mask, int(i), float(T_of_site(int(i))), t, tag, r)
            g = float(post_f[i])
            tol = ATOL + RTOL_PSI / max(d.R, 1e-6)
            checked += 1
            if abs(g - ph[i]) <= tol:
                continue
            fin = np.isfinite(d.phi_or)
            tie = abs(d.dE - d.theta) < TIE_E or (fin and (abs(d.phi_or) < TIE_PHI + tol or
                                                           abs(d.phi_or - TWO_PI) < TIE_PHI + tol))
            if storage and fin:
                tie = tie or (oracle.round_store(d.phi_or - tol, storage) !=
                              oracle.round_store(d.phi_or + tol, storage))
            if tie:
                explained += 1
            else:
                bad += 1
                msgs.append(f"site {int(i)} colour {colour} gpu={g:.7f} ora={ph[i]:.7f} "
                            f"dE={d.dE:.3e} th={d.theta:.3e} R={d.R:.3e}")
    return checked, explained, bad, "; ".join(msgs[:5])


def paired_over_seeds(run, seeds, floor_rel=1e-3):
    """run(seed) -> (AAE of the GPU run, AAE of the oracle's run) of one
    configuration and seed: both sides draw the same random numbers, so most
    seeds agree to rounding and a seed whose chains separated after a
    decision flip differs by Monte Carlo noise. Asserts that the mean paired
    difference is within 3 standard errors (plus floor_rel of the AAE, for a
    spread of zero) and returns the differences."""
    pairs = [run(s) for s in seeds]
    d = np.array([g - o for g, o in pairs])
    ref = float(np.mean([o for _, o in pairs]))
    se = float(d.std(ddof=1) / np.sqrt(len(d))) if len(d) > 1 else 0.0
    assert abs(d.mean()) <= 3.0 * se + floor_rel * ref, (d, se, ref)
    return d


# ------------------------------------------------------------ calibration --
def kpoint_brackets(et, pt, es, target, t_lo=1e-4, t_hi=2.0):
    """The oracle's k-point brackets after every iteration, rebuilt from its
    trace (mean e_b and temperature of every point, [n_iter, points, nblk])
    by the rule of the calibration: from the highest point whose mean is
    below e_s,b to the lowest point whose mean is not; the points' span when
    noise makes those cross. Returns [n_iter, 2, nblk] (lo, hi)."""
    n_iter, points, nblk = et.shape
    lo = np.full(nblk, float(t_lo))
    hi = np.full(nblk, float(t_hi))
    out = np.zeros((n_iter, 2, nblk))
    for k in range(n_iter):
        nlo, nhi = lo.copy(), hi.copy()
        for p in range(points):
            below = et[k, p] < es
            nlo = np.where(below & (pt[k, p] > nlo), pt[k, p], nlo)
            nhi = np.where(~below & (pt[k, p] < nhi), pt[k, p], nhi)
        cross = nlo > nhi
        nlo = np.where(cross, pt[k, 0], nlo)
        nhi = np.where(cross, pt[k, points - 1], nhi)
        lo = np.where(target, nlo, lo)
        hi = np.where(target, nhi, hi)
        out[k, 0], out[k, 1] = lo, hi
    return out


def explain_calibration(o, phi0, mask, st, T_gpu, T_ora, et, pt, n_meas, chains, target,
                        rtol=1e-4, n_sigma=8.0, max_parted=0.25):
    """Every targeted block of a k-point calibration (any number of points,
    warm or cold) is checked: either the GPU's T agrees with the oracle's
    (both run the same chains on the same random streams), or it left the
    oracle's brackets at an iteration k* where one of the oracle's points
    measured a mean e_b within n_sigma standard errors of e_s,b: there a
    comparison can come out either way between FP32 and FP64 chains. (Where
    the GPU's T stays inside every oracle bracket, its bracket contains the
    oracle's: it kept the points' span after a crossing the oracle did not
    see; k* is then the iteration and point nearest a tie.) The
    standard error is that of an uncorrelated mean over the n_meas measured
    sweeps of the chains (from the oracle's energy variance at that point's
    temperature); successive sweeps are correlated over a few sweeps, so
    8 of them are about 3.5 standard errors of the correlated mean. Returns
    the parted blocks [(b, k*, point)]."""
    es = st.es
    br = kpoint_brackets(et, pt, es, target)
    mid = 0.5 * (br[-1, 0] + br[-1, 1])
    np.testing.assert_allclose(np.where(target, mid, T_ora), T_ora, rtol=1e-12)
    parted = []
    for b in np.flatnonzero(target):
        if abs(T_gpu[b] - T_ora[b]) <= rtol * T_ora[b]:
            continue
        tol = 1e-6 * float(T_gpu[b])
        inside = (br[:, 0, b] - tol <= T_gpu[b]) & (T_gpu[b] <= br[:, 1, b] + tol)
        ks = np.flatnonzero(~inside)
        if ks.size:
            k = int(ks[0])
            j = int(np.argmin(np.abs(et[k, :, b] - es[b])))
        else:
            # The GPU's bracket contains the oracle's: with several points the
            # GPU kept the points' span where its means crossed and the
            # oracle's did not. The decision nearest a tie is the one to check.
            near = np.abs(et[:, :, b] - es[b])
            k, j = (int(v) for v in np.unravel_index(np.argmin(near), near.shape))
        parted.append((int(b), k, j))
    if parted:
        Tk = np.ascontiguousarray(T_ora, dtype=np.float64).copy()
        for b, k, j in parted:
            Tk[b] = pt[k, j, b]
        _, var_E, _, _ = o.energy_moments(np.ascontiguousarray(phi0[None].copy()), mask, Tk,
                                          200, 400, 7, st)
        for b, k, j in parted:
            se = np.sqrt(var_E[b] / (n_meas * chains)) / st.Nb[b]
            assert abs(et[k, j, b] - es[b]) <= n_sigma * se, (b, k, j, et[k, j, b], es[b], se)
    assert len(parted) <= max(1, int(max_parted * target.sum())), parted
    return parted
