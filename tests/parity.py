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


def compare_site_updates(gpu, ora, pre, diag, may_move):
    """Returns (n_sites_checked, n_explained_flips, n_bad, message)."""
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
    explained = may_move & ~ok & (or_tie | acc_tie)
    bad = may_move & ~ok & ~(or_tie | acc_tie)
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
