"""Pins of the oracle's energy moments and Newton calibration (the
differentiable form of the energy matching of Sec. 2.1 / 2.2.2).

Gaps isolated by samples are independent given the data, each with the 1-D
conditional density exp(-(sum of its bond energies) / T_b), so the block
energies' means, variances and covariances are exact by quadrature; for a
single block (or gaps whose bonds all belong to their own block) the
fluctuation identity d<E_b>/d beta_b = -Var(E_b) is exact, and the Newton
root is the exact root of <e_b>(T) = e_s,b.
"""
import numpy as np
import pytest

import oracle
from test_oracle_mc import TWO_PI, isolated_gap_law, neighbours


def isolated_problem(H, W, lb, seed, p=0.5, avoid_left_top_edges=False):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W]
    z = np.sin(yy / 2.7) + np.cos(xx / 3.1) + rng.normal(0, 0.3, (H, W))
    ok = ((yy + xx) % 2 == 0) & (rng.uniform(size=(H, W)) < p)
    if avoid_left_top_edges:
        ok &= (xx % lb != 0) & (yy % lb != 0)
    mask = ok.astype(np.uint8)
    o = oracle.Oracle(H, W, lb, seed=seed)
    phi, _, _, _ = o.transform(z.astype(np.float32), mask)
    return o, z, mask, phi


def exact_moments(o, phi, mask, T_blk, q=0.5, J=1.0):
    """Exact <E_b>, Var(E_b), Cov(E_b, E_right), Cov(E_b, E_down) of gaps isolated by
    samples; every gap at the temperature of its own block."""
    H, W, lb, nbx, nblk = o.H, o.W, o.lb, o.nbx, o.nblk

    def owner(y1, x1, y2, x2):
        oy, ox = min((y1, x1), (y2, x2))
        return (oy // lb) * nbx + ox // lb

    mean = np.zeros(nblk)
    cov = np.zeros((nblk, nblk))
    for y in range(H):
        for x in range(W):
            for (y2, x2) in ((y, x + 1), (y + 1, x)):
                if y2 < H and x2 < W and not mask[y, x] and not mask[y2, x2]:
                    mean[owner(y, x, y2, x2)] += -J * np.cos(q * (phi[y, x] - phi[y2, x2]))
    for y in range(H):
        for x in range(W):
            if not mask[y, x]:
                continue
            nb = neighbours(H, W, y, x)
            nodes, p = isolated_gap_law([phi[a, c] for (a, c) in nb], T_blk[(y // lb) * nbx + x // lb],
                                        q, J)
            f = np.zeros((nblk, nodes.size))          # this gap's energy in every block
            for (a, c) in nb:
                f[owner(y, x, a, c)] += -J * np.cos(q * (nodes - phi[a, c]))
            m = f @ p
            mean += m
            d = f - m[:, None]
            cov += (d * p) @ d.T
    right = np.array([cov[b, b + 1] if b % nbx != nbx - 1 else 0.0 for b in range(nblk)])
    down = np.array([cov[b, b + nbx] if b + nbx < nblk else 0.0 for b in range(nblk)])
    return mean, np.diag(cov).copy(), right, down


def batches(o, phi0, mask, T, st, n_batches=8, chains=8, n_eq=10, n_meas=150):
    out = []
    for k in range(n_batches):
        ph = np.repeat(phi0[None], chains, axis=0).copy()
        out.append(o.energy_moments(ph, mask, T, n_eq, n_meas, tag=1 + k, st=st))
    return [np.array([b[i] for b in out]) for i in range(4)]


def test_single_block_moments_match_quadrature():
    o, z, mask, phi = isolated_problem(10, 10, 10, seed=1)
    st = o.block_stats(phi, mask)
    T = np.array([0.25])
    mean_e, var, _, _ = batches(o, phi, mask, T, st)
    m_ex, v_ex, _, _ = exact_moments(o, phi, mask, T)
    Nb = st.Nb[0]
    est_m = mean_e[:, 0] * Nb
    se_m = est_m.std(ddof=1) / np.sqrt(len(est_m))
    assert abs(est_m.mean() - m_ex[0]) < 4 * se_m + 1e-9
    se_v = var[:, 0].std(ddof=1) / np.sqrt(len(var))
    assert abs(var[:, 0].mean() - v_ex[0]) < 4 * se_v + 1e-3 * v_ex[0]


def test_block_covariances_match_quadrature():
    # 2 x 2 blocks; gaps on the blocks' left / top edges hand a bond to the
    # neighbouring block, which correlates the two blocks' energies.
    o, z, mask, phi = isolated_problem(12, 12, 6, seed=4, p=0.6)
    st = o.block_stats(phi, mask)
    T = np.array([0.2, 0.35, 0.3, 0.15])
    _, var, cr, cd = batches(o, phi, mask, T, st)
    _, v_ex, r_ex, d_ex = exact_moments(o, phi, mask, T)
    assert np.abs(r_ex).max() > 1e-3 and np.abs(d_ex).max() > 1e-3
    for est, ex in ((var, v_ex), (cr, r_ex), (cd, d_ex)):
        se = est.std(ddof=1, axis=0) / np.sqrt(est.shape[0])
        assert np.all(np.abs(est.mean(axis=0) - ex) < 4 * se + 1e-3 * np.abs(v_ex).max()), (est.mean(0), ex)


def test_blocks_without_shared_gaps_are_uncorrelated():
    o, z, mask, phi = isolated_problem(12, 12, 6, seed=5, p=0.6, avoid_left_top_edges=True)
    _, v_ex, r_ex, d_ex = exact_moments(o, phi, mask, np.full(4, 0.25))
    np.testing.assert_allclose(r_ex, 0.0, atol=1e-15)
    np.testing.assert_allclose(d_ex, 0.0, atol=1e-15)


def test_newton_finds_the_exact_root():
    o, z, mask, phi = isolated_problem(10, 10, 10, seed=2)
    st = o.block_stats(phi, mask)
    es = st.es[0]
    Nb = st.Nb[0]
    # Exact root of <e>(T) = e_s by bisection on the quadrature curve.
    lo, hi = 1e-4, 2.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if exact_moments(o, phi, mask, np.array([mid]))[0][0] / Nb < es:
            lo = mid
        else:
            hi = mid
    T_star = 0.5 * (lo + hi)
    phi0 = o.init_block_mean(phi, mask, st)
    T, tr = o.calibrate_newton(phi0, mask, st, n_eq=10, n_meas=60, n_newton=8, chains=64,
                               T0=0.1, trace=True)
    assert abs(T[0] - T_star) / T_star < 0.03, (T[0], T_star, tr[:, 0])
    # Newton steps converge fast: the last three iterates agree within the
    # Monte Carlo noise of one iteration's estimate. One iterate's spread is
    # sigma_T = T*^2 / sqrt(n Var(E_b)) times sqrt(tau) (the fluctuation
    # identity turns the noise of the measured mean energy into noise of T;
    # n = 64 chains x 60 sweeps; tau, the energy's autocorrelation time,
    # a few sweeps): about 0.5 % x sqrt(tau) here, so 4 % holds the range of
    # three iterates with a wide margin.
    assert np.ptp(tr[-3:, 0]) / T_star < 0.04
    # every step stays within a factor 2 of the previous temperature
    r = tr[1:, 0] / tr[:-1, 0]
    assert np.all((r >= 0.5 - 1e-12) & (r <= 2 + 1e-12))


def test_newton_median_fallback_and_bounds():
    z = np.random.default_rng(0).normal(size=(16, 16)).astype(np.float32)
    mask = np.zeros((16, 16), np.uint8)
    mask[0:8, 0:8] = 1                     # block 0: no sample bond at all
    mask[9, 9] = mask[12, 3] = mask[3, 12] = 1
    o = oracle.Oracle(16, 16, 8, seed=9)
    phi, _, _, _ = o.transform(z, mask)
    st = o.block_stats(phi, mask)
    assert st.Nsp[0] == 0 and (st.Nsp[1:] > 0).all()
    phi0 = o.init_block_mean(phi, mask, st)
    T = o.calibrate_newton(phi0, mask, st, n_eq=5, n_meas=10, n_newton=4, chains=2, T0=0.1)
    assert T[0] == np.median(T[1:])
    assert np.all((T[1:] > 1e-4) & (T[1:] < 2.0))
