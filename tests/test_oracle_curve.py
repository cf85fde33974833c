"""Pins of the oracle's unconditional e(T) curve and of the calibration's
warm start from it (Sec. 2.1 energy matching on a data-free lattice).

The curve is pinned to what the mathematics fixes, not to itself:
  * T -> infinity: every proposal is accepted and the reflection preserves the
    uniform law, so after one sweep the angles are independent and uniform on
    [0, 2 pi]; a bond's mean energy is -J E[cos(q (a - b))] = -J (sin(q pi) /
    (q pi))^2 (= -4 / pi^2 at q = 1/2), and the sweep's bond mean has the
    variance (N_b v + 2 n_adj c) / N_b^2, with v the variance of one bond
    term and c the covariance of two bonds that share a site.
  * high T, first order in beta: <H>_beta = <H>_0 - beta Var_0(H) + O(beta^2).
  * low T, harmonic limit: -cos(q x) = -1 + q^2 x^2 / 2 + O(x^4); the
    L^2 - 1 non-zero modes (one mode, the uniform shift, costs nothing) hold
    T / 2 each, so e = -1 + (L + 1) T / (4 L) + O(T^2), whatever q and J.
The curve's inverse and the warm start's first-iteration points are pinned
to their definitions on constructed curves, and the warm-started calibration
to the exact energy matching of isolated gaps (quadrature), also when the
warm guess is wrong, and so is the calibration whose chains continue from one
iteration to the next.
"""
import math

import numpy as np
import pytest

import oracle

from test_oracle_mc import _isolated_block_energy_fn


def _bond_moments(q):
    """Mean, variance of cos(q (a - b)) and covariance of cos(q (a - b)) with
    cos(q (b - c)) for independent uniform a, b, c on [0, 2 pi]."""
    m1 = (math.sin(q * math.pi) / (q * math.pi)) ** 2          # |E e^{i q a}|^2
    m2 = 0.5 + 0.5 * (math.sin(2 * q * math.pi) / (2 * q * math.pi)) ** 2
    # E_a cos(q (a - b)) = Re(E[e^{i q a}] e^{-i q b}); then average the product over b
    n = 200000
    b = (np.arange(n) + 0.5) * (2 * math.pi / n)
    ea = np.sin(q * math.pi) / (q * math.pi) * np.cos(q * (math.pi - b))
    ec = np.sin(q * math.pi) / (q * math.pi) * np.cos(q * (b - math.pi))
    cov = float(np.mean(ea * ec)) - m1 * m1
    return m1, m2 - m1 * m1, cov


def _lattice_counts(L):
    n_b = 2 * L * (L - 1)
    n_adj = 4 * 1 + 4 * (L - 2) * 3 + (L - 2) ** 2 * 6     # pairs of bonds sharing a site
    return n_b, n_adj


def test_bond_moments_at_half():
    m1, v, c = _bond_moments(0.5)
    assert m1 == pytest.approx(4 / math.pi ** 2, rel=1e-12)
    assert v == pytest.approx(0.5 - 16 / math.pi ** 4, rel=1e-12)
    assert c == pytest.approx(2 / math.pi ** 2 - 16 / math.pi ** 4, rel=1e-6)


@pytest.mark.parametrize("q", [0.5, 0.3])
def test_infinite_temperature_limit(q):
    L, n_meas = 32, 8000
    e = oracle.energy_curve([1e12], L=L, n_eq=2, n_meas=n_meas, seed=11, q=q)[0]
    m1, v, c = _bond_moments(q)
    n_b, n_adj = _lattice_counts(L)
    sigma = math.sqrt((n_b * v + 2 * n_adj * c) / n_meas) / n_b
    assert abs(e - (-m1)) < 4 * sigma, (e, -m1, sigma)


def test_first_order_in_beta():
    L, n_meas, T = 32, 8000, 100.0
    e = oracle.energy_curve([T], L=L, n_eq=5, n_meas=n_meas, seed=12)[0]
    m1, v, c = _bond_moments(0.5)
    n_b, n_adj = _lattice_counts(L)
    var_h = n_b * v + 2 * n_adj * c
    pred = -m1 - (1.0 / T) * var_h / n_b
    sigma = math.sqrt(var_h / n_meas) / n_b
    # the first-order term (0.0056) is ~30 sigma; the beta^2 term is ~1e-5
    assert abs(e - pred) < 4 * sigma + 2e-5, (e, pred, sigma)
    assert abs(e - (-m1)) > 10 * sigma


@pytest.mark.parametrize("T,J", [(0.01, 1.0), (0.02, 1.0), (0.02, 2.0)])
def test_low_temperature_equipartition(T, J):
    L = 16
    e = oracle.energy_curve([T], L=L, n_eq=1000, n_meas=4000, seed=5, J=J)[0]
    pred = -J + (L + 1) * T / (4 * L)
    assert abs(e - pred) < 0.03 * (pred + J), (e, pred)


def test_curve_is_increasing_and_in_range():
    T = np.geomspace(0.002, 1.25, 12)
    e = oracle.energy_curve(T, L=32, n_eq=25, n_meas=20, seed=3)
    assert np.all(np.diff(e) > -2e-3)
    assert e[0] > -1.0 and e[-1] < -4 / math.pi ** 2


def test_curve_inverse_definition():
    T = np.array([0.1, 0.2, 0.4, 0.8])
    e = np.array([-0.9, -0.8, -0.6, -0.5])
    assert oracle.curve_T0(T, e, -0.7) == pytest.approx(0.3, rel=1e-15)
    assert oracle.curve_T0(T, e, -0.8) == pytest.approx(0.2, rel=1e-15)
    assert oracle.curve_T0(T, e, -0.95) == 0.1          # clamped below
    assert oracle.curve_T0(T, e, -0.9) == 0.1
    assert oracle.curve_T0(T, e, -0.1) == 0.8           # clamped above
    # a point that noise pushed below its predecessor is raised to it
    e2 = np.array([-0.9, -0.7, -0.75, -0.5])
    assert oracle.curve_T0(T, e2, -0.72) == pytest.approx(0.1 + 0.1 * 0.9, rel=1e-15)
    assert oracle.curve_T0(T, e2, -0.6) == pytest.approx(0.4 + 0.4 * 0.5, rel=1e-15)


def _isolated_problem():
    rng = np.random.default_rng(12)
    H, W, lb = 16, 16, 8
    yy, xx = np.mgrid[0:H, 0:W]
    z = np.sin(yy / 3.0) + np.cos(xx / 2.5) + rng.normal(0, 0.15 + 0.25 * (xx >= 8), (H, W))
    mask = (((yy + xx) % 2 == 0) & (rng.uniform(size=(H, W)) < 0.5)).astype(np.uint8)
    o = oracle.Oracle(H, W, lb, seed=3)
    phi, *_ = o.transform(z.astype(np.float32), mask)
    st = o.block_stats(phi, mask)
    return o, phi, mask, st


def _exact_roots(o, phi, mask, st):
    fn = _isolated_block_energy_fn(phi, mask, o.lb, o.nbx)
    lo, hi = np.full(o.nblk, 1e-4), np.full(o.nblk, 2.0)
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        E = fn(mid)
        e = np.array([E.get(b, 0.0) for b in range(o.nblk)]) / st.Nb
        lo = np.where(e < st.es, mid, lo)
        hi = np.where(e < st.es, hi, mid)
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("points", [2, 4])
def test_warm_first_iteration_brackets(points):
    """After the warm first iteration every block's bracket is [t_lo, first
    point], the span between two neighbouring points, or [last point, t_hi],
    with the points evenly spaced on [T0 / w, T0 w]; the side is the one
    where the exact <e_b>(T) crosses e_s,b, unless the measured means lay
    within Monte Carlo error of it."""
    o, phi, mask, st = _isolated_problem()
    exact = _exact_roots(o, phi, mask, st)
    phi0 = o.init_block_mean(phi, mask, st)
    w = 1.5
    for scale in (0.3, 1.1, 4.0):
        T0 = exact * scale
        T = o.calibrate_points(phi0, mask, st, n_eq=20, n_meas=40, n_iter=1, chains=8,
                               points=points, T0_warm=T0, warm=w)
        for b in range(o.nblk):
            a, c = T0[b] / w, T0[b] * w
            pts = a + np.arange(points) * (c - a) / (points - 1)
            edges = np.concatenate([[1e-4], pts, [2.0]])
            mids = 0.5 * (edges[:-1] + edges[1:])
            j = int(np.argmin(np.abs(mids - T[b])))
            assert abs(mids[j] - T[b]) <= 1e-12 * T[b], (b, T[b], mids)
            # the exact root's interval, or a neighbour of it (noise at a point near the root)
            k = int(np.searchsorted(edges, exact[b])) - 1
            assert abs(j - k) <= 1, (b, j, k, exact[b], edges)


def test_warm_calibration_matches_exact_energy_matching():
    """Warm-started trisection lands near the exact root as the cold one does,
    for a good guess and for guesses whose first bracket misses the root on
    either side."""
    o, phi, mask, st = _isolated_problem()
    exact = _exact_roots(o, phi, mask, st)
    phi0 = o.init_block_mean(phi, mask, st)
    cold = o.calibrate_points(phi0, mask, st, n_eq=20, n_meas=40, n_iter=16, chains=8, points=2)
    err_cold = np.abs(cold - exact) / exact
    for scale in (1.1, 0.3, 4.0):
        T = o.calibrate_points(phi0, mask, st, n_eq=20, n_meas=40, n_iter=16, chains=8,
                               points=2, T0_warm=exact * scale, warm=1.5)
        assert np.all(np.abs(T - exact) < 0.25 * exact + 5e-3), (scale, T, exact)
        err = np.abs(T - exact) / exact
        assert err.mean() < 2 * err_cold.mean() + 0.02


def test_warm_start_from_the_curve_runs_end_to_end():
    """T0 from the oracle's own curve, the warm start, and the median fill."""
    from paper_2212_01317_gb300 import synth
    z, m = synth.small_problem(40, 48, 0.5, seed=8, kind="disc")
    o = oracle.Oracle(40, 48, 8, seed=21)
    phi, *_ = o.transform(z, m)
    st = o.block_stats(phi, m)
    Tc = np.geomspace(0.002, 1.25, 40)
    ec = oracle.energy_curve(Tc, L=64, n_eq=6, n_meas=6, seed=21)
    T0 = o.warm_T0(st, Tc, ec)
    tgt = st.Nsp > 0
    assert np.all((T0[tgt] >= Tc[0]) & (T0[tgt] <= Tc[-1]))
    phi0 = o.init_block_mean(phi, m, st)
    T = o.calibrate_points(phi0, m, st, n_eq=6, n_meas=6, n_iter=6, points=2, T0_warm=T0,
                           warm=1.5)
    assert np.all((T > 1e-4) & (T < 2.0))
    med = oracle.Oracle.median_targeted(T, np.where(st.n_gap > 0, st.Nsp, 0))
    assert np.all(T[~tgt] == med)


@pytest.mark.parametrize("n_eq_next", [0, 5])
def test_continued_chains_match_exact_energy_matching(n_eq_next):
    """Chains that continue from one calibration iteration to the next (only
    the first restarts from the initial state) land on the exact root of the
    isolated-gap energy matching as the restarting ones do, cold and warm."""
    o, phi, mask, st = _isolated_problem()
    exact = _exact_roots(o, phi, mask, st)
    phi0 = o.init_block_mean(phi, mask, st)
    for T0 in (None, exact * 1.1):
        T = o.calibrate_points(phi0, mask, st, n_eq=20, n_meas=40, n_iter=16, chains=8,
                               points=2, T0_warm=T0, warm=1.5, n_eq_next=n_eq_next)
        assert np.all(np.abs(T - exact) < 0.25 * exact + 5e-3), (T, exact)


def test_continued_chains_restart_only_once():
    """One iteration is the same with or without continuation (the first
    iteration always restarts); later iterations start where the earlier ones
    stopped, so their measured energies differ from restarted chains'."""
    o, phi, mask, st = _isolated_problem()
    phi0 = o.init_block_mean(phi, mask, st)
    a = o.calibrate_points(phi0, mask, st, n_eq=5, n_meas=5, n_iter=1, points=2)
    b = o.calibrate_points(phi0, mask, st, n_eq=5, n_meas=5, n_iter=1, points=2, n_eq_next=0)
    np.testing.assert_array_equal(a, b)
    _, et_r, pt_r = o.calibrate_points(phi0, mask, st, n_eq=5, n_meas=5, n_iter=3, points=2,
                                       trace=True)
    _, et_c, pt_c = o.calibrate_points(phi0, mask, st, n_eq=5, n_meas=5, n_iter=3, points=2,
                                       n_eq_next=5, trace=True)
    np.testing.assert_array_equal(et_r[0], et_c[0])      # the first iteration restarts
    assert not np.array_equal(et_r[1:], et_c[1:])        # later ones continue
