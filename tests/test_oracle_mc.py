"""Pins for the oracle's conditional Monte Carlo (Sec. 2.1, Sec. 2.2.2).

Each test compares the oracle's chain with something computed without it:
  * dE of one update against the brute-force change of Eq. 1;
  * discretised angles, one T: exact enumeration of the conditional
    Boltzmann distribution exp(-H/T) over the gap configurations;
  * discretised angles, block-varying T: the stationary vector of the exact
    one-sweep transition matrix (colour 0 then colour 1), which has no Gibbs
    form;
  * continuous angles with and without over-relaxation, gaps isolated by
    data: per-gap conditional density exp(J/T sum_j cos q(phi - phi_j)) on
    [0, 2pi] integrated by composite Gauss-Legendre quadrature;
  * calibration in the isolated-gap setting: <e_b>(T) is exact by quadrature,
    so the temperature that matches e_s,b is known without simulation.
Monte Carlo errors come from batch means; bounds are 4 sigma.
"""
import numpy as np
import pytest

import oracle

PI = np.pi
TWO_PI = 2 * np.pi


def brute_energy(phi, q=0.5, J=1.0):
    return (-J * np.cos(q * (phi[:, :-1] - phi[:, 1:]))).sum() + \
           (-J * np.cos(q * (phi[:-1, :] - phi[1:, :]))).sum()


def batch_mean_se(x, nb=40):
    x = np.asarray(x, dtype=np.float64)
    n = (len(x) // nb) * nb
    m = x[:n].reshape(nb, -1).mean(axis=1)
    return x.mean(), m.std(ddof=1) / np.sqrt(nb)


def neighbours(H, W, y, x):
    out = []
    if x > 0: out.append((y, x - 1))
    if x + 1 < W: out.append((y, x + 1))
    if y > 0: out.append((y - 1, x))
    if y + 1 < H: out.append((y + 1, x))
    return out


def run_chain(o, phi0, mask, T_blk, n_sweeps, sites, tag=0, r=0):
    phi = np.ascontiguousarray(phi0, dtype=np.float64).copy()
    rec = np.zeros((n_sweeps, len(sites)))
    en = np.zeros(n_sweeps)
    idx = [y * phi.shape[1] + x for (y, x) in sites]
    flat = phi.reshape(-1)
    for t in range(1, n_sweeps + 1):
        o.halfstep(phi, mask, 0, T_blk, t=t, tag=tag, r=r)
        o.halfstep(phi, mask, 1, T_blk, t=t, tag=tag, r=r)
        rec[t - 1] = flat[idx]
        en[t - 1] = o.total_energy(phi)
    return rec, en, phi


# --------------------------------------------------------------------------- dE
@pytest.mark.parametrize("overrelax", [False, True])
def test_update_dE_matches_hamiltonian_change(overrelax):
    rng = np.random.default_rng(11)
    H, W = 7, 6
    phi = rng.uniform(0, TWO_PI, (H, W))
    mask = np.ones((H, W), np.uint8)
    o = oracle.Oracle(H, W, 3, seed=7, overrelax=overrelax)
    n_acc = n_or = 0
    for trial in range(200):
        y, x = rng.integers(0, H), rng.integers(0, W)
        i = int(y * W + x)
        before = brute_energy(phi)
        T = float(rng.choice([0.05, 0.3, 2.0]))
        d = o.update_site(phi.reshape(-1), mask, i, T, trial + 1, 0, trial % 5)
        after = brute_energy(phi)
        expect = d.dE if d.accepted else 0.0
        assert abs((after - before) - expect) < 1e-10
        assert 0.0 <= phi[y, x] <= TWO_PI
        assert d.accepted == (d.dE < d.theta) or abs(d.dE - d.theta) < 1e-12
        n_acc += d.accepted
        n_or += d.or_applied
    assert 0 < n_acc < 200
    if overrelax:
        assert n_or > 20
    else:
        assert n_or == 0


def test_halfstep_touches_only_gaps_of_its_colour_in_active_blocks():
    rng = np.random.default_rng(3)
    H, W, lb = 12, 10, 4
    phi = rng.uniform(0, TWO_PI, (H, W))
    mask = (rng.uniform(size=(H, W)) < 0.6).astype(np.uint8)
    o = oracle.Oracle(H, W, lb, seed=1)
    T = np.full(o.nblk, 0.5)
    active = (rng.uniform(size=o.nblk) < 0.5).astype(np.uint8)
    blk = o.block_index()
    for colour in (0, 1):
        new = phi.copy()
        o.halfstep(new, mask, colour, T, active, t=3)
        yy, xx = np.mgrid[0:H, 0:W]
        may = (mask == 1) & (((yy + xx) & 1) == colour) & (active[blk] == 1)
        assert np.array_equal(new[~may], phi[~may])
        assert np.count_nonzero(new[may] != phi[may]) > 0.5 * may.sum()


# ------------------------------------------------------------ exact enumeration
def _exact_discrete(phi_data, mask, K, T_of_site, q=0.5):
    """Exact stationary law of the discretised chain over the gap sites.

    T_of_site is None for the single-T Gibbs case (returns the Boltzmann law),
    else a dict site -> T and the stationary vector of the sweep matrix is
    returned."""
    H, W = mask.shape
    gaps = [(y, x) for y in range(H) for x in range(W) if mask[y, x]]
    n = len(gaps)
    levels = TWO_PI * np.arange(K) / K
    states = np.array(np.unravel_index(np.arange(K ** n), (K,) * n)).T  # [S, n]

    def energy(st):
        phi = phi_data.copy()
        for g, (y, x) in enumerate(gaps):
            phi[y, x] = levels[st[g]]
        return brute_energy(phi, q)

    E = np.array([energy(s) for s in states])
    return gaps, states, levels, E


def test_discrete_single_T_matches_boltzmann_enumeration():
    rng = np.random.default_rng(21)
    H, W, K, T = 3, 3, 8, 0.7
    mask = np.zeros((H, W), np.uint8)
    for (y, x) in [(0, 1), (1, 1), (1, 2), (2, 0)]:
        mask[y, x] = 1
    phi_data = rng.uniform(0, TWO_PI, (H, W))
    gaps, states, levels, E = _exact_discrete(phi_data, mask, K, None)
    w = np.exp(-(E - E.min()) / T)
    w /= w.sum()
    exact_phi = np.array([(w * levels[states[:, g]]).sum() for g in range(len(gaps))])
    exact_E = (w * E).sum()

    o = oracle.Oracle(H, W, 3, seed=5, overrelax=False, K=K)
    phi0 = phi_data.copy()
    for (y, x) in gaps:
        phi0[y, x] = 0.0
    rec, en, _ = run_chain(o, phi0, mask, np.full(o.nblk, T), 60000, gaps)
    rec, en = rec[1000:], en[1000:]
    for g in range(len(gaps)):
        m, se = batch_mean_se(rec[:, g])
        assert abs(m - exact_phi[g]) < 4 * se + 1e-3, (g, m, exact_phi[g], se)
    m, se = batch_mean_se(en)
    assert abs(m - exact_E) < 4 * se + 1e-3, (m, exact_E, se)


def test_discrete_block_T_matches_sweep_transition_matrix():
    rng = np.random.default_rng(8)
    H, W, K, lb = 2, 4, 6, 2
    mask = np.zeros((H, W), np.uint8)
    mask[:, 1:3] = 1                       # gaps (0,1) c1, (0,2) c0, (1,1) c0, (1,2) c1
    phi_data = rng.uniform(0, TWO_PI, (H, W))
    T_blk = np.array([0.15, 1.5])          # block 0: cols 0-1, block 1: cols 2-3
    gaps, states, levels, E = _exact_discrete(phi_data, mask, K, True)
    n = len(gaps)
    S = len(states)
    mult = K ** np.arange(n - 1, -1, -1)

    def site_kernel(g):
        y, x = gaps[g]
        T = T_blk[(y // lb) * 2 + x // lb]
        P = np.zeros((S, S))
        for s in range(S):
            for k in range(K):
                s2 = s + (k - states[s, g]) * mult[g]
                a = min(1.0, np.exp(-(E[s2] - E[s]) / T))
                P[s, s2] += a / K
                P[s, s] += (1 - a) / K
        return P

    def stationary(order):
        P = np.eye(S)
        for colour in order:
            for g, (y, x) in enumerate(gaps):
                if (y + x) & 1 == colour:
                    P = P @ site_kernel(g)
        pi = np.full(S, 1.0 / S)
        for _ in range(5000):
            pi = pi @ P
        return pi

    # Observables: each gap's angle and cos(phi_a - phi_b) of every gap-gap bond
    # (the single-site marginals do not see the colour order; bond correlations do).
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)
             if abs(gaps[a][0] - gaps[b][0]) + abs(gaps[a][1] - gaps[b][1]) == 1]
    assert len(pairs) == 4

    def observables(ang):           # ang [..., n]
        cols = [ang[..., g] for g in range(n)]
        cols += [np.cos(ang[..., a] - ang[..., b]) for (a, b) in pairs]
        return np.stack(cols, axis=-1)

    obs_states = observables(levels[states])
    exact = stationary((0, 1)) @ obs_states
    rev = stationary((1, 0)) @ obs_states

    o = oracle.Oracle(H, W, lb, seed=17, overrelax=False, K=K)
    phi0 = phi_data.copy()
    for (y, x) in gaps:
        phi0[y, x] = 0.0
    rec, _, _ = run_chain(o, phi0, mask, T_blk, 80000, gaps)
    obs = observables(rec[500:])
    ses = []
    for j in range(obs.shape[1]):
        m, se = batch_mean_se(obs[:, j])
        assert abs(m - exact[j]) < 4 * se + 1e-3, (j, m, exact[j], se)
        ses.append(se)
    # The reversed colour order has a different stationary law, and the
    # estimates are precise enough to tell the two apart.
    assert np.max(np.abs(rev - exact) / np.array(ses)) > 10


# -------------------------------------------------------- continuous quadrature
def _gl_nodes(panels=400, order=16):
    x, w = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(0, TWO_PI, panels + 1)
    a, b = edges[:-1, None], edges[1:, None]
    nodes = (0.5 * (b - a) * x[None, :] + 0.5 * (a + b)).ravel()
    weights = (0.5 * (b - a) * w[None, :]).ravel()
    return nodes, weights


def isolated_gap_law(nb_angles, T, q=0.5, J=1.0):
    """Normalised weights of the conditional density of one gap on the GL nodes."""
    nodes, weights = _gl_nodes()
    e = np.zeros_like(nodes)
    for pj in nb_angles:
        e += -J * np.cos(q * (nodes - pj))
    lw = -e / T
    dens = np.exp(lw - lw.max()) * weights
    return nodes, dens / dens.sum()


@pytest.mark.parametrize("overrelax", [False, True])
def test_continuous_isolated_gaps_match_quadrature(overrelax):
    rng = np.random.default_rng(31)
    H, W, T = 6, 7, 0.3
    gaps = [(0, 0), (0, 2), (1, 1), (1, 3), (2, 4), (3, 3), (4, 2), (5, 5)]
    mask = np.zeros((H, W), np.uint8)
    for (y, x) in gaps:
        assert (y + x) % 2 == 0
        mask[y, x] = 1
    phi = rng.uniform(0, TWO_PI, (H, W))
    o = oracle.Oracle(H, W, 7, seed=41, overrelax=overrelax)
    rec, _, _ = run_chain(o, phi, mask, np.full(o.nblk, T), 40000, gaps)
    rec = rec[200:]
    for g, (y, x) in enumerate(gaps):
        nodes, p = isolated_gap_law([phi[a, b] for (a, b) in neighbours(H, W, y, x)], T)
        mean = (p * nodes).sum()
        m, se = batch_mean_se(rec[:, g])
        assert abs(m - mean) < 4 * se + 1e-3, (g, m, mean, se)
        # second moment too
        m2, se2 = batch_mean_se(rec[:, g] ** 2)
        assert abs(m2 - (p * nodes ** 2).sum()) < 4 * se2 + 1e-3
    assert rec.min() >= 0.0 and rec.max() <= TWO_PI


# ------------------------------------------------------------------ calibration
def _isolated_block_energy_fn(phi, mask, lb, nbx, q=0.5, J=1.0):
    """Exact <E_b>(T) for gaps isolated by data: each gap contributes the
    expectation of its bonds under its own conditional density."""
    H, W = mask.shape

    def owner(y1, x1, y2, x2):
        oy, ox = min((y1, x1), (y2, x2))
        return (oy // lb) * nbx + ox // lb

    const = {}
    gap_terms = []   # (gap site, list of (block, partner angle))
    for y in range(H):
        for x in range(W):
            for (y2, x2) in ((y, x + 1), (y + 1, x)):
                if y2 >= H or x2 >= W:
                    continue
                b = owner(y, x, y2, x2)
                if not mask[y, x] and not mask[y2, x2]:
                    const[b] = const.get(b, 0.0) - J * np.cos(q * (phi[y, x] - phi[y2, x2]))
    for y in range(H):
        for x in range(W):
            if not mask[y, x]:
                continue
            terms = [(owner(y, x, a, c), phi[a, c]) for (a, c) in neighbours(H, W, y, x)]
            gap_terms.append(((y, x), terms))

    def fn(T_blk):
        T_of = lambda y, x: T_blk[(y // lb) * nbx + x // lb]
        E = dict(const)
        for (y, x), terms in gap_terms:
            nodes, p = isolated_gap_law([pa for (_, pa) in terms], T_of(y, x), q, J)
            for (b, pa) in terms:
                E[b] = E.get(b, 0.0) + (p * (-J * np.cos(q * (nodes - pa)))).sum()
        return E

    return fn


def test_calibration_matches_exact_energy_matching():
    rng = np.random.default_rng(12)
    H, W, lb = 16, 16, 8
    yy, xx = np.mgrid[0:H, 0:W]
    # Smooth data with a different roughness per block so that T_b differ.
    z = np.sin(yy / 3.0) + np.cos(xx / 2.5) + rng.normal(0, 0.15 + 0.25 * (xx >= 8), (H, W))
    mask = (((yy + xx) % 2 == 0) & (rng.uniform(size=(H, W)) < 0.5)).astype(np.uint8)
    o = oracle.Oracle(H, W, lb, seed=3)
    phi, zmin, zmax, _ = o.transform(z.astype(np.float32), mask)
    st = o.block_stats(phi, mask)
    phi0 = o.init_block_mean(phi, mask, st)
    chains, n_meas, n_bisect = 8, 40, 16
    T = o.calibrate(phi0, mask, st, n_eq=20, n_meas=n_meas, n_bisect=n_bisect, chains=chains,
                    T_lo=1e-4, T_hi=2.0)
    fn = _isolated_block_energy_fn(phi, mask, lb, o.nbx)
    es = st.es

    # Deterministic bisection on the exact curve, all blocks at once (the
    # blocks interact only through shared bonds, which the exact curve takes
    # into account via each gap's own temperature).
    lo, hi = np.full(o.nblk, 1e-4), np.full(o.nblk, 2.0)
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        E = fn(mid)
        e = np.array([E[b] / st.Nb[b] for b in range(o.nblk)])
        below = e < es
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    T_exact = 0.5 * (lo + hi)
    E_at = fn(T)
    for b in range(o.nblk):
        e_at = E_at[b] / st.Nb[b]
        # MC error of the block energy average (gaps only move a handful of bonds).
        assert abs(e_at - es[b]) < 0.02, (b, e_at, es[b])
        assert abs(T[b] - T_exact[b]) < 0.25 * T_exact[b] + 5e-3, (b, T[b], T_exact[b])
    # The blocks were built to differ: the calibrated temperatures must too.
    assert T_exact.max() > 1.5 * T_exact.min()


def test_median_fallback_for_blocks_without_sample_bonds():
    T = np.array([0.3, 0.1, 0.9, 0.5, 7.0])
    Nsp = np.array([2, 0, 5, 1, 0])
    assert oracle.Oracle.median_targeted(T, Nsp) == pytest.approx(0.5)
    Nsp = np.array([2, 3, 5, 1, 0])
    assert oracle.Oracle.median_targeted(T, Nsp) == pytest.approx(0.4)


# ------------------------------------------------------------------------- stop
def _stop_problem(seed=4):
    rng = np.random.default_rng(seed)
    H, W, lb = 20, 24, 4
    yy, xx = np.mgrid[0:H, 0:W]
    z = np.sin(yy / 4.0) * np.cos(xx / 5.0) + rng.normal(0, 0.2, (H, W))
    mask = (rng.uniform(size=(H, W)) < 0.45).astype(np.uint8)
    mask[0:4, 0:4] = 1        # block 0: all gaps -> no sample bonds (untargeted)
    mask[4:8, 8:12] = 0       # a block with no gaps
    return z.astype(np.float32), mask, lb


def test_stop_rule_against_energy_trace():
    z, mask, lb = _stop_problem()
    H, W = mask.shape
    o = oracle.Oracle(H, W, lb, seed=9)
    phi, *_ = o.transform(z, mask)
    st = o.block_stats(phi, mask)
    phi0 = o.init_block_mean(phi, mask, st)
    T = np.random.default_rng(1).uniform(0.02, 0.6, o.nblk)
    n_max = 60
    _, stop, n, tr = o.simulate_one(phi0, mask, T, st, n_max, r=2, trace=True)
    es = st.es
    sigma = np.sign(es - tr[0])
    targeted = st.Nsp > 0
    has_gap = st.n_gap > 0
    assert np.all(stop[~has_gap] == 0)
    for b in np.where(targeted & has_gap)[0]:
        hit = [t for t in range(1, n + 1) if sigma[b] * (tr[t, b] - es[b]) >= 0]
        assert stop[b] == (hit[0] if hit else n_max), b
    last_targeted = stop[targeted & has_gap].max()
    for b in np.where(~targeted & has_gap)[0]:
        assert stop[b] == last_targeted
    assert n == stop.max()


def test_stopped_blocks_freeze_and_data_never_change():
    z, mask, lb = _stop_problem(seed=6)
    H, W = mask.shape
    o = oracle.Oracle(H, W, lb, seed=10)
    phi, *_ = o.transform(z, mask)
    st = o.block_stats(phi, mask)
    phi0 = o.init_block_mean(phi, mask, st)
    T = np.full(o.nblk, 0.2)
    E0 = o.block_energy(phi0)
    sigma, active, stop = o.stop_init(E0, st)
    blk = o.block_index()
    cur = phi0.copy()
    n_max = 40
    for t in range(1, n_max + 1):
        prev = cur.copy()
        was_active = active.copy()
        o.halfstep(cur, mask, 0, T, active, t=t, r=1)
        o.halfstep(cur, mask, 1, T, active, t=t, r=1)
        frozen = was_active[blk] == 0
        assert np.array_equal(cur[frozen], prev[frozen])
        assert np.array_equal(cur[mask == 0], phi0[mask == 0])
        assert cur.min() >= 0 and cur.max() <= TWO_PI
        left = o.stop_update(t, n_max, o.block_energy(cur), st, sigma, active, stop)
        if left == 0:
            break
    ph2, stop2, _, _ = o.simulate_one(phi0, mask, T, st, n_max, r=1)
    assert np.array_equal(stop, stop2)
    assert np.array_equal(cur, ph2)


def test_openmp_thread_count_is_bitwise_invisible():
    z, mask, lb = _stop_problem(seed=2)
    res = []
    for threads in (1, 4):
        r = oracle.gapfill(z, mask, lb, R=3, seed=77, n_bisect=4, n_eq=5, n_meas=5,
                           threads=threads)
        res.append(r)
    assert np.array_equal(res[0].pred.view(np.uint32), res[1].pred.view(np.uint32))
    assert np.array_equal(res[0].T, res[1].T)
    assert np.array_equal(res[0].stop_sweeps, res[1].stop_sweeps)


def test_block_mean_init_is_closer_to_equilibrium_than_random():
    """Sec. 3.3.3: starting from per-block sample averages shortens equilibration."""
    z, mask, lb = _stop_problem(seed=13)
    H, W = mask.shape
    o = oracle.Oracle(H, W, lb, seed=21)
    phi, *_ = o.transform(z, mask)
    st = o.block_stats(phi, mask)
    es_all = st.Es.sum() / st.Nsp.sum()
    e_blk = o.total_energy(o.init_block_mean(phi, mask, st)) / st.Nb.sum()
    e_rnd = np.mean([o.total_energy(o.init_random(phi, mask, r)) / st.Nb.sum()
                     for r in range(4)])
    assert abs(e_blk - es_all) < abs(e_rnd - es_all)


def test_one_point_k_section_is_the_bisection():
    from paper_2212_01317_gb300 import synth
    z, m = synth.small_problem(20, 24, 0.5, seed=6)
    o = oracle.Oracle(20, 24, 6, seed=12)
    phi, *_ = o.transform(z, m)
    st = o.block_stats(phi, m)
    phi0 = o.init_block_mean(phi, m, st)
    a = o.calibrate(phi0, m, st, n_eq=4, n_meas=4, n_bisect=7, chains=2)
    b = o.calibrate_points(phi0, m, st, n_eq=4, n_meas=4, n_iter=7, chains=2, points=1)
    np.testing.assert_array_equal(a, b)


def test_trisection_matches_exact_energy_matching():
    # Isolated gaps: <e_b>(T) is exact by quadrature; 16 trisection steps
    # narrow the bracket below the bisection's 24 steps, and the noisy
    # estimate lands near the exact root as the bisection's does.
    rng = np.random.default_rng(12)
    H, W, lb = 16, 16, 8
    yy, xx = np.mgrid[0:H, 0:W]
    z = np.sin(yy / 3.0) + np.cos(xx / 2.5) + rng.normal(0, 0.15 + 0.25 * (xx >= 8), (H, W))
    mask = (((yy + xx) % 2 == 0) & (rng.uniform(size=(H, W)) < 0.5)).astype(np.uint8)
    o = oracle.Oracle(H, W, lb, seed=3)
    phi, *_ = o.transform(z.astype(np.float32), mask)
    st = o.block_stats(phi, mask)
    phi0 = o.init_block_mean(phi, mask, st)
    T3 = o.calibrate_points(phi0, mask, st, n_eq=20, n_meas=40, n_iter=16, chains=8, points=2)
    T2 = o.calibrate(phi0, mask, st, n_eq=20, n_meas=40, n_bisect=24, chains=8)
    fn = _isolated_block_energy_fn(phi, mask, lb, o.nbx)
    lo, hi = np.full(o.nblk, 1e-4), np.full(o.nblk, 2.0)
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        E = fn(mid)
        e = np.array([E.get(b, 0.0) for b in range(o.nblk)]) / st.Nb
        lo = np.where(e < st.es, mid, lo)
        hi = np.where(e < st.es, hi, mid)
    exact = 0.5 * (lo + hi)
    # the same bounds as the bisection's pin above, and no worse than it on average
    assert np.all(np.abs(T3 - exact) < 0.25 * exact + 5e-3), (T3, exact)
    E_at = fn(T3)
    for b in range(o.nblk):
        assert abs(E_at[b] / st.Nb[b] - st.es[b]) < 0.02
    err3 = np.abs(T3 - exact) / exact
    err2 = np.abs(T2 - exact) / exact
    assert err3.mean() < 2 * err2.mean() + 0.02
