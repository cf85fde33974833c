"""Pins of the oracle's sampling variant of the conditional mean (Sec. 2.1
predicts with the mean of the conditional distribution; the variant takes it
from one chain's successive states after an equilibration instead of from
independent realizations each stopped at local equilibrium).

  * isolated gaps (every gap's neighbours are data): the conditional law of
    each gap is known by quadrature, so the chains' sample means must land on
    the exact conditional means within the spread over independent chains;
  * the sums are the states after sweeps n_equil + 1 .. n_equil + n_samples,
    nothing else: checked against the half-steps run one by one, and data
    sites never contribute.
"""
import numpy as np

import oracle

from test_oracle_mc import TWO_PI, isolated_gap_law, neighbours


def _isolated(seed=31):
    rng = np.random.default_rng(seed)
    H, W = 6, 7
    gaps = [(0, 0), (0, 2), (1, 1), (1, 3), (2, 4), (3, 3), (4, 2), (5, 5)]
    mask = np.zeros((H, W), np.uint8)
    for (y, x) in gaps:
        mask[y, x] = 1
    phi = rng.uniform(0, TWO_PI, (H, W))
    return H, W, gaps, mask, phi


def test_sample_means_match_the_exact_conditional_means():
    H, W, gaps, mask, phi = _isolated()
    T = 0.3
    o = oracle.Oracle(H, W, 7, seed=43)
    n_chains, n_equil, n_samples = 16, 20, 2500
    means = np.zeros((n_chains, len(gaps)))
    Tb = np.full(o.nblk, T)
    for r in range(n_chains):
        s = o.sample_chain(phi.ravel(), mask, Tb, n_equil, n_samples, r)
        means[r] = [s[y * W + x] / n_samples for (y, x) in gaps]
    for g, (y, x) in enumerate(gaps):
        nodes, p = isolated_gap_law([phi[a, b] for (a, b) in neighbours(H, W, y, x)], T)
        exact = (p * nodes).sum()
        m = means[:, g].mean()
        se = means[:, g].std(ddof=1) / np.sqrt(n_chains)
        assert abs(m - exact) < 4 * se + 1e-3, (g, m, exact, se)


def test_sample_sums_are_the_states_after_the_equilibration():
    H, W, gaps, mask, phi = _isolated(seed=5)
    mask[3, 4] = 1                          # a gap next to a gap
    o = oracle.Oracle(H, W, 4, seed=7)
    Tb = np.linspace(0.05, 0.6, o.nblk)
    n_equil, n_samples, r = 3, 4, 5
    s = o.sample_chain(phi.ravel(), mask, Tb, n_equil, n_samples, r)
    ph = phi.ravel().copy()
    want = np.zeros(H * W)
    for t in range(1, n_equil + n_samples + 1):
        o.halfstep(ph, mask, 0, Tb, t=t, tag=0, r=r)
        o.halfstep(ph, mask, 1, Tb, t=t, tag=0, r=r)
        if t > n_equil:
            want += np.where(mask.ravel() != 0, ph, 0.0)
    np.testing.assert_array_equal(s, want)
    assert np.all(s[mask.ravel() == 0] == 0.0)
    # sums accumulate into a given array
    acc = np.full(H * W, 1.0)
    o.sample_chain(phi.ravel(), mask, Tb, n_equil, n_samples, r, sum_out=acc)
    np.testing.assert_array_equal(acc, want + 1.0)
