"""The sampling variant of the conditional mean (mpr_sample_chains: chains
that equilibrate, then contribute their state after every further sweep)
through the C-ABI.

  * lockstep with the oracle's sample_chain on the same random streams:
    the per-site sums over chains and samples agree to FP32 rounding, for
    lane groups of two and eight and both start states;
  * on isolated gaps the chains' means land on the exact conditional means
    (quadrature), in FP32 and in BF16 state;
  * samples and realizations share the running mean; argument checks.
"""
import numpy as np
import pytest

import oracle
from paper_2212_01317_gb300 import mpr, synth
from paper_2212_01317_gb300.mpr import GapFiller, MprError, MPR_EINVAL, MPR_ESTATE

from test_oracle_mc import TWO_PI, isolated_gap_law, neighbours

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def make(z, m, lb, **opt):
    v = np.where(m != 0, np.nan, z).astype(np.float32)
    return GapFiller(v, m, lb, **opt)


@pytest.mark.parametrize("group,init", [(2, 0), (8, 0), (8, 1)])
def test_sample_sums_match_oracle(group, init):
    H, W, lb = 28, 36, 8
    z, m = synth.small_problem(H, W, 0.5, seed=group + 3 * init, kind="random")
    seed = 0xABC0 + group
    gf = make(z, m, lb, seed=seed, group=group, init=init)
    T = np.random.default_rng(group).uniform(0.05, 0.5, gf.nblk).astype(np.float32)
    gf.set_temperatures(T)
    n_chains, n_equil, n_samples = 3, 2, 3
    gf.sample_chains(n_chains, n_equil, n_samples)
    s_gpu = np.zeros(H * W)
    count = mpr.mpr_get_accumulator(gf.ctx, s_gpu)
    info = gf.refresh()
    gf.close()
    assert count == n_chains * n_samples
    assert info.gap_updates == n_chains * (n_equil + n_samples) * int(m.sum())
    o = oracle.Oracle(H, W, lb, seed=seed)
    phi, *_ = o.transform(z, m)
    st = o.block_stats(phi, m)
    s_ora = np.zeros(H * W)
    for r in range(n_chains):
        start = o.init_random(phi, m, r) if init else o.init_block_mean(phi, m, st)
        o.sample_chain(start, m, T.astype(np.float64), n_equil, n_samples, r, sum_out=s_ora)
    g = m.ravel() != 0
    assert np.all(s_gpu[~g] == 0.0)
    np.testing.assert_allclose(s_gpu[g], s_ora[g], rtol=0, atol=2e-4 * count)


def _isolated():
    """Gaps only on colour-0 sites, so every gap's neighbours are data."""
    rng = np.random.default_rng(31)
    H, W = 6, 7
    gaps = [(0, 0), (0, 2), (1, 1), (1, 3), (2, 4), (3, 3), (4, 2), (5, 5)]
    mask = np.zeros((H, W), np.uint8)
    for (y, x) in gaps:
        mask[y, x] = 1
    z = rng.uniform(0.0, 1.0, (H, W)).astype(np.float32)
    return H, W, gaps, mask, z


@pytest.mark.parametrize("storage,tol", [(0, 1e-3), (1, 1e-2)])
def test_sample_means_match_exact_conditional_means(storage, tol):
    H, W, gaps, mask, z = _isolated()
    T = 0.3
    n_chains, n_equil, n_samples = 16, 20, 2500
    gf = make(z, mask, 7, seed=99, group=8, storage=storage)
    gf.set_temperatures(np.full(gf.nblk, T, np.float32))
    means = np.zeros((n_chains, len(gaps)))
    for c in range(n_chains):
        # one chain per call: the running sum of that chain alone
        mpr.mpr_set_accumulator(gf.ctx, np.zeros(H * W), 0)
        gf.sample_chains(1, n_equil, n_samples)
        s = np.zeros(H * W)
        mpr.mpr_get_accumulator(gf.ctx, s)
        means[c] = [s[y * W + x] / n_samples for (y, x) in gaps]
    gf.close()
    phi, *_ = oracle.Oracle(H, W, 7).transform(z, mask)
    phi = phi.reshape(H, W)
    for g, (y, x) in enumerate(gaps):
        nodes, p = isolated_gap_law([phi[a, b] for (a, b) in neighbours(H, W, y, x)], T)
        exact = (p * nodes).sum()
        m = means[:, g].mean()
        se = means[:, g].std(ddof=1) / np.sqrt(n_chains)
        assert abs(m - exact) < 4 * se + tol, (g, m, exact, se)


def test_samples_and_realizations_share_the_mean():
    z, m = synth.small_problem(32, 32, 0.4, seed=8)
    gf = make(z, m, 8, seed=5)
    gf.set_temperatures(np.full(gf.nblk, 0.2, np.float32))
    gf.simulate(4)
    gf.sample_chains(2, 3, 5)
    s = np.zeros(32 * 32)
    assert mpr.mpr_get_accumulator(gf.ctx, s) == 4 + 2 * 5
    pred, _ = gf.predict()
    gf.close()
    info_min, info_max = float(z[m == 0].min()), float(z[m == 0].max())
    g = m != 0
    assert pred[g].min() >= info_min - 1e-5 and pred[g].max() <= info_max + 1e-5
    expect = info_min + (info_max - info_min) * (s.reshape(32, 32) / 14) / TWO_PI
    np.testing.assert_allclose(pred[g], expect[g], rtol=1e-5, atol=1e-5)


def test_sample_arguments_are_checked():
    z, m = synth.small_problem(24, 24, 0.5, seed=3)
    gf = make(z, m, 8, seed=1)
    with pytest.raises(MprError) as ex:
        gf.sample_chains(2, 2, 2)
    assert ex.value.status == MPR_ESTATE          # no temperatures yet
    gf.set_temperatures(np.full(gf.nblk, 0.2, np.float32))
    for args in [(0, 2, 2), (2, -1, 2), (2, 2, 0), (2, 60000, 6000)]:
        with pytest.raises(MprError) as ex:
            gf.sample_chains(*args)
        assert ex.value.status == MPR_EINVAL
    gf.sim_begin(2)
    with pytest.raises(MprError) as ex:
        gf.sample_chains(2, 2, 2)
    assert ex.value.status == MPR_ESTATE
    gf.sim_end()
    gf.close()
