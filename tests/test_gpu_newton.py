"""Differentiable energy matching on the GPU (through the C-ABI and the
torch.autograd.Function built on it), against the oracle.

  * block-energy moments of the calibration chains: same chains as the
    oracle's (same Philox streams), element by element;
  * the backward (vector-Jacobian product) kernel against the formula
    applied to the returned moments;
  * the fluctuation identity against common-random-number finite
    differences on a single block (where it is exact);
  * Newton calibration against the oracle's Newton calibration and against
    bisection;
  * the autograd Function's forward / backward.
"""
import numpy as np
import pytest

import oracle
from paper_2212_01317_gb300 import mpr, synth
from paper_2212_01317_gb300.mpr import GapFiller, MprError

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def make(z, m, lb, **opt):
    v = np.where(m != 0, np.nan, z).astype(np.float32)
    return GapFiller(v, m, lb, **opt)


def moments(gf, beta, n_eq, n_meas, tag, restart):
    out = [np.zeros(gf.nblk) for _ in range(4)]
    mpr.mpr_energy_moments(gf.ctx, np.ascontiguousarray(beta, np.float32), n_eq, n_meas, tag,
                           restart, *out)
    return out


@pytest.mark.parametrize("chains", [1, 2, 6])
def test_moments_match_oracle(torch, chains):
    H, W, lb = 40, 36, 8
    z, m = synth.small_problem(H, W, 0.5, seed=17)
    gf = make(z, m, lb, seed=99, cal_chains=chains)
    rng = np.random.default_rng(1)
    beta = rng.uniform(3.0, 30.0, gf.nblk).astype(np.float32)
    got = moments(gf, beta, 5, 12, 3, True)
    o = oracle.Oracle(H, W, lb, seed=99)
    phi, _, _, _ = o.transform(z, m)
    st = o.block_stats(phi, m)
    phi0 = o.init_block_mean(phi, m, st)
    ph = np.repeat(phi0[None], chains, axis=0).copy()
    T = (1.0 / beta.astype(np.float64))
    # the chains run at beta exactly: T = 1 / beta in FP64 gives the same decisions
    want = o.energy_moments(ph, m, T, 5, 12, tag=3, st=st)
    close = np.abs(got[0] - want[0]) <= 1e-5
    assert close.mean() >= 0.9, close.mean()
    for k in (1, 2, 3):
        ok = np.abs(got[k] - want[k]) <= 1e-3 * (np.abs(want[1]).max() + 1)
        assert ok[close].mean() >= 0.9
    # continuing the chains differs from restarting them
    cont = moments(gf, beta, 0, 4, 4, False)
    fresh = moments(gf, beta, 0, 4, 4, True)
    assert not np.allclose(cont[0], fresh[0])
    gf.close()


def test_vjp_kernel_is_the_formula(torch):
    H, W, lb = 48, 40, 8
    z, m = synth.small_problem(H, W, 0.5, seed=5)
    gf = make(z, m, lb, seed=1, cal_chains=4)
    beta = np.full(gf.nblk, 12.0, np.float32)
    y, var, cr, cd = moments(gf, beta, 5, 10, 1, True)
    _, _, Nb, _, _ = gf.block_stats()
    nbx = gf.info.nbx
    g = np.random.default_rng(2).normal(size=gf.nblk)
    out = np.zeros(gf.nblk)
    mpr.mpr_energy_vjp(gf.ctx, g, out)
    # dense Jacobian J[a, b] = -Cov(E_a, E_b) / N_a on the five-point stencil
    J = np.zeros((gf.nblk, gf.nblk))
    for b in range(gf.nblk):
        J[b, b] = -var[b] / Nb[b]
        if b % nbx != nbx - 1:
            J[b, b + 1] = -cr[b] / Nb[b]
            J[b + 1, b] = -cr[b] / Nb[b + 1]
        if b + nbx < gf.nblk:
            J[b, b + nbx] = -cd[b] / Nb[b]
            J[b + nbx, b] = -cd[b] / Nb[b + nbx]
    np.testing.assert_allclose(out, g @ J, rtol=1e-12, atol=1e-15)
    gf.close()


def test_fluctuation_identity_against_crn_finite_differences(torch):
    # One block: the identity is exact; common random numbers (same tag,
    # fresh chains) make the finite difference precise enough to compare.
    H = W = 24
    z, m = synth.small_problem(H, W, 0.4, seed=8)
    gf = make(z, m, 24, seed=3, cal_chains=64)
    _, _, Nb, _, _ = gf.block_stats()
    fd, fl = [], []
    for tag in (1, 2, 3, 4):
        b0 = 10.0
        h = 0.25
        yp = moments(gf, [b0 + h], 20, 60, tag, True)[0][0]
        ym = moments(gf, [b0 - h], 20, 60, tag, True)[0][0]
        _, var, _, _ = moments(gf, [b0], 20, 60, tag, True)
        fd.append((yp - ym) / (2 * h))
        fl.append(-var[0] / Nb[0])
    fd, fl = np.array(fd), np.array(fl)
    se = np.hypot(fd.std(ddof=1), fl.std(ddof=1)) / 2
    assert abs(fd.mean() - fl.mean()) < 4 * se + 0.08 * abs(fl.mean()), (fd, fl)
    gf.close()


def test_newton_calibration_matches_oracle_and_bisection(torch):
    H, W, lb = 48, 48, 8
    z, m = synth.small_problem(H, W, 0.5, seed=23, xi=6.0)
    opts = dict(seed=11, cal_chains=2, n_eq=10, n_meas=20)
    gn = make(z, m, lb, cal_method=1, n_newton=6, t_init=0.1, **opts)
    Tn = gn.calibrate()
    o = oracle.Oracle(H, W, lb, seed=11)
    phi, _, _, _ = o.transform(z, m)
    st = o.block_stats(phi, m)
    phi0 = o.init_block_mean(phi, m, st)
    To = o.calibrate_newton(phi0, m, st, n_eq=10, n_meas=20, n_newton=6, chains=2, T0=0.1)
    # The chains continue from one iteration to the next, so a decision that
    # flips on rounding (FP32 vs FP64) separates a block's chain for good:
    # most blocks agree to 1e-4, the rest within the Monte Carlo spread.
    close = np.abs(Tn - To) <= 1e-4 * To
    assert close.mean() >= 0.6, close.mean()
    assert np.median(np.abs(Tn - To) / To) < 0.02
    gb = make(z, m, lb, **opts)
    Tb = gb.calibrate()
    # Blocks whose sample energy no temperature reaches send bisection to the
    # bracket's floor and Newton towards it; compare the others.
    ok = Tb > 1e-3
    rel = np.abs(Tn - Tb)[ok] / Tb[ok]
    assert np.median(rel) < 0.25, np.median(rel)
    # the Newton temperatures fit the energies about as well as bisection's
    yn = moments(gn, 1.0 / Tn, 20, 200, 7, True)[0]
    yb = moments(gb, 1.0 / Tb, 20, 200, 7, True)[0]
    t = (st.Nsp > 0) & ok
    assert np.mean(np.abs(yn - st.es)[t]) < 1.5 * np.mean(np.abs(yb - st.es)[t]) + 1e-3
    gn.close()
    gb.close()


def test_newton_step_is_the_update_rule(torch):
    """One Newton iteration = the chains' moments at t_init (same fresh chains
    and tag as mpr_energy_moments with restart, tag 1) and the damped step
    applied to them, block by block."""
    H, W, lb = 40, 48, 8
    z, m = synth.small_problem(H, W, 0.5, seed=29)
    opts = dict(seed=4, cal_chains=2, n_eq=8, n_meas=16)
    g1 = make(z, m, lb, cal_method=1, n_newton=1, t_init=0.07, **opts)
    T1 = g1.calibrate()
    g2 = make(z, m, lb, **opts)
    y, var, _, _ = moments(g2, np.full(g2.nblk, 1 / np.float32(0.07), np.float32), 8, 16, 1, True)
    Es, Nsp, Nb, _, _ = g2.block_stats()
    es = Es / Nsp
    t0 = np.float64(np.float32(0.07))
    bn = 1 / t0 + (y - es) * Nb / var
    tn = np.where(bn > 0, 1 / np.where(bn > 0, bn, 1), 2 * t0)
    tn = np.clip(tn, 0.5 * t0, 2 * t0)
    want = np.clip(tn, np.float32(1e-4), np.float32(2.0)).astype(np.float32)
    np.testing.assert_allclose(T1, want, rtol=2e-6)
    g1.close()
    g2.close()


def test_autograd_function(torch):
    from paper_2212_01317_gb300.autograd import BlockEnergy, block_moments
    H, W, lb = 32, 40, 8
    z, m = synth.small_problem(H, W, 0.5, seed=4)
    gf = make(z, m, lb, seed=5, cal_chains=2)
    beta = torch.full((gf.nblk,), 8.0, device="cuda", requires_grad=True)
    y = BlockEnergy.apply(beta, gf.ctx, 5, 10, 2, True)
    w = torch.linspace(-1, 1, gf.nblk, device="cuda", dtype=torch.float64)
    (w * y).sum().backward()
    # same run through the plain calls
    y2, var, cr, cd = moments(gf, np.full(gf.nblk, 8.0, np.float32), 5, 10, 2, True)
    # (block sums use FP32 atomics, whose order varies from run to run)
    np.testing.assert_allclose(y.detach().cpu().numpy(), y2, rtol=1e-7)
    g = np.zeros(gf.nblk)
    mpr.mpr_energy_vjp(gf.ctx, w.cpu().numpy(), g)
    np.testing.assert_allclose(beta.grad.cpu().numpy(), g.astype(np.float32), rtol=1e-4,
                               atol=1e-6 * np.abs(g).max())
    # the library's Newton calibration (mpr_calibrate, cal_method = 1) moves
    # the chains' energies, measured through the autograd module, towards
    # their targets
    Es, Nsp, Nb, _, _ = gf.block_stats()
    t = Nsp > 0
    e = np.where(t, Es / np.maximum(Nsp, 1), 0.0)
    gn = make(z, m, lb, seed=5, cal_chains=2, cal_method=1, n_newton=5, n_eq=10, n_meas=20,
              t_init=0.05)
    b1 = torch.tensor(1.0 / gn.calibrate(), dtype=torch.float32, device="cuda")
    gn.close()
    y_end = block_moments(gf.ctx, b1, 10, 40, 9, True)[0].cpu().numpy()
    y_start = block_moments(gf.ctx, torch.full((gf.nblk,), 20.0, device="cuda"), 10, 40, 9,
                            True)[0].cpu().numpy()
    assert np.mean(np.abs(y_end - e)[t]) < 0.5 * np.mean(np.abs(y_start - e)[t])
    gf.close()


def test_moments_state_rules(torch):
    z, m = synth.small_problem(20, 20, 0.5, seed=1)
    gf = make(z, m, 4)
    with pytest.raises(MprError):
        mpr.mpr_energy_vjp(gf.ctx, np.zeros(gf.nblk), np.zeros(gf.nblk))   # no moments yet
    with pytest.raises(MprError):
        moments(gf, np.zeros(gf.nblk), 1, 1, 1, True)                     # beta must be > 0
    with pytest.raises(MprError):
        moments(gf, np.ones(gf.nblk), 1, 1, 0, True)                      # tag 0 is reserved
    gf.set_temperatures(np.full(gf.nblk, 0.1, np.float32))
    gf.sim_begin(2)
    with pytest.raises(MprError):
        moments(gf, np.ones(gf.nblk), 1, 1, 1, True)                      # batch open
    gf.sim_end()
    gf.close()
