"""The unconditional e(T) curve and the calibration paths that read it
(Sec. 2.1 energy matching on a data-free lattice), through the C-ABI.

  * the measured curve after one sweep, temperature by temperature, against
    the oracle's on the same random streams (FP32 against FP64 arithmetic:
    equal to rounding unless a Metropolis decision flipped);
  * the default curve (25 + 20 sweeps) against the oracle's within the Monte
    Carlo spread of the oracle's curve over seeds;
  * the warm-started calibration (trisection and 4 points) against the
    oracle's on the same curve and random streams; graph and host-launched
    forms agree;
  * cal_method = 2 (T read off the curve) against the oracle's inverse;
  * argument checks.
"""
import numpy as np
import pytest

import oracle
from paper_2212_01317_gb300 import mpr, synth
from paper_2212_01317_gb300.mpr import GapFiller, MprError, MPR_EINVAL

from parity import explain_calibration

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def make(z, m, lb, **opt):
    v = np.where(m != 0, np.nan, z).astype(np.float32)
    return GapFiller(v, m, lb, **opt)


def test_curve_after_one_sweep_matches_oracle():
    z, m = synth.small_problem(24, 24, 0.5, seed=1)
    # (the curve's random streams use the key (0, 0) whatever the seed)
    gf = make(z, m, 8, seed=0x1234_5678_9ABC, n_eq=0, n_meas=1)
    T, e = gf.energy_curve()
    gf.close()
    assert T.size == mpr.MPR_CURVE_POINTS
    assert np.all(np.diff(T) > 0)
    np.testing.assert_allclose(T[[0, -1]], [0.002, 1.25], rtol=1e-6)
    eo = oracle.energy_curve(T.astype(np.float64), L=64, n_eq=0, n_meas=1, seed=0)
    d = np.abs(e - eo)
    # no flipped decision: FP32 rounding of 8064 bond terms; a flip moves one
    # site and changes e by about 4 / 8064
    assert (d > 2e-5).sum() <= 2, d
    assert d.max() < 3e-3


def test_default_curve_matches_oracle_within_monte_carlo_spread():
    z, m = synth.small_problem(24, 24, 0.5, seed=2)
    gf = make(z, m, 8, seed=77)
    T, e = gf.energy_curve()
    gf.close()
    Td = T.astype(np.float64)
    eo = oracle.energy_curve(Td, L=64, n_eq=25, n_meas=20, seed=0)
    spread = np.std([oracle.energy_curve(Td, L=64, n_eq=25, n_meas=20, seed=s)
                     for s in range(1000, 1006)], axis=0, ddof=1)
    # the two runs share their random streams, so they differ by less than two
    # independent runs; bound by 5 standard deviations of a difference
    assert np.all(np.abs(e - eo) <= 5 * np.sqrt(2) * spread + 1e-6), (e - eo, spread)
    # the curve rises with T
    assert np.all(np.diff(e) > -5 * spread[1:] - 1e-6)


@pytest.mark.parametrize("points,chains,mode", [(2, 1, 1), (2, 2, 1), (4, 1, 1), (2, 1, 3)])
def test_warm_calibration_matches_oracle(points, chains, mode):
    H, W, lb = 48, 40, 8
    z, m = synth.small_problem(H, W, 0.5, seed=H + points + chains, kind="disc")
    seed, n_iter, w = 41, 8, 1.5
    o = oracle.Oracle(H, W, lb, seed=seed)
    phi, *_ = o.transform(z, m)
    st = o.block_stats(phi, m)
    phi0 = o.init_block_mean(phi, m, st)
    Tc = np.geomspace(0.002, 1.25, 40).astype(np.float32)
    ec = oracle.energy_curve(Tc.astype(np.float64), L=64, n_eq=6, n_meas=6, seed=seed)
    opts = dict(seed=seed, n_eq=6, n_meas=6, n_bisect=n_iter, cal_chains=chains,
                cal_points=points, cal_warm=w)
    gf = make(z, m, lb, cal_mode=mode, **opts)
    gf.set_energy_curve(Tc, ec)
    T = gf.calibrate()
    gf.close()
    T0 = o.warm_T0(st, Tc.astype(np.float64), ec)
    To, et, pt = o.calibrate_points(phi0, m, st, n_eq=6, n_meas=6, n_iter=n_iter, chains=chains,
                                    points=points, T0_warm=T0, warm=w, trace=True)
    target = (st.Nsp > 0) & (st.n_gap > 0)
    explain_calibration(o, phi0, m, st, T, To, et, pt, 6, chains, target)
    assert np.all((T > 1e-4) & (T < 2.0))
    if mode == 1:
        # the host-launched form runs the same launches
        gf = make(z, m, lb, cal_mode=3, **opts)
        gf.set_energy_curve(Tc, ec)
        np.testing.assert_allclose(gf.calibrate(), T, rtol=1e-6)
        gf.close()


def test_warm_first_iteration_points_on_the_device():
    """One warm iteration: every targeted block's T is the midpoint of
    [t_lo, T0/w], [T0/w, T0 w] or [T0 w, t_hi] (FP32 points from FP64 T0)."""
    H, W, lb = 40, 48, 8
    z, m = synth.small_problem(H, W, 0.5, seed=5, kind="random")
    seed, w = 9, 1.5
    o = oracle.Oracle(H, W, lb, seed=seed)
    phi, *_ = o.transform(z, m)
    st = o.block_stats(phi, m)
    Tc = np.geomspace(0.002, 1.25, 40).astype(np.float32)
    ec = oracle.energy_curve(Tc.astype(np.float64), L=64, n_eq=4, n_meas=4, seed=seed)
    gf = make(z, m, lb, seed=seed, n_eq=4, n_meas=4, n_bisect=1, cal_points=2, cal_warm=w)
    gf.set_energy_curve(Tc, ec)
    T = gf.calibrate()
    gf.close()
    T0 = o.warm_T0(st, Tc.astype(np.float64), ec)
    tgt = (st.Nsp > 0) & (st.n_gap > 0)
    for b in np.flatnonzero(tgt):
        a, c = np.float32(T0[b] / w), np.float32(T0[b] * w)
        mids = [np.float32(0.5) * (np.float32(1e-4) + a), np.float32(0.5) * (a + c),
                np.float32(0.5) * (c + np.float32(2.0))]
        assert min(abs(float(x) - float(T[b])) for x in mids) <= 1e-6 * float(T[b]), (b, T[b], mids)


def test_curve_method_reads_the_curve():
    H, W, lb = 40, 48, 8
    z, m = synth.small_problem(H, W, 0.45, seed=6, kind="disc")
    o = oracle.Oracle(H, W, lb, seed=3)
    phi, *_ = o.transform(z, m)
    st = o.block_stats(phi, m)
    Tc = np.geomspace(0.002, 1.25, 40).astype(np.float32)
    ec = oracle.energy_curve(Tc.astype(np.float64), L=64, n_eq=6, n_meas=6, seed=3)
    gf = make(z, m, lb, seed=3, cal_method=2)
    gf.set_energy_curve(Tc, ec)
    T = gf.calibrate()
    gf.close()
    T0 = o.warm_T0(st, Tc.astype(np.float64), ec)
    tgt = (st.Nsp > 0) & (st.n_gap > 0)
    np.testing.assert_allclose(T[tgt], T0[tgt].astype(np.float32), rtol=2e-7)
    med = np.float32(np.median(T[tgt]))
    np.testing.assert_allclose(T[~tgt], med, rtol=1e-6)


def test_curve_is_shared_by_contexts_with_the_same_parameters():
    """The measured curve is a function of q, J, over-relaxation, n_eq and
    n_meas: contexts with other seeds or fields read the same numbers; other
    parameters give another curve (over-relaxation off: the oracle's)."""
    z, m = synth.small_problem(24, 24, 0.5, seed=4)
    z2, m2 = synth.small_problem(40, 32, 0.3, seed=5)
    curves = []
    for zz, mm, seed in [(z, m, 1), (z2, m2, 99), (z, m, 7)]:
        gf = make(zz, mm, 8, seed=seed, n_eq=3, n_meas=2)
        curves.append(gf.energy_curve())
        gf.close()
    for T, e in curves[1:]:
        np.testing.assert_array_equal(T, curves[0][0])
        np.testing.assert_array_equal(e, curves[0][1])
    gf = make(z, m, 8, seed=1, n_eq=3, n_meas=2, overrelax=0)
    T, e = gf.energy_curve()
    gf.close()
    assert not np.array_equal(e, curves[0][1])
    eo = oracle.energy_curve(T.astype(np.float64), L=64, n_eq=3, n_meas=2, seed=0,
                             overrelax=False)
    assert np.median(np.abs(e - eo)) < 2e-5


def test_curve_method_with_the_measured_curve_fills_a_field():
    z, m = synth.small_problem(64, 64, 0.6, seed=7, kind="random")
    gf = make(z, m, 16, seed=5, cal_method=2)
    T = gf.calibrate()
    Tc, _ = gf.energy_curve()
    assert np.all((T >= Tc[0]) & (T <= Tc[-1]))
    gf.simulate(4)
    pred, (aae, _) = gf.predict(truth=z)
    gf.close()
    assert np.isfinite(pred).all() and aae > 0


def test_curve_arguments_are_checked():
    z, m = synth.small_problem(24, 24, 0.5, seed=3)
    gf = make(z, m, 8, seed=1)
    for T, e in [(np.array([0.1], np.float32), np.array([-0.9])),
                 (np.array([0.1, 0.1], np.float32), np.array([-0.9, -0.8])),
                 (np.array([0.1, 0.05], np.float32), np.array([-0.9, -0.8])),
                 (np.array([-0.1, 0.2], np.float32), np.array([-0.9, -0.8])),
                 (np.array([0.1, 0.2], np.float32), np.array([-0.9, np.nan])),
                 (np.linspace(0.01, 1, 65).astype(np.float32), np.linspace(-1, -0.5, 65))]:
        with pytest.raises(MprError) as ex:
            gf.set_energy_curve(T, e)
        assert ex.value.status == MPR_EINVAL
    gf.close()
    for bad in (dict(cal_warm=1.5, cal_points=1), dict(cal_warm=0.5, cal_points=2),
                dict(cal_warm=1.5, cal_points=2, cal_method=1), dict(cal_method=3)):
        with pytest.raises(MprError) as ex:
            make(z, m, 8, **bad)
        assert ex.value.status == MPR_EINVAL
    # the default curve widened by w = 1.7 leaves the bracket (0.002 / 1.7 is
    # inside, 1.25 * 1.7 is not)
    gf = make(z, m, 8, cal_warm=1.7, cal_points=2, n_bisect=2, n_eq=2, n_meas=2)
    with pytest.raises(MprError) as ex:
        gf.calibrate()
    assert ex.value.status == MPR_EINVAL
    gf.close()
