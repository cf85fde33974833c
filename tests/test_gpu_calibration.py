"""Calibration launch paths (GPU, through the C-ABI).

The per-block bisection of Sec. 2.1 / 2.2.2 runs either as one CUDA graph
(a device-side loop of per-half-step launches) or as one persistent
cooperative kernel with grid barriers. Both consume the same random streams
and the same arithmetic, so they must give the same temperatures. The
persistent kernel's barrier waits are bounded: a test hook makes every wait
give up, the call reports MPR_ETIMEOUT, and the device stays usable.
"""
import numpy as np
import pytest

from paper_2212_01317_gb300 import synth
from paper_2212_01317_gb300.mpr import GapFiller, MprError, MPR_EINVAL, MPR_ETIMEOUT

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


@pytest.mark.parametrize("H,W,lb,chains,kind", [(48, 40, 8, 1, "random"), (64, 64, 16, 2, "disc"),
                                                (37, 53, 8, 5, "random"), (96, 96, 32, 1, "disc")])
def test_persistent_equals_graph(H, W, lb, chains, kind):
    z, m = synth.small_problem(H, W, 0.55, seed=H + lb, kind=kind)
    opts = dict(seed=77, n_eq=6, n_meas=5, n_bisect=8, cal_chains=chains)
    Ts = []
    for mode in (1, 2):
        gf = make(z, m, lb, cal_mode=mode, **opts)
        Ts.append(gf.calibrate())
        gf.close()
    np.testing.assert_allclose(Ts[0], Ts[1], rtol=1e-6)


def test_barrier_timeout_is_reported_and_device_stays_usable():
    z, m = synth.small_problem(40, 40, 0.5, seed=3)
    # (sim_tail = 0: the hook applies to every grid barrier of the context,
    # and the simulation below is to run the per-launch loop.)
    gf = make(z, m, 8, cal_mode=2, barrier_test=1, wait_ms=100, n_bisect=2, n_eq=2, n_meas=2,
              sim_tail=0)
    with pytest.raises(MprError) as e:
        gf.calibrate()
    assert e.value.status == MPR_ETIMEOUT
    # The same context and a new one still work.
    gf.set_temperatures(np.full(gf.nblk, 0.2, np.float32))
    gf.simulate(2)
    pred, _ = gf.predict()
    assert np.isfinite(pred).all()
    gf.close()
    gf2 = make(z, m, 8, cal_mode=2, n_bisect=2, n_eq=2, n_meas=2)
    T = gf2.calibrate()
    assert np.all(T > 0)
    gf2.close()


# cal_sweep 0 picks the flat half-step at these sizes; 2 forces the warp form.
@pytest.mark.parametrize("cal_sweep", [0, 2])
@pytest.mark.parametrize("chains,kind", [(1, "random"), (3, "disc")])
def test_trisection_matches_oracle(chains, kind, cal_sweep):
    import oracle
    H, W, lb = 48, 40, 8
    z, m = synth.small_problem(H, W, 0.5, seed=H + chains, kind=kind)
    opts = dict(seed=31, n_eq=6, n_meas=6, n_bisect=10, cal_chains=chains, cal_sweep=cal_sweep)
    gf = make(z, m, lb, cal_points=2, **opts)
    T = gf.calibrate()
    gf.close()
    o = oracle.Oracle(H, W, lb, seed=31)
    phi, *_ = o.transform(z, m)
    st = o.block_stats(phi, m)
    phi0 = o.init_block_mean(phi, m, st)
    To, et, pt = o.calibrate_points(phi0, m, st, n_eq=6, n_meas=6, n_iter=10, chains=chains,
                                    points=2, trace=True)
    # A targeted block without gap sites has e_b = e_s,b exactly, so its
    # comparisons (and its T, which no site uses) follow the last bit of two
    # equal numbers computed in different orders: it takes the median instead.
    target = (st.Nsp > 0) & (st.n_gap > 0)
    explain_calibration(o, phi0, m, st, T, To, et, pt, 6, chains, target)
    med = np.float32(np.median(T[target]))
    np.testing.assert_allclose(T[~target], med, rtol=1e-6)
    # the graph and the host-launched forms agree
    gf = make(z, m, lb, cal_points=2, cal_mode=3, **opts)
    np.testing.assert_allclose(gf.calibrate(), T, rtol=1e-6)
    gf.close()


@pytest.mark.parametrize("cal_sweep", [0, 2])
@pytest.mark.parametrize("points,chains", [(4, 1), (8, 1), (4, 2)])
def test_k_point_calibration_matches_oracle(points, chains, cal_sweep):
    """Calibration with 4 or 8 temperatures per block and iteration (lane r of
    the chains at point r mod points; the bracket shrinks to the span between
    the highest point whose mean energy is below e_s,b and the lowest point
    whose mean is not) against the oracle's k-point calibration on the same
    random streams, block by block (tests/parity.py explain_calibration); the
    graph and the host-launched forms agree."""
    import oracle
    H, W, lb = 48, 40, 8
    z, m = synth.small_problem(H, W, 0.5, seed=H + points, kind="random")
    n_iter = 6
    opts = dict(seed=37, n_eq=6, n_meas=6, n_bisect=n_iter, cal_chains=chains, cal_sweep=cal_sweep)
    gf = make(z, m, lb, cal_points=points, **opts)
    T = gf.calibrate()
    gf.close()
    o = oracle.Oracle(H, W, lb, seed=37)
    phi, *_ = o.transform(z, m)
    st = o.block_stats(phi, m)
    phi0 = o.init_block_mean(phi, m, st)
    To, et, pt = o.calibrate_points(phi0, m, st, n_eq=6, n_meas=6, n_iter=n_iter, chains=chains,
                                    points=points, trace=True)
    target = (st.Nsp > 0) & (st.n_gap > 0)
    explain_calibration(o, phi0, m, st, T, To, et, pt, 6, chains, target)
    assert np.all((T > 1e-4) & (T < 2.0))
    gf = make(z, m, lb, cal_points=points, cal_mode=3, **opts)
    np.testing.assert_allclose(gf.calibrate(), T, rtol=1e-6)
    gf.close()


def _continued(points, chains, warm, n_next, n_iter, seed, H=48, W=40, lb=8, modes=(1, 3)):
    import oracle
    z, m = synth.small_problem(H, W, 0.5, seed=H + points + n_next, kind="disc")
    o = oracle.Oracle(H, W, lb, seed=seed)
    phi, *_ = o.transform(z, m)
    st = o.block_stats(phi, m)
    phi0 = o.init_block_mean(phi, m, st)
    opts = dict(seed=seed, n_eq=6, n_meas=6, n_bisect=n_iter, cal_chains=chains,
                cal_points=points, cal_continue=n_next, cal_warm=warm)
    Tc = np.geomspace(0.002, 1.25, 40).astype(np.float32)
    ec = oracle.energy_curve(Tc.astype(np.float64), L=64, n_eq=6, n_meas=6, seed=seed)
    Ts = []
    for mode in modes:
        gf = make(z, m, lb, cal_mode=mode, **opts)
        gf.set_energy_curve(Tc, ec)
        Ts.append(gf.calibrate())
        gf.close()
    T0 = o.warm_T0(st, Tc.astype(np.float64), ec) if warm > 0 else None
    return o, z, m, st, phi0, Ts, T0


@pytest.mark.parametrize("points,chains,warm,n_next", [(1, 1, 0.0, 5), (2, 1, 0.0, 0),
                                                       (2, 2, 1.5, 4), (4, 1, 1.5, 3)])
def test_continued_chains_match_oracle(points, chains, warm, n_next):
    """Calibration whose chains continue from one iteration to the next
    (cal_continue: only the first iteration restarts; later ones run n_next
    equilibration sweeps from where the previous stopped) against the
    oracle's, block by block, over the first two iterations (the first
    continued one included): the chains still run in lockstep there. Later,
    a Metropolis decision that FP32 and FP64 took differently carries over
    into every later iteration of its chain, so longer runs are compared in
    distribution (next test). Graph and host-launched forms agree."""
    seed = 53
    o, z, m, st, phi0, Ts, T0 = _continued(points, chains, warm, n_next, 2, seed)
    np.testing.assert_allclose(Ts[0], Ts[1], rtol=1e-6)
    To, et, pt = o.calibrate_points(phi0, m, st, n_eq=6, n_meas=6, n_iter=2, chains=chains,
                                    points=points, T0_warm=T0, warm=warm or 1.5,
                                    n_eq_next=n_next, trace=True)
    target = (st.Nsp > 0) & (st.n_gap > 0)
    explain_calibration(o, phi0, m, st, Ts[0], To, et, pt, 6, chains, target)


@pytest.mark.parametrize("points,warm,n_next", [(2, 1.5, 5), (1, 0.0, 5)])
def test_continued_chains_agree_with_oracle_in_distribution(points, warm, n_next):
    """Over a whole calibration the GPU's per-block temperatures differ from
    the oracle's (same random streams, chains continued) by no more than two
    runs of the oracle with different seeds differ from each other."""
    seed, n_iter = 61, 10
    o, z, m, st, phi0, Ts, T0 = _continued(points, 1, warm, n_next, n_iter, seed, H=64, W=64,
                                           modes=(1,))
    kw = dict(n_eq=6, n_meas=6, n_iter=n_iter, points=points, T0_warm=T0, warm=warm or 1.5,
              n_eq_next=n_next)
    To = o.calibrate_points(phi0, m, st, **kw)
    import oracle
    o2 = oracle.Oracle(*m.shape, 8, seed=seed + 1)
    To2 = o2.calibrate_points(phi0, m, st, **kw)
    target = (st.Nsp > 0) & (st.n_gap > 0)
    d_gpu = np.abs(np.log(Ts[0][target] / To[target]))
    d_seed = np.abs(np.log(To2[target] / To[target]))
    assert np.median(d_gpu) <= 2 * np.median(d_seed) + 1e-3, (np.median(d_gpu), np.median(d_seed))
    assert np.mean(d_gpu) <= 2 * np.mean(d_seed) + 1e-3


def test_continued_chains_count_their_sweeps():
    z, m = synth.small_problem(40, 40, 0.5, seed=4)
    gf = make(z, m, 8, seed=1, n_eq=6, n_meas=4, n_bisect=5, cal_points=2, cal_continue=2)
    gf.calibrate()
    info = gf.refresh()
    gf.close()
    sweeps = (6 + 4) + 4 * (2 + 4)
    assert info.cal_gap_updates == sweeps * 2 * int(m.sum())


def test_calibration_sweep_forms():
    """cal_sweep: an unknown form is refused at create; the flat and the warp
    half-steps make the same moves from the same random numbers and differ
    only in the FP32 order of the block sums, so their temperatures agree
    block by block unless a comparison sat at a tie (the oracle tests above
    explain each form's blocks); the sweep count is the same."""
    z, m = synth.small_problem(64, 64, 0.5, seed=9, kind="disc")
    with pytest.raises(MprError) as e:
        make(z, m, 8, cal_sweep=3)
    assert e.value.status == MPR_EINVAL
    Ts, ups = [], []
    for form in (1, 2):
        gf = make(z, m, 8, seed=3, n_eq=6, n_meas=6, n_bisect=8, cal_points=2, cal_sweep=form)
        Ts.append(gf.calibrate())
        ups.append(gf.refresh().cal_gap_updates)
        gf.close()
    assert ups[0] == ups[1]
    close = np.abs(Ts[0] - Ts[1]) <= 1e-5 * Ts[0]
    assert close.mean() >= 0.9, close.mean()
