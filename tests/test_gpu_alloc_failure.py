"""Allocation failures, injected on the host (the alloc_test hook refuses the
context's k-th device allocation without calling the allocator), for every k
a pipeline reaches: the call that needed the allocation returns MPR_ENOMEM,
the context stays usable (the same call succeeds when retried), the results
equal those of a run without the failure, and nothing leaks. No GPU fault is
involved: the refused allocation never reaches the device.
"""
import numpy as np
import pytest

from paper_2212_01317_gb300 import mpr, synth
from paper_2212_01317_gb300.mpr import GapFiller, GapFiller3, MprError, MPR_ENOMEM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _retrying(fn, failures):
    """Runs fn; an MPR_ENOMEM from the hook is recorded and fn retried once."""
    try:
        return fn()
    except MprError as e:
        assert e.status == MPR_ENOMEM and "alloc_test" in str(e), e
        failures.append(fn)
        return fn()


def pipeline_2d(z, m, k):
    failures = []
    opts = dict(seed=5, group=8, storage=1, cal_points=2, cal_warm=1.5, n_bisect=4, n_eq=3,
                n_meas=3, n_max=30, sweep_form=4, alloc_test=k)
    v = np.where(m != 0, np.nan, z).astype(np.float32)
    try:
        gf = GapFiller(v, m, 8, **opts)
    except MprError as e:
        assert e.status == MPR_ENOMEM
        return "create", None
    try:
        T = _retrying(gf.calibrate, failures)
        _retrying(lambda: gf.smooth_temperatures(8, 1), failures)   # site temperatures
        _retrying(lambda: gf.set_temperatures(T), failures)
        _retrying(lambda: gf.simulate(6), failures)
        _retrying(lambda: gf.sample_chains(2, 2, 2), failures)
        _retrying(lambda: gf.sim_begin(2), failures)
        s = _retrying(lambda: gf.get_state(1), failures)
        gf.sim_end()
        pred, sc = _retrying(lambda: gf.predict(truth=z), failures)
    finally:
        gf.close()
    assert len(failures) <= 1
    return ("run" if failures else None), (T, s, pred, sc)


def test_every_refused_allocation_of_a_2d_pipeline():
    import torch
    z, m = synth.small_problem(40, 48, 0.5, seed=12, kind="disc")
    _, ref = pipeline_2d(z, m, 0)
    mpr.mpr_release_cached_memory()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    seen = 0
    for k in range(1, 400):
        where, got = pipeline_2d(z, m, k)
        if where is None:
            break                     # k is past the pipeline's last allocation
        seen += 1
        if got is not None:
            for a, b in zip(got[:3], ref[:3]):
                np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-6)
    assert seen > 20                  # create, calibration, curve, tiles, SST, buffers
    mpr.mpr_release_cached_memory()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (4 << 20)


def test_every_refused_allocation_of_a_3d_pipeline():
    z, m = synth.small_problem(24, 20, 0.5, seed=3)
    vol = np.stack([z + 0.1 * i for i in range(6)]).astype(np.float32)
    msk = np.stack([m] * 6).astype(np.uint8)

    def run(k):
        failures = []
        try:
            g3 = GapFiller3(np.where(msk != 0, np.nan, vol), msk, 4, seed=2, n_bisect=3, n_eq=2,
                            n_meas=2, n_max=20, alloc_test=k)
        except MprError as e:
            assert e.status == MPR_ENOMEM
            return "create", None
        try:
            T = _retrying(g3.calibrate, failures)
            _retrying(lambda: g3.simulate(4), failures)
            pred, _ = _retrying(lambda: g3.predict(truth=vol), failures)
        finally:
            g3.close()
        return ("run" if failures else None), (T, pred)

    _, ref = run(0)
    seen = 0
    for k in range(1, 200):
        where, got = run(k)
        if where is None:
            break
        seen += 1
        if got is not None:
            for a, b in zip(got, ref):
                np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-6)
    assert seen > 10
