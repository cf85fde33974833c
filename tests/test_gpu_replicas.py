"""Realizations split across contexts, through the C-ABI on one GPU.

Each context stands for one rank of a job that shares a field: it runs a
disjoint range of realization indices (mpr_set_realization_base), exports its
per-site sums (mpr_get_accumulator), and one context takes the added sums
back (mpr_set_accumulator) and predicts. The ranks run one after another, so
nothing waits on anything else. The result must equal one context that ran
every index: same chains (Sec. 2.1, realizations differ only in their random
numbers), so the same sums up to the order of the FP64 additions.
"""
import numpy as np
import pytest

from paper_2212_01317_gb300 import mpr, replicas, synth

pytestmark = pytest.mark.gpu


def field():
    z, m = synth.small_problem(72, 60, 0.5, seed=21)
    return z, m, np.where(m != 0, np.nan, z).astype(np.float32)


@pytest.mark.parametrize("world,R", [(2, 7), (3, 12), (4, 3)])
def test_split_realizations_equal_one_context(world, R):
    z, m, v = field()
    one = mpr.GapFiller(v, m, 8, seed=5)
    T = one.calibrate()
    one.simulate(R)
    ref, ref_err = one.predict(z)
    ref_acc = np.zeros(m.shape)
    assert mpr.mpr_get_accumulator(one.ctx, ref_acc) == R
    one.close()
    total = np.zeros(m.shape)
    n = 0
    for rank in range(world):
        gf = mpr.GapFiller(v, m, 8, seed=5)
        gf.set_temperatures(T)
        first, count = replicas.shard_realizations(R, world, rank)
        mpr.mpr_set_realization_base(gf.ctx, first)
        if count:
            gf.simulate(count)
        acc = np.zeros(m.shape)
        n += mpr.mpr_get_accumulator(gf.ctx, acc)
        total += acc
        if rank < world - 1:
            gf.close()
    assert n == R
    assert (total[m == 0] == 0).all()
    np.testing.assert_allclose(total, ref_acc, rtol=1e-13, atol=1e-10)
    mpr.mpr_set_accumulator(gf.ctx, total, n)
    out, err = gf.predict(z)
    gf.close()
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-5 * (np.nanmax(v) - np.nanmin(v)))
    assert np.array_equal(out[m == 0], z[m == 0])
    np.testing.assert_allclose(err, ref_err, rtol=1e-5)


def test_accumulator_calls_check_state_and_arguments():
    z, m, v = field()
    gf = mpr.GapFiller(v, m, 8, seed=5)
    gf.set_temperatures(np.full(gf.nblk, 0.05, np.float32))
    with pytest.raises(mpr.MprError):
        mpr.mpr_set_realization_base(gf.ctx, -1)
    gf.sim_begin(2)
    with pytest.raises(mpr.MprError):
        mpr.mpr_get_accumulator(gf.ctx, np.zeros(m.shape))
    with pytest.raises(mpr.MprError):
        mpr.mpr_set_realization_base(gf.ctx, 4)
    gf.sim_end()
    with pytest.raises(mpr.MprError):
        mpr.mpr_set_accumulator(gf.ctx, np.zeros(m.shape), -1)
    # Round trip through the caller's buffer, device pointers included.
    torch = pytest.importorskip("torch")
    a = torch.zeros(m.shape, dtype=torch.float64, device="cuda")
    assert mpr.mpr_get_accumulator(gf.ctx, a) == 2
    mpr.mpr_set_accumulator(gf.ctx, a * 2, 4)     # twice the sums, twice the count
    p2, _ = gf.predict()
    mpr.mpr_set_accumulator(gf.ctx, a, 2)
    p1, _ = gf.predict()
    np.testing.assert_allclose(p2, p1, rtol=0, atol=1e-6)
    gf.close()
