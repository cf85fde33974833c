"""The staged half-step (sweep form 4: the other colour's (cos, sin) of q phi
staged in shared memory per tile) through the C-ABI.

  * one half-step element by element against the FP64 oracle (the same
    Philox draws), for tiles equal to a block (l_b = 8, 16), several tiles
    per block (32, 64), partial tiles (17, 24, 40) and odd widths, with
    running and stopped (block, realization) pairs;
  * whole sweeps against the one-warp-per-pair form (same arithmetic and
    random numbers; only the order of the FP32 energy sums differs): the
    stop sweeps agree and, where all of them do, the states are
    bit-identical, in the FP32, BF16 and FP16 state;
  * a batch of uneven fields in one canvas (tiles at slice borders, absent
    sites between fields) against the same form.
Tolerances: tests/parity.py.
"""
import numpy as np
import pytest

import oracle
from paper_2212_01317_gb300 import mpr, synth
from paper_2212_01317_gb300.mpr import BatchFiller, GapFiller

from parity import TWO_PI, checkerboard, compare_site_updates

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()


def make(z, m, lb, **opt):
    v = z.copy()
    v[m != 0] = np.nan
    return GapFiller(v, m, lb, **opt)


@pytest.mark.parametrize("H,W,lb,R,kind", [(45, 38, 8, 8, "random"), (70, 67, 16, 11, "random"),
                                           (66, 97, 32, 8, "disc"), (50, 77, 24, 9, "random"),
                                           (41, 45, 17, 16, "random"), (130, 131, 64, 8, "disc"),
                                           (83, 40, 40, 8, "random")])
@pytest.mark.parametrize("colour", [0, 1])
def test_tile_halfstep_lockstep(H, W, lb, R, kind, colour):
    z, m = synth.small_problem(H, W, 0.55, seed=H + lb + colour, kind=kind)
    seed = 0x5EED0000 + lb
    gf = make(z, m, lb, seed=seed, group=8, sweep_form=4)
    o = oracle.Oracle(H, W, lb, seed=seed)
    rng = np.random.default_rng(lb + colour)
    T = rng.uniform(0.02, 1.2, gf.nblk).astype(np.float32)
    gf.set_temperatures(T)
    gf.sim_begin(R)
    assert gf.refresh().group == 8
    pre = []
    for r in range(R):
        s = gf.get_state(r).astype(np.float32)
        g = m != 0
        s[g] = rng.uniform(0, TWO_PI, g.sum()).astype(np.float32)
        gf.set_state(r, s)
        pre.append(s)
    running = (rng.uniform(size=(R, gf.nblk)) < 0.7).astype(np.uint8)
    gf.set_running(running)
    t, tag = 23, 0
    gf.halfstep(colour, t, tag)
    blk = o.block_index()
    cb = checkerboard(H, W)
    total = flips = 0
    for r in range(R):
        post = gf.get_state(r)
        ph = pre[r].astype(np.float64)
        diag = o.halfstep(ph, m, colour, T.astype(np.float64), running[r], t=t, tag=tag, r=r,
                          diag=True).reshape(H, W)
        may = (m != 0) & (cb == colour) & (running[r][blk] == 1)
        n, f, bad, msg = compare_site_updates(post, ph, pre[r], diag, may)
        assert bad == 0, f"r={r}: {msg}"
        total += n
        flips += f
        assert post.min() >= 0 and post.max() <= TWO_PI
    assert total > 50 * R
    assert flips <= max(2, total // 2000)
    gf.close()


def run_sweeps(z, m, lb, form, R, storage, T, n_sweeps=12):
    gf = make(z, m, lb, seed=11, group=8, sweep_form=form, n_max=60, storage=storage)
    gf.set_temperatures(T)
    gf.sim_begin(R)
    gf.sim_sweep(n_sweeps)
    states = [gf.get_state(r) for r in range(R)]
    stop = gf.get_stop(R)[0]
    e = gf.block_e(R)
    gf.sim_end()
    gf.close()
    return states, stop, e


@pytest.mark.parametrize("H,W,lb,storage", [(96, 80, 16, 0), (96, 96, 32, 0), (130, 129, 64, 0),
                                            (75, 91, 17, 0), (96, 96, 32, 1), (80, 90, 16, 2)])
def test_tile_form_agrees_with_warp_form(H, W, lb, storage):
    z, m = synth.small_problem(H, W, 0.6, seed=lb + storage, kind="disc")
    nblk = ((H + lb - 1) // lb) * ((W + lb - 1) // lb)
    T = np.random.default_rng(lb).uniform(0.03, 0.4, nblk).astype(np.float32)
    R = 13
    s0, st0, e0 = run_sweeps(z, m, lb, 0, R, storage, T)
    s4, st4, e4 = run_sweeps(z, m, lb, 4, R, storage, T)
    assert np.mean(st4 == st0) >= 0.99
    np.testing.assert_allclose(e4, e0, rtol=0, atol=5e-6)
    if np.array_equal(st4, st0):          # the usual case: no tie moved a stop
        for r in range(R):
            assert np.array_equal(s4[r], s0[r])


def test_tile_form_in_a_batch():
    """Fields of uneven size in one canvas: the staged form computes what the
    one-warp-per-pair form computes (tiles at slice borders see no bond to
    the neighbouring field)."""
    shapes = [(37, 53, "random", 0.45), (64, 64, "disc", 0.6), (20, 90, "random", 0.3),
              (48, 40, "random", 0.7), (33, 17, "random", 0.5)]
    vals, masks = [], []
    for k, (h, w, kind, p) in enumerate(shapes):
        z, m = synth.small_problem(h, w, p, seed=70 + k, kind=kind)
        z = (z * (1 + k) + 5 * k).astype(np.float32)
        vals.append(np.where(m != 0, np.nan, z).astype(np.float32))
        masks.append(m)
    R = 10
    res = []
    for form in (0, 4):
        bf = BatchFiller(vals, masks, 16, seed=9, group=8, sweep_form=form, n_max=50)
        T = np.random.default_rng(3).uniform(0.05, 0.5, bf.info.nblk).astype(np.float32)
        bf.set_temperatures(T)
        bf.simulate(R)
        outs, _ = bf.predict()
        res.append((outs, mpr.mpr_get_info(bf.ctx).gap_updates))
        bf.close()
    (o0, u0), (o4, u4) = res
    assert abs(u4 - u0) <= max(1, u0 // 2000)
    if u4 == u0:
        for a, b in zip(o0, o4):
            np.testing.assert_array_equal(a, b)
    else:
        for a, b in zip(o0, o4):
            assert np.mean(np.abs(a - b) < 1e-5) > 0.98
