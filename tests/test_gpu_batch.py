"""Many fields in one context (mpr_create_batch), through the C-ABI.

Each field of a batch must compute what it computes alone (mpr_create with
slice_id + k): its own transform range, Eq. 2 statistics, random streams
(site numbering within the field), median fallback and stop bookkeeping,
and no bond to another field. The single-field path is checked against the
oracle elsewhere, so the batch is checked against it field by field.
"""
import numpy as np
import pytest

from paper_2212_01317_gb300 import mpr, synth
from paper_2212_01317_gb300.mpr import BatchFiller, GapFiller

pytestmark = pytest.mark.gpu

SHAPES = [(37, 53, "random", 0.45), (64, 64, "disc", 0.6), (20, 90, "random", 0.3),
          (48, 40, "random", 0.7), (9, 9, "random", 0.5)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def fields(lb=8):
    out = []
    for k, (h, w, kind, p) in enumerate(SHAPES):
        z, m = synth.small_problem(h, w, p, seed=40 + k, kind=kind)
        z = (z * (1 + k) + 10 * k).astype(np.float32)          # different value ranges
        out.append((z, m, np.where(m != 0, np.nan, z).astype(np.float32)))
    return out


def block_rects(bf):
    lb = bf.info.block
    return [(y0 // lb, x0 // lb, (h + lb - 1) // lb, (w + lb - 1) // lb)
            for (y0, x0, h, w) in bf.layout]


def scatter_blocks(bf, per_field, fill=1.0):
    canvas = np.full((bf.info.nby, bf.info.nbx), fill, np.float32)
    for (by, bx, nby, nbx), v in zip(block_rects(bf), per_field):
        canvas[by:by + nby, bx:bx + nbx] = np.asarray(v, np.float32).reshape(nby, nbx)
    return canvas.ravel()


def test_layout_and_block_statistics():
    fs = fields()
    bf = BatchFiller([v for (_, _, v) in fs], [m for (_, m, _) in fs], 8, seed=3)
    info = bf.info
    assert info.n_slices == len(fs)
    occ = np.zeros((info.height, info.width), np.int32)
    for (y0, x0, h, w), (z, m, v) in zip(bf.layout, fs):
        assert (h, w) == m.shape and (y0 + x0) % 2 == 0 and y0 % 8 == 0 and x0 % 8 == 0
        occ[y0:y0 + h, x0:x0 + w] += 1
    assert occ.max() == 1
    n = info.nblk
    Es, Nsp, Nb, ma, ng = (np.zeros(n), np.zeros(n, np.int32), np.zeros(n, np.int32),
                           np.zeros(n, np.float32), np.zeros(n, np.int32))
    mpr.mpr_get_block_stats(bf.ctx, Es, Nsp, Nb, ma, ng)
    for k, (z, m, v) in enumerate(fs):
        gf = GapFiller(v, m, 8, seed=3, slice_id=k)
        e1, nsp1, nb1, ma1, ng1 = gf.block_stats()
        np.testing.assert_allclose(bf.block_slice(k, Es), e1, rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(bf.block_slice(k, Nsp), nsp1)
        np.testing.assert_array_equal(bf.block_slice(k, Nb), nb1)
        np.testing.assert_array_equal(bf.block_slice(k, ng), ng1)
        np.testing.assert_allclose(bf.block_slice(k, ma), ma1, rtol=1e-6, atol=1e-7)
        gf.close()
    bf.close()


@pytest.mark.parametrize("storage", [0, 1])
def test_fields_compute_what_they_compute_alone(storage):
    fs = fields()
    R = 6
    rng = np.random.default_rng(5)
    bf = BatchFiller([v for (_, _, v) in fs], [m for (_, m, _) in fs], 8, seed=9, slice_id=20,
                     n_max=60, storage=storage)
    Ts = [rng.uniform(0.03, 0.4, nby * nbx).astype(np.float32)
          for (_, _, nby, nbx) in block_rects(bf)]
    bf.set_temperatures(scatter_blocks(bf, Ts))
    bf.simulate(R)
    preds, errs = bf.predict([z for (z, _, _) in fs])
    for k, (z, m, v) in enumerate(fs):
        gf = GapFiller(v, m, 8, seed=9, slice_id=20 + k, n_max=60, storage=storage)
        gf.set_temperatures(Ts[k])
        gf.simulate(R)
        p1, (a1, r1) = gf.predict(z)
        gf.close()
        g = m != 0
        scale = float(z[m == 0].max() - z[m == 0].min())
        close = np.abs(preds[k] - p1) <= 1e-5 * scale
        assert close[g].mean() >= 0.98, (k, close[g].mean())
        assert np.array_equal(preds[k][~g], z[~g])
        assert abs(errs[k, 0] - a1) <= 0.02 * a1 + 1e-6
    bf.close()


def test_calibration_per_field():
    fs = fields()
    bf = BatchFiller([v for (_, _, v) in fs], [m for (_, m, _) in fs], 8, seed=2, n_bisect=10,
                     n_eq=6, n_meas=6)
    T = bf.calibrate()
    for k, (z, m, v) in enumerate(fs):
        gf = GapFiller(v, m, 8, seed=2, slice_id=k, n_bisect=10, n_eq=6, n_meas=6)
        T1 = gf.calibrate()
        gf.close()
        Tk = bf.block_slice(k, T)
        assert (np.abs(Tk - T1) <= 1e-6 * T1).mean() >= 0.9, (k, Tk, T1)
    bf.close()


def test_canvas_predict_and_limits():
    fs = fields()
    bf = BatchFiller([v for (_, _, v) in fs], [m for (_, m, _) in fs], 8, seed=1, n_max=20)
    bf.set_temperatures(np.full(bf.info.nblk, 0.1, np.float32))
    bf.simulate(2)
    canvas = np.zeros((bf.info.height, bf.info.width), np.float32)
    mpr.mpr_predict(bf.ctx, canvas)
    inside = np.zeros(canvas.shape, bool)
    preds, _ = bf.predict()
    for (y0, x0, h, w), p in zip(bf.layout, preds):
        inside[y0:y0 + h, x0:x0 + w] = True
        np.testing.assert_array_equal(canvas[y0:y0 + h, x0:x0 + w], p)
    assert (canvas[~inside] == 0).all()
    bf.close()
    # mixed block sizes are refused
    g = [(10, 10, 4), (10, 10, 8)]
    z = np.zeros((10, 10), np.float32)
    m = np.zeros((10, 10), np.uint8)
    with pytest.raises(mpr.MprError):
        mpr.mpr_create_batch(g, [m, m], [z, z])


def test_simulate_graph_equals_host_loop():
    fs = fields()
    outs = []
    for graph in (0, 1):
        bf = BatchFiller([v for (_, _, v) in fs], [m for (_, m, _) in fs], 8, seed=4, n_max=80,
                         sim_graph=graph)
        bf.set_temperatures(np.full(bf.info.nblk, 0.08, np.float32))
        bf.simulate(5)
        outs.append((bf.predict()[0], mpr.mpr_get_info(bf.ctx).gap_updates))
        bf.close()
    for (z, m, v), a, b in zip(fs, outs[0][0], outs[1][0]):
        scale = float(z[m == 0].max() - z[m == 0].min())
        assert (np.abs(a - b) <= 1e-5 * scale)[m != 0].mean() >= 0.98
    assert abs(outs[0][1] - outs[1][1]) <= 0.02 * outs[0][1]


def test_pair_tail_equals_host_loop_on_a_batch():
    """The pair-per-CTA stop tail on a batch of fields (a realization pair's
    units span every field; each field keeps its own per-realization count of
    running targeted blocks) gives the per-launch loop's results."""
    fs = fields()
    outs = []
    for tail in (0, 4096):
        bf = BatchFiller([v for (_, _, v) in fs], [m for (_, m, _) in fs], 8, seed=4, n_max=80,
                         pair_tail=tail)
        bf.set_temperatures(np.full(bf.info.nblk, 0.08, np.float32))
        bf.simulate(5)
        outs.append((bf.predict()[0], mpr.mpr_get_info(bf.ctx).gap_updates))
        bf.close()
    for (z, m, v), a, b in zip(fs, outs[0][0], outs[1][0]):
        scale = float(z[m == 0].max() - z[m == 0].min())
        assert (np.abs(a - b) <= 1e-5 * scale)[m != 0].mean() >= 0.98
    assert abs(outs[0][1] - outs[1][1]) <= max(1, outs[0][1] // 2000)


def test_autotune_picks_a_candidate_and_keeps_results():
    z, m = synth.small_problem(96, 80, 0.5, seed=8)
    v = np.where(m != 0, np.nan, z).astype(np.float32)
    T = np.full(((96 + 7) // 8) * ((80 + 7) // 8), 0.1, np.float32)
    preds = []
    for tune in (False, True):
        gf = GapFiller(v, m, 8, seed=6, n_max=50)
        gf.set_temperatures(T)
        if tune:
            t = mpr.mpr_autotune(gf.ctx, 12, 3)
            assert (t.group, t.form) in {(8, 0), (8, 3), (8, 4), (2, 0)}
            assert all(x > 0 for x in t.ms) and t.trial_ms >= sum(t.ms)
            assert gf.refresh().realizations == 0 and gf.info.gap_updates == 0
        gf.simulate(12)
        preds.append(gf.predict()[0])
        gf.close()
    scale = float(z[m == 0].max() - z[m == 0].min())
    assert (np.abs(preds[0] - preds[1]) <= 1e-5 * scale)[m != 0].mean() >= 0.98


@pytest.mark.parametrize("kind", ["device", "pinned", "mixed"])
def test_host_and_device_buffers_give_the_same_batch(kind):
    """Inputs and outputs in pageable host, pinned host or device memory (host
    buffers go through a contiguous device staging copy, device ones straight
    into the canvas): the same temperatures and predictions, bit for bit."""
    import torch
    fs = fields()
    grids = [(m.shape[0], m.shape[1], 8) for (_, m, _) in fs]
    opts = dict(seed=17, group=8, n_bisect=4, n_eq=3, n_meas=3, n_max=40)

    def run(values, masks, outs_of, truths):
        ctx = mpr.mpr_create_batch(grids, masks, values, mpr.mpr_default_options(**opts))
        try:
            info = mpr.mpr_get_info(ctx)
            T = np.zeros(info.nblk, np.float32)
            mpr.mpr_calibrate(ctx, T)
            mpr.mpr_simulate(ctx, 6)
            outs = outs_of()
            err = np.zeros(2 * len(fs))
            mpr.mpr_predict_batch(ctx, outs, truths, err)
            torch.cuda.synchronize()
            preds = [o.cpu().numpy() if hasattr(o, "cpu") else o for o in outs]
        finally:
            mpr.mpr_destroy(ctx)
        return T, preds, err

    host = run([v for (_, _, v) in fs], [m for (_, m, _) in fs],
               lambda: [np.zeros(m.shape, np.float32) for (_, m, _) in fs],
               [z for (z, _, _) in fs])
    dev = torch.device("cuda", 0)
    if kind == "device":
        vals = [torch.from_numpy(v).to(dev) for (_, _, v) in fs]
        masks = [torch.from_numpy(m).to(dev) for (_, m, _) in fs]
        truths = [torch.from_numpy(z).to(dev) for (z, _, _) in fs]
        outs_of = lambda: [torch.zeros(m.shape, dtype=torch.float32, device=dev) for (_, m, _) in fs]
    elif kind == "pinned":
        vals = [torch.from_numpy(v).pin_memory() for (_, _, v) in fs]
        masks = [torch.from_numpy(m).pin_memory() for (_, m, _) in fs]
        truths = [torch.from_numpy(z).pin_memory() for (z, _, _) in fs]
        outs_of = lambda: [torch.zeros(m.shape, dtype=torch.float32).pin_memory() for (_, m, _) in fs]
    else:   # fields alternate between device and pageable host memory
        vals = [torch.from_numpy(v).to(dev) if k % 2 else v for k, (_, _, v) in enumerate(fs)]
        masks = [m if k % 2 else torch.from_numpy(m).to(dev) for k, (_, m, _) in enumerate(fs)]
        truths = [z for (z, _, _) in fs]
        outs_of = lambda: [torch.zeros(m.shape, dtype=torch.float32, device=dev) if k % 3 == 0
                           else np.zeros(m.shape, np.float32) for k, (_, m, _) in enumerate(fs)]
    other = run(vals, masks, outs_of, truths)
    assert np.array_equal(host[0], other[0])
    for a, b in zip(host[1], other[1]):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    # (AAE / RASE: FP64 sums over atomics, equal up to their order)
    np.testing.assert_allclose(host[2], other[2], rtol=1e-12)
