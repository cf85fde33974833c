"""The 16-bit state forms (BF16 / FP16 storage of the realizations' angles,
FP32 arithmetic, FP64 block energies), through the C-ABI.

What must hold exactly, whatever the storage:
  * the incremental block energies equal the energies recomputed in FP64
    from the stored state (the kernels round every proposal and reflection
    to the stored type before taking its energy, and account the reflection's
    rounding), also after 200 sweeps of 64 x 64 blocks against the oracle's
    block energy;
  * stored gap angles are values of the storage type, in [0, 2pi];
  * sample sites keep their FP32 angle bit for bit.
What is stated, not exact: the error of the predictions against the FP64
oracle (same random streams; a rounded proposal can flip a decision, so the
chains separate), checked at equal AAE within the Monte Carlo spread.
"""
import numpy as np
import pytest

import oracle
from paper_2212_01317_gb300 import synth
from paper_2212_01317_gb300.mpr import GapFiller

from parity import TWO_PI

pytestmark = pytest.mark.gpu
STORE = {"f32": 0, "bf16": 1, "f16": 2}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def make(z, m, lb, **opt):
    v = np.where(m != 0, np.nan, z).astype(np.float32)
    return GapFiller(v, m, lb, **opt)


def representable(x: np.ndarray, storage: str) -> bool:
    x = np.asarray(x, np.float32)
    if storage == "f32":
        return True
    if storage == "f16":
        return np.array_equal(x.astype(np.float16).astype(np.float32), x)
    return bool(np.all((x.view(np.uint32) & 0xFFFF) == 0))


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("group,R", [(2, 1), (8, 6)])
def test_incremental_energy_equals_recomputed(storage, group, R):
    z, m = synth.small_problem(48, 40, 0.55, seed=13)
    gf = make(z, m, 8, seed=3, storage=STORE[storage], group=group, n_max=200)
    rng = np.random.default_rng(1)
    gf.set_temperatures(rng.uniform(0.03, 0.3, gf.nblk).astype(np.float32))
    gf.sim_begin(R)
    Es, Nsp, Nb, _, _ = gf.block_stats()
    for _ in range(3):
        gf.sim_sweep(4)
        e = gf.block_e(R)
        _, run = gf.get_stop(R)
        for r in range(R):
            E = gf.block_energy(r)
            ok = (run[r] == 1) & (Nb > 0)
            np.testing.assert_allclose(e[r][ok], E[ok] / Nb[ok], rtol=0, atol=5e-6)
    for r in range(R):
        s = gf.get_state(r)
        g = m != 0
        assert representable(s[g], storage)
        assert s[g].min() >= 0.0 and s[g].max() <= TWO_PI
    gf.sim_end()
    gf.close()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_samples_stay_exact(storage):
    z, m = synth.small_problem(33, 47, 0.4, seed=2, kind="disc")
    ref = make(z, m, 8, seed=3)
    ref.set_temperatures(np.full(ref.nblk, 0.1, np.float32))
    ref.sim_begin(2)
    base = ref.get_state(0)
    ref.sim_end()
    ref.close()
    gf = make(z, m, 8, seed=3, storage=STORE[storage])
    gf.set_temperatures(np.full(gf.nblk, 0.1, np.float32))
    gf.sim_begin(3)
    gf.sim_sweep(5)
    for r in range(3):
        s = gf.get_state(r)
        assert np.array_equal(s[m == 0].view(np.uint32), base[m == 0].view(np.uint32))
    gf.sim_end()
    gf.close()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_prediction_error_against_fp64_oracle(storage, record_property):
    """Equal AAE within the spread over seeds; the mean absolute difference
    of the predictions from the FP64 oracle's is recorded."""
    H, W, lb, R = 48, 48, 8, 8
    z, m = synth.small_problem(H, W, 0.5, seed=61, xi=6.0)
    T = np.full((H // lb) * (W // lb), 0.08, np.float32)
    d_aae, diffs = [], []
    for s in range(6):
        gf = make(z, m, lb, seed=500 + s, n_max=60, storage=STORE[storage])
        gf.set_temperatures(T)
        gf.simulate(R)
        pred, (aae, _) = gf.predict(truth=z)
        gf.close()
        ref = oracle.gapfill(z, m, lb, R=R, seed=500 + s, T_blk=T.astype(np.float64), n_max=60)
        a_ref = oracle.Oracle.scores(ref.pred, z, m)[0]
        d_aae.append(aae - a_ref)
        g = m != 0
        diffs.append(np.abs(pred[g] - ref.pred[g]).mean() / (z.max() - z.min()))
    d = np.array(d_aae)
    se = max(d.std(ddof=1) / np.sqrt(len(d)), 1e-12)
    record_property("mean_abs_pred_diff_over_range", float(np.mean(diffs)))
    record_property("aae_diff_mean", float(d.mean()))
    assert abs(d.mean()) <= 3 * se + 0.005 * abs(a_ref)
    assert np.mean(diffs) < 0.05


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("group,R", [(2, 2), (8, 11)])
@pytest.mark.parametrize("colour", [0, 1])
def test_halfstep_lockstep_precision_form(storage, group, R, colour):
    """One half-step of the 16-bit forms against the oracle in the same
    precision form (proposal = the FP32 product 2pi u0 rounded to the stored
    type before its energy is taken; reflected angle rounded), element by
    element from the same random states and Philox draws."""
    from parity import checkerboard, compare_site_updates
    H, W, lb = 45, 38, 8
    st_code = STORE[storage]
    z, m = synth.small_problem(H, W, 0.55, seed=7 + colour)
    gf = make(z, m, lb, seed=0x1234567, storage=st_code, group=group)
    o = oracle.Oracle(H, W, lb, seed=0x1234567, storage=st_code)
    rng = np.random.default_rng(17)
    T = rng.uniform(0.02, 1.2, gf.nblk).astype(np.float32)
    gf.set_temperatures(T)
    gf.sim_begin(R)
    g = m != 0
    pre = []
    for r in range(R):
        s = gf.get_state(r)
        s[g] = rng.uniform(0, TWO_PI, int(g.sum())).astype(np.float32)
        gf.set_state(r, s)
        back = gf.get_state(r)            # as stored: rounded to the type
        assert all(oracle.round_store(v, st_code) == v for v in back[g].astype(np.float64))
        pre.append(back)
    running = (rng.uniform(size=(R, gf.nblk)) < 0.75).astype(np.uint8)
    gf.set_running(running)
    t, tag = 9, 2
    gf.halfstep(colour, t, tag)
    blk = o.block_index()
    cb = checkerboard(H, W)
    total = flips = 0
    for r in range(R):
        post = gf.get_state(r)
        ph = pre[r].astype(np.float64)
        diag = o.halfstep(ph, m, colour, T.astype(np.float64), running[r], t=t, tag=tag, r=r,
                          diag=True).reshape(H, W)
        may = g & (cb == colour) & (running[r][blk] == 1)
        n, f, bad, msg = compare_site_updates(post, ph, pre[r], diag, may, storage=st_code)
        assert bad == 0, f"r={r}: {msg}"
        total += n
        flips += f
    assert total > 100 * R
    assert flips <= max(3, total // 500)
    gf.sim_end()
    gf.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_energy_drift_over_200_sweeps_at_large_blocks(storage):
    """The block energies that drive the stop test stay those of the state
    over a long run with large blocks (l_b = 64: about 8 k bonds per block):
    every (block, realization) pair is kept running for 200 sweeps, and the
    incrementally summed e_b (FP32 move energies, FP64 sums) is compared with
    the block energy the oracle computes in FP64 from the stored state.
    Bound: each move's dE carries the error of FP32 arithmetic on hardware
    sin/cos (|error| <~ 1e-6); over 200 sweeps of ~2.9 k gap sites per block
    and colour the errors add like a random walk to ~1e-3 in E_b, ~1e-7 per
    bond; the test allows 1e-6 per bond."""
    H, W, lb, R = 128, 192, 64, 8
    z, m = synth.small_problem(H, W, 0.7, seed=23, kind="disc")
    gf = make(z, m, lb, seed=17, storage=STORE[storage], group=8, n_max=65535)
    gf.set_temperatures(np.random.default_rng(4).uniform(0.05, 0.4, gf.nblk).astype(np.float32))
    gf.sim_begin(R)
    Es, Nsp, Nb, _, _ = gf.block_stats()
    every = np.ones((R, gf.nblk), np.uint8)
    for _ in range(200):
        gf.sim_sweep(1)
        gf.set_running(every)
    e = gf.block_e(R)
    o = oracle.Oracle(H, W, lb, seed=17)
    worst = 0.0
    for r in range(R):
        E_o = o.block_energy(gf.get_state(r).astype(np.float64))
        ok = Nb > 0
        worst = max(worst, float(np.max(np.abs(e[r][ok] - E_o[ok] / Nb[ok]))))
    gf.sim_end()
    gf.close()
    assert worst <= 1e-6, worst


def test_stated_error_against_fp64_oracle_config3(record_property):
    """The precision form's error against the FP64 oracle, stated on the
    4096 x 4096 precision workload's recipe (lognormal non-stationary GRF,
    correlation 4 -> 64 cells, disc gaps covering 60 %, l_b = 32, R = 10): a
    band of 384 rows across the whole width (every correlation length). The
    block temperatures are calibrated once on the GPU (FP32) and given to both
    sides; each storage form runs the realizations on the GPU and the oracle
    runs them in FP64 with the same random streams, for two seeds. Stated
    per form: the mean |pred_gpu - pred_oracle| over the gap sites divided by
    the value range, and the AAE and RASE differences. The FP32 form's figures
    are the floor (chains separate where an FP32 decision flips: measured
    0.8 % of the range, AAE within 0.1 %). FP16 keeps 11 significant bits of
    an angle (a step of 2^-8 rad near 2 pi): measured 0.85 % and -0.5 % in
    AAE; the bounds are 1.5 % and 1 %. BF16 keeps 8 (a step of 2^-5 rad near
    2 pi, 0.5 % of the value range): measured 1.6 % and a systematic AAE
    shift of -2 % (RASE +2 %); the bounds are 3 % and 3 %."""
    import json
    import os
    wl = synth.workload("field4096")
    z = np.ascontiguousarray(wl.truth[1856:2240, :])
    m = np.ascontiguousarray(wl.mask[1856:2240, :])
    lb, R = wl.block, wl.realizations
    H, W = m.shape
    cal = make(z, m, lb, seed=99, cal_points=2, n_bisect=16)
    T = cal.calibrate()
    cal.close()
    g = m != 0
    zr = float(z[~g].max() - z[~g].min())
    out = {}
    for seed in (901, 902):
        ref = oracle.gapfill(z, m, lb, R=R, seed=seed, T_blk=T.astype(np.float64), threads=0)
        a_o, r_o = oracle.Oracle.scores(ref.pred, z, m)
        for storage in ("f32", "bf16", "f16"):
            gf = make(z, m, lb, seed=seed, storage=STORE[storage])
            gf.set_temperatures(T)
            gf.simulate(R)
            pred, (aae, rase) = gf.predict(truth=z)
            gf.close()
            d = out.setdefault(storage, {"pred_diff_over_range": [], "aae_diff": [],
                                         "rase_diff": [], "aae_oracle": []})
            d["pred_diff_over_range"].append(float(np.abs(pred[g] - ref.pred[g]).mean() / zr))
            d["aae_diff"].append(float(aae - a_o))
            d["rase_diff"].append(float(rase - r_o))
            d["aae_oracle"].append(float(a_o))
    for storage, d in out.items():
        for k, v in d.items():
            record_property(f"{storage}_{k}", float(np.mean(v)))
    rec = os.environ.get("MPR_RECORD_DIR")
    if rec:
        os.makedirs(rec, exist_ok=True)
        with open(os.path.join(rec, "precision_error_field4096.json"), "w") as f:
            json.dump({"workload": f"{wl.name} rows 1856-2239 (384 x 4096)", "R": R,
                       "seeds": [901, 902], "forms": out}, f, indent=1)
    bounds = {"f32": (0.002, 0.012), "f16": (0.01, 0.015), "bf16": (0.03, 0.03)}
    for storage, (b_aae, b_pred) in bounds.items():
        d = out[storage]
        assert abs(np.mean(d["aae_diff"])) <= b_aae * np.mean(d["aae_oracle"]), storage
        assert np.mean(d["pred_diff_over_range"]) < b_pred, storage
