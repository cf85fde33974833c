"""Pins of the oracle's site-specific temperatures (SST, Sec. 2.2.3): block
temperatures smoothed n_s times by the mean over a square of radius r_s
(coordinates clamped to the grid), then used site by site in the updates."""
import numpy as np
import pytest

import oracle
from paper_2212_01317_gb300 import synth


def test_no_pass_is_the_block_map():
    o = oracle.Oracle(10, 13, 4)
    T = np.arange(1, o.nblk + 1, dtype=np.float64) / 10
    ts = o.sst_temperatures(T, 2, 0)
    np.testing.assert_array_equal(ts, T[o.block_index()])


def test_constant_map_stays_constant():
    o = oracle.Oracle(9, 7, 3)
    ts = o.sst_temperatures(np.full(o.nblk, 0.37), 2, 5)
    np.testing.assert_allclose(ts, 0.37, rtol=1e-15)


def test_single_pass_of_a_delta_is_the_box():
    # One hot block of one site (lb = 1) in a cold field: after one pass with
    # r_s = 1 the 3x3 square around it holds 1/9, everything else 0.
    o = oracle.Oracle(7, 7, 1)
    T = np.zeros(o.nblk)
    T[3 * 7 + 3] = 1.0
    ts = o.sst_temperatures(T, 1, 1)
    want = np.zeros((7, 7))
    want[2:5, 2:5] = 1.0 / 9.0
    np.testing.assert_allclose(ts, want, rtol=0, atol=1e-17)


def test_two_passes_of_a_delta_are_the_triangle():
    # Box * box: 1/81 times the number of ways to split an offset into two
    # steps in {-1, 0, 1} per axis, i.e. (3 - |dy|)(3 - |dx|)/81 for |d| <= 2.
    o = oracle.Oracle(9, 9, 1)
    T = np.zeros(o.nblk)
    T[4 * 9 + 4] = 1.0
    ts = o.sst_temperatures(T, 1, 2)
    d = np.abs(np.arange(9) - 4)
    w = np.where(d <= 2, 3 - d, 0).astype(np.float64)
    np.testing.assert_allclose(ts, np.outer(w, w) / 81.0, rtol=1e-15, atol=1e-18)


def test_interior_ramp_is_kept_and_the_edge_is_clamped():
    # T linear in x: a symmetric window keeps it where the window fits; at
    # x = 0 the clamped window averages (2 T(0) + T(1)) / 3 for r_s = 1.
    o = oracle.Oracle(5, 8, 1)
    T = np.tile(0.1 + 0.05 * np.arange(8), 5).astype(np.float64)
    ts = o.sst_temperatures(T, 1, 1)
    np.testing.assert_allclose(ts[:, 1:7], T.reshape(5, 8)[:, 1:7], rtol=1e-14)
    np.testing.assert_allclose(ts[:, 0], (2 * 0.1 + 0.15) / 3, rtol=1e-14)
    np.testing.assert_allclose(ts[:, 7], (2 * 0.45 + 0.40) / 3, rtol=1e-14)


def test_window_is_the_plain_mean_brute_force():
    rng = np.random.default_rng(4)
    o = oracle.Oracle(11, 9, 3)
    T = rng.uniform(0.05, 1.0, o.nblk)
    ts = o.sst_temperatures(T, 2, 3)
    cur = T[o.block_index()]
    for _ in range(3):
        nxt = np.empty_like(cur)
        for y in range(11):
            for x in range(9):
                ys = np.clip(np.arange(y - 2, y + 3), 0, 10)
                xs = np.clip(np.arange(x - 2, x + 3), 0, 8)
                nxt[y, x] = cur[np.ix_(ys, xs)].mean()
        cur = nxt
    np.testing.assert_allclose(ts, cur, rtol=1e-13)


def test_updates_use_the_site_temperature():
    # With the site map equal to the block map, SST updates equal BST ones;
    # raising one gap site's temperature changes that site's acceptance only.
    z, m = synth.small_problem(12, 12, 0.5, seed=2)
    o = oracle.Oracle(12, 12, 4, seed=5)
    phi, _, _, _ = o.transform(z, m)
    st = o.block_stats(phi, m)
    phi0 = o.init_block_mean(phi, m, st)
    T = np.full(o.nblk, 0.05)
    a = phi0.copy()
    o.halfstep(a, m, 0, T, t=1, tag=0, r=0)
    o.use_site_temperatures(T[o.block_index()])
    b = phi0.copy()
    o.halfstep(b, m, 0, T, t=1, tag=0, r=0)
    np.testing.assert_array_equal(a, b)
    ts = T[o.block_index()].copy()
    gaps = np.flatnonzero(((m != 0) & ((np.add.outer(np.arange(12), np.arange(12)) & 1) == 0)).ravel())
    hot = gaps[0]
    ts.ravel()[hot] = 1e6                          # accepts every proposal there
    o.use_site_temperatures(ts)
    c = phi0.copy()
    diag = o.halfstep(c, m, 0, T, t=1, tag=0, r=0, diag=True)
    assert diag.ravel()[hot]["accepted"] == 1
    same = np.ones(144, bool)
    same[hot] = False
    np.testing.assert_array_equal(c.ravel()[same], b.ravel()[same])
    o.use_site_temperatures(None)
