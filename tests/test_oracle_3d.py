"""Pins of the oracle's 3-D grids (6-neighbour stencil, cubic blocks).

The 3-D functions are written separately from the 2-D ones (only the update
arithmetic given a site's neighbours is shared), so the reductions pin them:
a grid one layer deep is the 2-D grid, and a grid one site wide and high is
a 2-D column (bonds along z there are the 2-D bonds along y, with the same
site indices, blocks and random numbers). The rest is checked against
brute force: bond counts, the energy partition over blocks, every update's
dE against the change of the total energy, and the colour of updated sites.
"""
import numpy as np
import pytest

import oracle
from paper_2212_01317_gb300 import synth


def field3(D, H, W, p, seed):
    rng = np.random.default_rng(seed)
    z = rng.normal(size=(D, H, W)).cumsum(axis=2).astype(np.float32)
    m = (rng.uniform(size=(D, H, W)) < p).astype(np.uint8)
    return z, m


def total_energy3(phi, q=0.5, J=1.0):
    e = 0.0
    for ax in range(3):
        a = np.moveaxis(phi, ax, 0)
        e += -J * np.cos(q * (a[1:] - a[:-1])).sum()
    return e


@pytest.mark.parametrize("H,W,lb", [(13, 17, 4), (8, 8, 8), (9, 20, 3)])
def test_one_layer_is_the_2d_grid(H, W, lb):
    z, m = synth.small_problem(H, W, 0.45, seed=H)
    o2 = oracle.Oracle(H, W, lb, seed=77)
    o3 = oracle.Oracle3(1, H, W, lb, seed=77)
    phi, zmin, zmax, _ = o2.transform(z, m)
    s2 = o2.block_stats(phi, m)
    s3 = o3.block_stats(phi[None], m[None])
    for f in ("Es", "Nsp", "Nb", "mean_angle", "n_gap", "n_sample"):
        np.testing.assert_array_equal(getattr(s2, f), getattr(s3, f))
    assert s2.global_mean == s3.global_mean
    p0 = o2.init_block_mean(phi, m, s2)
    np.testing.assert_array_equal(p0[None], o3.init_block_mean(phi[None], m[None], s3))
    np.testing.assert_array_equal(o2.block_energy(p0), o3.block_energy(p0[None]))
    T = np.random.default_rng(1).uniform(0.05, 0.5, o2.nblk)
    for colour in (0, 1):
        a, b = p0.copy(), p0[None].copy()
        d2 = o2.halfstep(a, m, colour, T, t=3, tag=2, r=5, diag=True)
        d3 = o3.halfstep(b, m[None], colour, T, t=3, tag=2, r=5, diag=True)
        np.testing.assert_array_equal(a[None], b)
        np.testing.assert_array_equal(d2["accepted"], d3["accepted"])
    r2 = oracle.gapfill(z, m, lb, R=2, seed=9, n_bisect=3, n_eq=3, n_meas=3, n_max=15)
    r3 = oracle.gapfill3(z[None], m[None], lb, R=2, seed=9, n_bisect=3, n_eq=3, n_meas=3,
                         n_max=15)
    np.testing.assert_array_equal(r2.T, r3.T)
    np.testing.assert_array_equal(r2.pred[None], r3.pred)


def test_one_column_along_z_is_a_2d_column():
    n, lb = 37, 5
    rng = np.random.default_rng(3)
    z = rng.normal(size=n).cumsum().astype(np.float32)
    m = (rng.uniform(size=n) < 0.5).astype(np.uint8)
    o2 = oracle.Oracle(n, 1, lb, seed=11)
    o3 = oracle.Oracle3(n, 1, 1, lb, seed=11)
    phi, *_ = o2.transform(z.reshape(n, 1), m.reshape(n, 1))
    s2 = o2.block_stats(phi, m.reshape(n, 1))
    s3 = o3.block_stats(phi.reshape(n, 1, 1), m.reshape(n, 1, 1))
    for f in ("Es", "Nsp", "Nb", "n_gap"):
        np.testing.assert_array_equal(getattr(s2, f), getattr(s3, f))
    p0 = o2.init_block_mean(phi, m.reshape(n, 1), s2)
    T = np.full(o2.nblk, 0.2)
    for r in range(3):
        a, _, ta, _ = o2.simulate_one(p0, m.reshape(n, 1), T, s2, 40, r)
        b, _, tb = o3.simulate_one(p0.reshape(n, 1, 1), m.reshape(n, 1, 1), T, s3, 40, r)
        np.testing.assert_array_equal(a.ravel(), b.ravel())
        assert ta == tb


def test_bond_counts_and_energy_partition():
    D, H, W, lb = 5, 7, 6, 3
    z, m = field3(D, H, W, 0.4, 2)
    o = oracle.Oracle3(D, H, W, lb, seed=1)
    phi, *_ = oracle.Oracle.transform(z.reshape(D * H, W), m.reshape(D * H, W))
    phi = phi.reshape(D, H, W)
    st = o.block_stats(phi, m)
    assert st.Nb.sum() == 3 * D * H * W - H * W - D * W - D * H
    assert (st.n_gap + st.n_sample).sum() == D * H * W
    np.testing.assert_allclose(o.block_energy(phi).sum(), total_energy3(phi), rtol=1e-12)
    # sample-sample bonds only, by brute force
    es = 0.0
    for ax in range(3):
        a = np.moveaxis(phi, ax, 0)
        ma = np.moveaxis(m, ax, 0)
        both = (ma[1:] == 0) & (ma[:-1] == 0)
        es += (-np.cos(0.5 * (a[1:] - a[:-1])))[both].sum()
    np.testing.assert_allclose(st.Es.sum(), es, rtol=1e-12)
    # hand count: a single 2 x 2 x 2 block of samples owns 12 bonds
    o2 = oracle.Oracle3(2, 2, 2, 2)
    s2 = o2.block_stats(np.zeros((2, 2, 2)), np.zeros((2, 2, 2), np.uint8))
    assert s2.Nb[0] == 12 and s2.Nsp[0] == 12 and s2.Es[0] == -12.0


def test_updates_change_the_total_energy_by_de_and_keep_their_colour():
    D, H, W, lb = 4, 6, 5, 2
    z, m = field3(D, H, W, 0.6, 4)
    o = oracle.Oracle3(D, H, W, lb, seed=5, overrelax=False)
    phi = np.random.default_rng(0).uniform(0, 2 * np.pi, (D, H, W))
    T = np.full(o.nblk, 0.3)
    for i in np.flatnonzero(m.ravel())[:40]:
        before = total_energy3(phi)
        trial = phi.copy()
        d = o.update_site(trial, m, int(i), 0.3, 2, 0, 1)
        prop = phi.copy()
        prop.ravel()[i] = d.phi_prop
        assert abs(d.dE - (total_energy3(prop) - before)) < 1e-9
    cz, cy, cx = np.mgrid[0:D, 0:H, 0:W]
    for colour in (0, 1):
        a = phi.copy()
        o.halfstep(a, m, colour, T, t=1, tag=0, r=0)
        moved = a != phi
        assert not (moved & (m == 0)).any()
        assert not (moved & (((cx + cy + cz) & 1) != colour)).any()
