"""Pins for Eq. 1 / Eq. 2 and the owned-bond block attribution of Sec. 2.2.2.

The expected numbers in the two hand examples are worked out by hand in the
comments below (angles chosen so that every cos(q dphi) is 1, 1/2, 0, -1/2 or
-1), independently of the oracle's loops.
"""
import numpy as np
import pytest

import oracle

PI = np.pi


def brute_total_energy(phi, q=0.5, J=1.0):
    """Eq. 1 summed over unordered nearest-neighbour pairs via array differences."""
    h = -J * np.cos(q * (phi[:, :-1] - phi[:, 1:])).sum()
    v = -J * np.cos(q * (phi[:-1, :] - phi[1:, :])).sum()
    return h + v


def test_hand_example_3x3_lb2():
    # Angles k * 2pi/3, so q*dphi = (pi/3) dk and -cos gives -1, -1/2, +1/2, +1.
    k = np.array([[0, 1, 2], [3, 0, 1], [2, 3, 0]], dtype=np.float64)
    phi = k * 2 * PI / 3
    mask = np.array([[0, 0, 1], [0, 1, 0], [0, 0, 0]], dtype=np.uint8)
    o = oracle.Oracle(3, 3, 2)
    st = o.block_stats(phi, mask)
    # Block 0 (rows 0-1, cols 0-1) owns 8 bonds; its energy is
    # (-1/2 + 1) + (-1/2 - 1/2) + (1 - 1/2) + (-1/2 + 1) = 1/2. Sample pairs:
    # (0,0)-(0,1) -1/2, (0,0)-(1,0) +1, (1,0)-(2,0) -1/2 -> E_s = 0, N_SP = 3.
    # Block 1 (rows 0-1, col 2) owns the two down bonds (-1/2 each); the only
    # sample pair is (1,2)-(2,2) -> E_s = -1/2, N_SP = 1.
    # Block 2 (row 2, cols 0-1) owns (2,0)-(2,1) -1/2 and (2,1)-(2,2) +1, both
    # sample pairs -> E_s = 1/2, N_SP = 2. Block 3 (corner site) owns nothing.
    np.testing.assert_array_equal(st.Nb, [8, 2, 2, 0])
    np.testing.assert_array_equal(st.Nsp, [3, 1, 2, 0])
    np.testing.assert_allclose(st.Es, [0.0, -0.5, 0.5, 0.0], atol=1e-12)
    np.testing.assert_allclose(o.block_energy(phi), [0.5, -1.0, 0.5, 0.0], atol=1e-12)
    np.testing.assert_array_equal(st.n_gap, [1, 1, 0, 0])
    np.testing.assert_array_equal(st.n_sample, [3, 1, 2, 1])
    # Sample mean angles: k = (0+1+3)/3, 1, (2+3)/2, 0; global (0+1+3+1+2+3+0)/7.
    np.testing.assert_allclose(st.mean_angle, np.array([4 / 3, 1, 2.5, 0]) * 2 * PI / 3,
                               atol=1e-12)
    assert abs(st.global_mean - (10 / 7) * 2 * PI / 3) < 1e-12
    assert abs(o.total_energy(phi)) < 1e-12


def test_hand_example_4x5_lb3_partial_blocks():
    # Angles k * pi with k in {0,1,2}: -cos(q dphi) is -1 (dk=0), 0 (dk=1), +1 (dk=2).
    k = np.array([[0, 1, 2, 0, 1],
                  [1, 1, 0, 2, 2],
                  [2, 0, 0, 1, 0],
                  [0, 2, 1, 1, 2]], dtype=np.float64)
    phi = k * PI
    mask = np.array([[0, 0, 0, 1, 0],
                     [0, 1, 0, 0, 0],
                     [0, 0, 0, 0, 1],
                     [1, 0, 0, 0, 0]], dtype=np.uint8)
    o = oracle.Oracle(4, 5, 3)
    st = o.block_stats(phi, mask)
    # Block 0 (3x3) owns 18 bonds, including the ones that leave it to the
    # right (col 2 -> col 3) and down (row 2 -> row 3). Per site (right+down):
    # 0, -1, 2, -1, 0, 0, 2, 0, 0 -> E = 2. Its 12 sample pairs sum to 2.
    # Block 1 (3x2) owns 9 bonds: 1, 0, -1, 1, -1, 1 per site -> E = 1; sample
    # pairs (0,4)D 0, (1,3)R -1, (1,3)D 0, (2,3)D -1 -> E_s = -2, N_SP = 4.
    # Block 2 (1x3) owns 3 right bonds +1, 0, -1 -> E = 0; sample pairs 0, -1.
    # Block 3 (1x2) owns one bond, 0, a sample pair.
    np.testing.assert_array_equal(st.Nb, [18, 9, 3, 1])
    np.testing.assert_array_equal(st.Nsp, [12, 4, 2, 1])
    np.testing.assert_allclose(st.Es, [2.0, -2.0, -1.0, 0.0], atol=1e-12)
    np.testing.assert_allclose(o.block_energy(phi), [2.0, 1.0, 0.0, 0.0], atol=1e-12)
    np.testing.assert_array_equal(st.n_gap, [1, 2, 1, 0])
    np.testing.assert_allclose(st.mean_angle, [0.75 * PI, 1.5 * PI, 1.5 * PI, 1.5 * PI],
                               atol=1e-12)
    assert abs(o.total_energy(phi) - 3.0) < 1e-12


@pytest.mark.parametrize("H,W,lb", [(1, 1, 1), (1, 7, 3), (7, 1, 2), (9, 13, 4), (16, 16, 8),
                                    (33, 17, 16), (20, 20, 32)])
def test_bond_count_and_energy_partition(H, W, lb):
    rng = np.random.default_rng(H * 100 + W)
    phi = rng.uniform(0, 2 * PI, (H, W))
    mask = (rng.uniform(size=(H, W)) < 0.4).astype(np.uint8)
    o = oracle.Oracle(H, W, lb)
    st = o.block_stats(phi, mask)
    assert st.Nb.sum() == 2 * H * W - H - W
    E = o.block_energy(phi)
    assert abs(E.sum() - brute_total_energy(phi)) < 1e-9
    assert abs(o.total_energy(phi) - brute_total_energy(phi)) < 1e-9
    # Sample-sample pairs: count and energy against a brute-force pair scan.
    s = mask == 0
    hp = s[:, :-1] & s[:, 1:]
    vp = s[:-1, :] & s[1:, :]
    assert st.Nsp.sum() == hp.sum() + vp.sum()
    es_tot = (-np.cos(0.5 * (phi[:, :-1] - phi[:, 1:]))[hp]).sum() + \
             (-np.cos(0.5 * (phi[:-1, :] - phi[1:, :]))[vp]).sum()
    assert abs(st.Es.sum() - es_tot) < 1e-9
    assert st.n_gap.sum() == mask.sum() and st.n_sample.sum() == s.sum()


def test_transform_roundtrip_and_copy():
    rng = np.random.default_rng(5)
    z = rng.normal(size=(12, 9)).astype(np.float32)
    mask = (rng.uniform(size=z.shape) < 0.5).astype(np.uint8)
    phi, zmin, zmax, deg = oracle.Oracle.transform(z, mask)
    s = mask == 0
    assert not deg
    assert zmin == float(z[s].min()) and zmax == float(z[s].max())
    assert phi[s].min() == 0.0 and abs(phi[s].max() - 2 * PI) < 1e-15
    # Back-transform of the data angles returns the data (round trip).
    back = zmin + (zmax - zmin) * phi / (2 * PI)
    np.testing.assert_allclose(back[s], z[s], rtol=0, atol=1e-6)
    # Prediction copies samples bitwise and keeps gaps inside [zmin, zmax].
    mean_phi = np.where(s, phi, rng.uniform(0, 2 * PI, z.shape))
    pred = oracle.Oracle.backtransform(mean_phi, mask, z, zmin, zmax)
    assert np.array_equal(pred[s].view(np.uint32), z[s].view(np.uint32))
    assert pred[~s].min() >= np.float32(zmin) and pred[~s].max() <= np.float32(zmax)


def test_transform_degenerate_constant_data():
    z = np.full((4, 4), 3.5, dtype=np.float32)
    mask = np.zeros((4, 4), np.uint8)
    mask[1, 2] = 1
    phi, zmin, zmax, deg = oracle.Oracle.transform(z, mask)
    assert deg and zmin == zmax == 3.5 and np.all(phi == 0)
    pred = oracle.Oracle.backtransform(np.zeros((4, 4)), mask, z, zmin, zmax)
    assert np.all(pred == 3.5)


def test_scores_eqs_3_4():
    truth = np.array([1, 2, 3, 4], dtype=np.float32)
    pred = np.array([1, 0, 3, 7], dtype=np.float32)
    mask = np.array([0, 1, 0, 1], dtype=np.uint8)
    aae, rase = oracle.Oracle.scores(pred, truth, mask)
    assert aae == pytest.approx((2 + 3) / 2)
    assert rase == pytest.approx(np.sqrt((4 + 9) / 2))
