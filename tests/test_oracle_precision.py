"""Pins of the oracle's precision form (stored gap angles in BF16 or FP16,
the task's precision option): the rounding to the stored type, checked
against numpy's own FP16 conversion and against the definition of
round-to-nearest-even for BF16 (no formula is retyped), and the chain in
that form: updated gap angles are values of the stored type, samples and
the other colour never move, and the exact form is unchanged."""
import numpy as np
import pytest

import oracle

TWO_PI = 2.0 * np.pi


def _f32_bits(x):
    return np.asarray(x, np.float32).view(np.uint32)


def test_fp16_rounding_matches_numpy():
    rng = np.random.default_rng(0)
    vals = np.concatenate([
        rng.uniform(0, TWO_PI, 4000),
        rng.uniform(0, 1e-4, 2000),                    # FP16 subnormals and the normal edge
        10.0 ** rng.uniform(-9, 0.8, 2000),
        np.array([0.0, 6.103515625e-05, 5.9604644775390625e-08, 2.9802322387695312e-08,
                  TWO_PI]),
    ])
    # exact ties between FP16 neighbours, in the normal and the subnormal range
    h = np.arange(1, 3000, dtype=np.uint16).view(np.float16).astype(np.float64)
    ties = (h[:-1] + h[1:]) / 2
    h2 = (np.arange(0x3C00, 0x4600, 7, dtype=np.uint16)).view(np.float16).astype(np.float64)
    ties = np.concatenate([ties, h2 + np.spacing(np.float16(h2)).astype(np.float64) / 2])
    for v in np.concatenate([vals, ties]):
        want = float(np.float16(np.float32(v)))
        assert oracle.round_store(v, 2) == want, v


def test_bf16_rounding_is_nearest_even():
    rng = np.random.default_rng(1)
    vals = np.concatenate([rng.uniform(0, TWO_PI, 5000), 10.0 ** rng.uniform(-8, 0.8, 2000)])
    # exact ties: FP32 values with the low 16 bits 0x8000
    base = rng.integers(0x30000000, 0x40C90000, 500, dtype=np.uint32) & 0xFFFF0000
    ties = (base | 0x8000).view(np.float32).astype(np.float64)
    for v in np.concatenate([vals, ties]):
        f = np.float32(v)
        r = oracle.round_store(v, 1)
        rb = int(_f32_bits(r))
        assert rb & 0xFFFF == 0, v                          # a BF16 value
        lo = int(_f32_bits(f)) & 0xFFFF0000                 # the two BF16 neighbours of f
        hi = lo + 0x10000
        flo = float(np.uint32(lo).view(np.float32))
        fhi = float(np.uint32(hi).view(np.float32))
        assert rb in (lo, hi), v
        dlo, dhi = abs(float(f) - flo), abs(float(f) - fhi)
        if dlo != dhi:
            assert rb == (lo if dlo < dhi else hi), v
        else:
            assert (rb >> 16) & 1 == 0, v                   # tie: the even one


def test_exact_form_is_the_identity():
    for v in (0.0, 1e-30, 0.3, TWO_PI):
        assert oracle.round_store(v, 0) == v


@pytest.mark.parametrize("storage", [1, 2])
def test_chain_in_precision_form_stores_values_of_the_type(storage):
    H, W, lb = 24, 20, 4
    rng = np.random.default_rng(5)
    m = (rng.uniform(size=(H, W)) < 0.5).astype(np.uint8)
    phi = rng.uniform(0, TWO_PI, (H, W))
    phi[m != 0] = [oracle.round_store(v, storage) for v in phi[m != 0]]
    o = oracle.Oracle(H, W, lb, seed=11, storage=storage)
    T = rng.uniform(0.05, 0.8, o.nblk)
    cb = (np.add.outer(np.arange(H), np.arange(W)) & 1)
    for t in range(1, 6):
        for c in (0, 1):
            before = phi.copy()
            o.halfstep(phi, m, c, T, None, t=t, tag=0, r=3)
            moved = phi != before
            assert not (moved & ((m == 0) | (cb != c))).any()
            assert moved[(m != 0) & (cb == c)].any()
            g = m != 0
            assert all(oracle.round_store(v, storage) == v for v in phi[g])
            assert phi[g].min() >= 0.0 and phi[g].max() <= TWO_PI
    assert (phi != 0).any()


def test_precision_form_keeps_the_chain_close_to_the_exact_one():
    """Over a few hundred sweeps at moderate T the mean energy per bond of the
    precision-form chain matches the exact chain's within the Monte Carlo
    spread (rounding moves angles by at most half an ulp of the type)."""
    H, W, lb = 24, 24, 8
    rng = np.random.default_rng(2)
    m = (rng.uniform(size=(H, W)) < 0.6).astype(np.uint8)
    z = np.cumsum(rng.normal(size=(H, W)), axis=1) * 0.1
    means = {}
    for storage in (0, 1, 2):
        o = oracle.Oracle(H, W, lb, seed=3, storage=storage)
        phi, *_ = o.transform(z, m)
        T = np.full(o.nblk, 0.3)
        es = []
        for t in range(1, 301):
            for c in (0, 1):
                o.halfstep(phi, m, c, T, None, t=t, tag=0, r=0)
            if t > 50:
                es.append(o.block_energy(phi).sum())
        means[storage] = (np.mean(es), np.std(es) / np.sqrt(len(es) / 10))
    for storage in (1, 2):
        d = abs(means[storage][0] - means[0][0])
        assert d < 4 * np.hypot(means[storage][1], means[0][1]) + 1e-3 * abs(means[0][0])
