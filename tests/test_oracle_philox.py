"""Pins for the oracle's random numbers.

Philox4x32-10 (Salmon et al., SC'11) is checked against NVIDIA's curand host
generator, an implementation independent of ours: its CPU Philox generator with
seed s emits, for output block j (4 words), Philox4x32-10 with key
(s_lo, s_hi) and counter (j >> 16 as the 64-bit (c0, c1) pair, j & 0xffff, 0).
"""
import ctypes
import ctypes.util
import glob
import os

import numpy as np
import pytest

import oracle

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    cands = []
    for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
              "/usr/local/cuda/targets/x86_64-linux/lib"):
        cands += sorted(glob.glob(os.path.join(d, "libcurand.so*")))
    name = ctypes.util.find_library("curand")
    if name:
        cands.append(name)
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def _curand_words(lib, seed: int, offset_words: int, n: int) -> np.ndarray:
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset_words)) == 0
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
        return out
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 20221203])
@pytest.mark.parametrize("block0", [0, 7, 65530, 65536 * 3 + 11, (1 << 40) + 12345])
def test_philox_matches_curand_host(seed, block0):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    nblocks = 24
    words = _curand_words(lib, seed, 4 * block0, 4 * nblocks).reshape(nblocks, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in range(nblocks):
        blk = block0 + j
        hi = blk >> 16
        ctr = [hi & 0xFFFFFFFF, (hi >> 32) & 0xFFFFFFFF, blk & 0xFFFF, 0]
        got = oracle.philox4x32_10(ctr, key)
        np.testing.assert_array_equal(got, words[j], err_msg=f"block {blk}")


def test_u01_exact_and_open_interval():
    xs = [0, 1, 255, 256, 0x7FFFFFFF, 0x80000000, 0xFFFFFF00, 0xFFFFFFFF, 0x12345678]
    for x in xs:
        u = oracle.u01(x)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u           # exactly representable in FP32
        k = u * 2.0 ** 24
        assert k == int(k) and int(k) % 2 == 1     # odd multiple of 2^-24
    assert oracle.u01(0) == 2.0 ** -24
    assert oracle.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24


def test_site_uniforms_counter_layout():
    """Realization r uses words 2(r&1), 2(r&1)+1 of counter (i, t | tag<<16, r>>1, 0)."""
    o = oracle.Oracle(8, 8, 4, seed=0xDEADBEEF12345678, slice_id=3)
    key = [0x12345678, 0xDEADBEEF ^ 3]
    for (i, t, tag, r) in [(0, 1, 0, 0), (5, 7, 0, 1), (63, 200, 3, 6), (17, 45, 24, 9)]:
        w = oracle.philox4x32_10([i, t | (tag << 16), r >> 1, 0], key)
        o_ = 2 * (r & 1)
        assert o.site_uniforms(i, t, tag, r) == (oracle.u01(w[o_]), oracle.u01(w[o_ + 1]))


def test_uniforms_are_uniform():
    """Kolmogorov-Smirnov on 20000 proposal draws over sites and sweeps."""
    from scipy import stats
    o = oracle.Oracle(100, 100, 10, seed=99)
    u = np.array([o.site_uniforms(i, t, 0, 0)[0] for i in range(2000) for t in range(1, 11)])
    assert stats.kstest(u, "uniform").pvalue > 1e-3
