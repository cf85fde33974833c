"""The allocation-free block-statistics entry point, through the C-ABI.

mpr_block_stats_noalloc serves callers that must not allocate device memory
when they call (they reserve all of it up front, cannot afford cudaFree's
device-wide synchronisation on their path, or run under memory pressure). It
works in a scratch array the library keeps on the device, so this file
checks that two calls in a row, on fields of different size and value
range, each give what mpr_create + mpr_get_block_stats give for the same
field, that the shared scratch carries nothing from one call into the next,
that a call (after a warm-up call) allocates no device memory, also on a
non-default stream, and that oversized grids and host pointers are rejected. The file sorts last
so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_2212_01317_gb300 import mpr, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def reference(z, m, lb):
    v = np.where(m != 0, np.nan, z).astype(np.float32)
    gf = mpr.GapFiller(v, m, lb)
    Es, Nsp, Nb, ma, ng = gf.block_stats()
    zr = (gf.info.zmin, gf.info.zmax)
    gf.close()
    return Es, Nsp, Nb, ma, ng, zr


def buffers(torch, z, m, lb):
    """Device inputs and outputs (outputs pre-filled with a marker)."""
    H, W = m.shape
    nblk = ((H + lb - 1) // lb) * ((W + lb - 1) // lb)
    dev = torch.device("cuda")
    v = torch.from_numpy(np.where(m != 0, np.nan, z).astype(np.float32)).to(dev)
    mk = torch.from_numpy(np.ascontiguousarray(m, dtype=np.uint8)).to(dev)
    outs = (torch.full((nblk,), -7.0, dtype=torch.float64, device=dev),
            torch.full((nblk,), -7, dtype=torch.int32, device=dev),
            torch.full((nblk,), -7, dtype=torch.int32, device=dev),
            torch.full((nblk,), -7.0, dtype=torch.float32, device=dev),
            torch.full((nblk,), -7, dtype=torch.int32, device=dev),
            torch.full((2,), -7.0, dtype=torch.float64, device=dev))
    return mk, v, outs


def call(torch, H, W, lb, mk, v, outs, stream=None):
    st = mpr.mpr_block_stats_noalloc(H, W, lb, mk, v, *outs,
                                     cuda_stream=None if stream is None else stream.cuda_stream)
    torch.cuda.synchronize()
    assert st == mpr.MPR_OK
    return tuple(t.cpu().numpy() for t in outs[:5]) + (tuple(outs[5].cpu().numpy()),)


def noalloc(torch, z, m, lb):
    H, W = m.shape
    mk, v, outs = buffers(torch, z, m, lb)
    return call(torch, H, W, lb, mk, v, outs)


def check(got, ref):
    Es, Nsp, Nb, ma, ng, zr = got
    rEs, rNsp, rNb, rma, rng_, rzr = ref
    np.testing.assert_allclose(Es, rEs, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(Nsp, rNsp)
    np.testing.assert_array_equal(Nb, rNb)
    np.testing.assert_array_equal(ng, rng_)
    np.testing.assert_allclose(ma, rma, rtol=1e-6, atol=1e-7)
    assert zr == rzr


def test_two_calls_in_a_row_match_the_context_path(torch_cuda):
    za, ma_ = synth.small_problem(37, 53, 0.45, seed=5)
    zb, mb = synth.small_problem(96, 80, 0.6, seed=9, kind="disc")
    zb = (zb * 40.0 + 1000.0).astype(np.float32)      # another value range
    mb[0:8, 0:8] = 1                                  # a block with no sample
    ref_a = reference(za, ma_, 8)
    ref_b = reference(zb, mb, 16)
    check(noalloc(torch_cuda, za, ma_, 8), ref_a)
    check(noalloc(torch_cuda, zb, mb, 16), ref_b)
    check(noalloc(torch_cuda, za, ma_, 8), ref_a)     # nothing carried over


def test_a_call_allocates_nothing(torch_cuda):
    """After one warm-up call (which may load the library's module onto the
    device), a call on a non-default stream changes neither the device's free
    memory nor the torch allocator's counts, and still gives the context
    path's statistics."""
    torch = torch_cuda
    z, m = synth.small_problem(72, 88, 0.5, seed=13)
    ref = reference(z, m, 8)
    H, W = m.shape
    mk, v, outs = buffers(torch, z, m, 8)
    call(torch, H, W, 8, mk, v, outs)                 # warm-up
    side = torch.cuda.Stream()
    free0, _ = torch.cuda.mem_get_info()
    alloc0, resv0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    for t in outs:
        t.fill_(-7)
    torch.cuda.synchronize()
    got = call(torch, H, W, 8, mk, v, outs, stream=side)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.memory_reserved() == resv0
    check(got, ref)


def test_limits_and_pointer_kinds(torch_cuda):
    dev = torch_cuda.device("cuda")
    small = torch_cuda.zeros(16, device=dev)
    H = W = 512                                       # 512*512 one-cell blocks > the limit
    assert (H * W) > mpr.MPR_NOALLOC_MAX_BLOCKS
    st = mpr.mpr_block_stats_noalloc(H, W, 1, small, small, small, small, small, small, small,
                                     small)
    assert st == mpr.MPR_EINVAL
    z, m = synth.small_problem(8, 8, 0.3, seed=1)
    host = np.zeros(4, np.float64)
    st = mpr.mpr_block_stats_noalloc(8, 8, 4, m, z, host, host, host, host, host, host)
    assert st == mpr.MPR_EINVAL
