// Eq. 2 per block: the sample-bond energy E_s,b, its bond count N_SP,b, the
// owned bonds N_b, and the block's sample-angle sum, sample count and gap
// counts per colour. One warp per block; lane l takes the block's sites l,
// l + 32, ... and every site owns its right and down bonds (a bond belongs to
// the block of its left / upper site). Sums in FP64, then over the warp.
//
// Shared by the context path (k_block_stats: canvas masks, where 2 marks an
// absent site and no bond reaches one) and the allocation-free entry point
// (k_na_block_stats: the caller's mask, nonzero = gap), so both compute the
// statistics with the same arithmetic in the same order.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "mpr_internal.h"

namespace mpr {

struct BlockSums {
    double es, sm;               // E_s,b; sum of the sample angles
    int nsp, nb, ns, g0, g1;     // N_SP,b, N_b, samples, gaps of colour 0 / 1
};

template <bool kCanvas>
__device__ __forceinline__ void owned_bond(const float* __restrict__ values,
                                           const uint8_t* __restrict__ mask, int64_t j, bool gap,
                                           double pi, double zmin, double scale, double q,
                                           double J, BlockSums& r) {
    const uint8_t mj = mask[j];
    if (kCanvas && mj == MASK_ABSENT) return;
    ++r.nb;
    if (!gap && mj == 0) {
        const double pj = ((double)values[j] - zmin) * scale;
        r.es += -J * cos(q * (pi - pj));
        ++r.nsp;
    }
}

// Sites [x0, x1) x [y0, y1) of a W-wide grid; right_ok / down_ok: the bonds
// across the block's right / lower edge exist. phi = (z - zmin) * scale.
// Every lane of the warp calls it and gets the block's totals.
template <bool kCanvas>
__device__ __forceinline__ BlockSums block_sums(const float* __restrict__ values,
                                                const uint8_t* __restrict__ mask, int W, int y0,
                                                int x0, int y1, int x1, bool right_ok,
                                                bool down_ok, double zmin, double scale, double q,
                                                double J, bool active) {
    BlockSums r{0.0, 0.0, 0, 0, 0, 0, 0};
    const int lane = threadIdx.x & 31;
    const int bw = x1 - x0, nsite = (y1 - y0) * bw;
    for (int j = lane; j < nsite && active; j += 32) {
        const int y = y0 + j / bw, x = x0 + j % bw;
        const int64_t i = (int64_t)y * W + x;
        const uint8_t mi = mask[i];
        if (kCanvas && mi == MASK_ABSENT) continue;
        const bool gap = kCanvas ? mi == MASK_GAP : mi != 0;
        const double pi = gap ? 0.0 : ((double)values[i] - zmin) * scale;
        if (gap) {
            if (((x + y) & 1) == 0) ++r.g0; else ++r.g1;
        } else {
            r.sm += pi;
            ++r.ns;
        }
        if (x + 1 < x1 || right_ok) owned_bond<kCanvas>(values, mask, i + 1, gap, pi, zmin, scale, q, J, r);
        if (y + 1 < y1 || down_ok) owned_bond<kCanvas>(values, mask, i + W, gap, pi, zmin, scale, q, J, r);
    }
    for (int d = 16; d > 0; d >>= 1) {
        r.es += __shfl_xor_sync(0xffffffffu, r.es, d);
        r.sm += __shfl_xor_sync(0xffffffffu, r.sm, d);
        r.nsp += __shfl_xor_sync(0xffffffffu, r.nsp, d);
        r.nb += __shfl_xor_sync(0xffffffffu, r.nb, d);
        r.ns += __shfl_xor_sync(0xffffffffu, r.ns, d);
        r.g0 += __shfl_xor_sync(0xffffffffu, r.g0, d);
        r.g1 += __shfl_xor_sync(0xffffffffu, r.g1, d);
    }
    return r;
}

}  // namespace mpr
