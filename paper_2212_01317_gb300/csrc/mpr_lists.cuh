// Gap-list entries: the description of one gap site that every half-step
// reads (its coordinates, its block, which of its four neighbours exist and
// are gaps, and which of its bonds another block owns). Shared by the
// block-major lists (mpr_kernels.cu) and the tile-major lists of the staged
// half-step (mpr_tile.cu), so both describe a site identically.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "mpr_internal.h"

namespace mpr {

// A block's sites [x0, x1) x [y0, y1) (clipped to the canvas) and whether the
// block across each edge belongs to the same slice (no bond joins two slices).
struct BlockFrame {
    int b, x0, x1, y0, y1, slice;
    bool l_ok, r_ok, u_ok, d_ok;
};

__device__ __forceinline__ BlockFrame block_frame(const Geom& g, const int32_t* __restrict__ of_block,
                                                  int b) {
    BlockFrame fr;
    fr.b = b;
    const int by = b / g.nbx, bx = b % g.nbx;
    fr.y0 = by * g.lb;
    fr.x0 = bx * g.lb;
    fr.y1 = min(g.H, fr.y0 + g.lb);
    fr.x1 = min(g.W, fr.x0 + g.lb);
    fr.slice = of_block[b];
    fr.l_ok = bx > 0 && of_block[b - 1] == fr.slice;
    fr.r_ok = bx + 1 < g.nbx && of_block[b + 1] == fr.slice;
    fr.u_ok = by > 0 && of_block[b - g.nbx] == fr.slice;
    fr.d_ok = by + 1 < g.nby && of_block[b + g.nbx] == fr.slice;
    return fr;
}

// The site's left or up bond is owned by the neighbouring block.
__device__ __forceinline__ bool block_edge(const BlockFrame& fr, int y, int x) {
    return (x == fr.x0 && fr.l_ok) || (y == fr.y0 && fr.u_ok);
}

// The entry of gap site (y, x) of block fr: .x = y << 16 | x,
// .y = b << META_SHIFT | flags (NB_*: the neighbour exists, i.e. lies in the
// canvas, in the same slice and is not absent; GAP_*: it is a gap site;
// EDGE_L / EDGE_U: the left / up bond belongs to the block on that side).
__device__ __forceinline__ uint2 gap_entry(const Geom& g, const uint8_t* __restrict__ mask,
                                           const BlockFrame& fr, int y, int x) {
    const int64_t i = (int64_t)y * g.W + x;
    uint32_t f = 0;
    const bool hl = (x > fr.x0 || fr.l_ok) && mask[i - 1] != MASK_ABSENT;
    const bool hr = (x + 1 < fr.x1 || fr.r_ok) && mask[i + 1] != MASK_ABSENT;
    const bool hu = (y > fr.y0 || fr.u_ok) && mask[i - g.W] != MASK_ABSENT;
    const bool hd = (y + 1 < fr.y1 || fr.d_ok) && mask[i + g.W] != MASK_ABSENT;
    if (hl) { f |= NB_L; if (mask[i - 1] == MASK_GAP) f |= GAP_L; }
    if (hr) { f |= NB_R; if (mask[i + 1] == MASK_GAP) f |= GAP_R; }
    if (hu) { f |= NB_U; if (mask[i - g.W] == MASK_GAP) f |= GAP_U; }
    if (hd) { f |= NB_D; if (mask[i + g.W] == MASK_GAP) f |= GAP_D; }
    if (hl && x == fr.x0) f |= EDGE_L;
    if (hu && y == fr.y0) f |= EDGE_U;
    return make_uint2(((uint32_t)y << 16) | (uint32_t)x, ((uint32_t)fr.b << META_SHIFT) | f);
}

}  // namespace mpr
