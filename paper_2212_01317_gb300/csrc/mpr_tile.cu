// The realizations' checkerboard half-step (Sec. 2.2.2; Eq. 1 energies) with
// the other colour staged in shared memory.
//
// One CTA takes one tile (a rectangle of at most 16 x 32 sites inside one
// temperature block) for the eight realizations of one lane group. It first
// stages, for every other-colour site of the tile and its one-site halo, the
// (cos q phi_j, sin q phi_j) of the eight realizations: a gap neighbour's
// angles come from the batch state, a sample neighbour's from the staging
// table, and a site that is no neighbour (outside the canvas, absent, or in
// another slice) stages zeros. Each staged value is then read by up to four
// gap sites of the tile's own colour, which walk the tile's compacted gap
// list, one thread per (gap site, realization pair). The arithmetic of an
// update is that of the other half-step forms (site_update, add_energy_lu),
// on the same random numbers, so the forms agree bit for bit up to the order
// of the FP32 energy sums.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mpr_device.cuh"
#include "mpr_internal.h"
#include "mpr_launch.h"
#include "mpr_lists.cuh"
#include "mpr_sweep.cuh"

namespace mpr {

namespace {

constexpr int kTileThreads = 128;
constexpr int kTileWarps = kTileThreads / 32;
constexpr int kStageSites = kTileStageRows * kTileStageCols;

// Sites of tile t and of its staged halo.
struct TileFrame {
    int b;                   // block
    int ty0, ty1, tx0, tx1;  // the tile's sites [tx0, tx1) x [ty0, ty1)
    int hx_lo, ncol, nrow;   // staged half-columns hx_lo .. hx_lo + ncol - 1, rows ty0 - 1 .. ty1
    bool l_ok, r_ok, u_ok, d_ok;  // the sites just across each side are bonded neighbours
};

__device__ __forceinline__ TileFrame tile_frame(const Geom& g, const Tiles& tl,
                                                const int32_t* __restrict__ of_block, int t) {
    TileFrame tf;
    const int tpb = tl.tpx * tl.tpy;
    tf.b = t / tpb;
    const int j = t - tf.b * tpb;
    const int jy = j / tl.tpx, jx = j - jy * tl.tpx;
    const BlockFrame fr = block_frame(g, of_block, tf.b);
    tf.ty0 = fr.y0 + jy * tl.th;
    tf.ty1 = min(fr.y1, tf.ty0 + tl.th);
    tf.tx0 = fr.x0 + jx * tl.tw;
    tf.tx1 = min(fr.x1, tf.tx0 + tl.tw);
    tf.l_ok = tf.tx0 > fr.x0 || fr.l_ok;
    tf.r_ok = tf.tx1 < fr.x1 || fr.r_ok;
    tf.u_ok = tf.ty0 > fr.y0 || fr.u_ok;
    tf.d_ok = tf.ty1 < fr.y1 || fr.d_ok;
    tf.hx_lo = (tf.tx0 - 1) >> 1;
    tf.ncol = (tf.tx1 >> 1) - tf.hx_lo + 1;
    tf.nrow = tf.ty1 - tf.ty0 + 2;
    return tf;
}

// Staging table: per colour and half-site, the sample angle (Sec. 2.1
// transform) at a sample site, NaN at a gap site, -1 at an absent site and at
// the padding half-site of an odd-width row.
__global__ void k_stage_table(Geom g, const uint8_t* __restrict__ mask,
                              const float* __restrict__ dang, float* __restrict__ stab) {
    const int64_t plane = (int64_t)g.H * g.Wh;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * plane;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / plane);
        const int64_t r = i - c * plane;
        const int y = (int)(r / g.Wh), h = (int)(r - (int64_t)y * g.Wh);
        const int x = 2 * h + ((c ^ y) & 1);
        float v = -1.0f;
        if (x < g.W) {
            const uint8_t m = mask[(int64_t)y * g.W + x];
            if (m == MASK_GAP) v = __int_as_float(0x7fc00000);
            else if (m != MASK_ABSENT) v = dang[i];
        }
        stab[i] = v;
    }
}

// Gap sites of each colour in every tile: one warp per tile.
__global__ void k_tile_count(Geom g, Tiles tl, const int32_t* __restrict__ of_block,
                             const uint8_t* __restrict__ mask, int32_t* __restrict__ cnt0,
                             int32_t* __restrict__ cnt1) {
    const int t = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= tl.n) return;
    const TileFrame tf = tile_frame(g, tl, of_block, t);
    const int tw = max(0, tf.tx1 - tf.tx0), n = max(0, tf.ty1 - tf.ty0) * tw;
    int n0 = 0, n1 = 0;
    for (int j = lane; j < n; j += 32) {
        const int y = tf.ty0 + j / tw, x = tf.tx0 + j % tw;
        if (mask[(int64_t)y * g.W + x] == MASK_GAP) {
            if (((x + y) & 1) == 0) ++n0; else ++n1;
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        n0 += __shfl_xor_sync(0xffffffffu, n0, d);
        n1 += __shfl_xor_sync(0xffffffffu, n1, d);
    }
    if (lane == 0) {
        cnt0[t] = n0;
        cnt1[t] = n1;
    }
}

// The tile-major lists: one warp per tile writes the tile's gap entries of
// both colours, ballot-compacted, block-edge entries first, then row-major.
__global__ void k_tile_lists(Geom g, Tiles tl, const int32_t* __restrict__ of_block,
                             const uint8_t* __restrict__ mask, const int32_t* __restrict__ start0,
                             const int32_t* __restrict__ start1, uint2* __restrict__ list0,
                             uint2* __restrict__ list1) {
    const int t = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= tl.n) return;
    const TileFrame tf = tile_frame(g, tl, of_block, t);
    const BlockFrame fr = block_frame(g, of_block, tf.b);
    const int tw = max(0, tf.tx1 - tf.tx0), n = max(0, tf.ty1 - tf.ty0) * tw;
    int o0 = start0[t], o1 = start1[t];
    for (int pass = 0; pass < 2; ++pass) {
        for (int j0 = 0; j0 < n; j0 += 32) {
            const int j = j0 + lane;
            bool take = false;
            int y = 0, x = 0, c = 0;
            if (j < n) {
                y = tf.ty0 + j / tw;
                x = tf.tx0 + j % tw;
                take = mask[(int64_t)y * g.W + x] == MASK_GAP && block_edge(fr, y, x) == (pass == 0);
                c = (x + y) & 1;
            }
            const unsigned m0 = __ballot_sync(0xffffffffu, take && c == 0);
            const unsigned m1 = __ballot_sync(0xffffffffu, take && c == 1);
            if (take) {
                const uint2 e = gap_entry(g, mask, fr, y, x);
                const unsigned below = (1u << lane) - 1u;
                if (c == 0) list0[o0 + __popc(m0 & below)] = e;
                else list1[o1 + __popc(m1 & below)] = e;
            }
            o0 += __popc(m0);
            o1 += __popc(m1);
        }
    }
}

// One half-step of colour a.colour over every (tile, lane group) item whose
// block still runs in that lane group; items are tile-major, lane group
// minor, so the CTAs working at one time share tiles' table and list reads.
template <typename S>
__global__ void __launch_bounds__(kTileThreads, 8) k_sweep_tile(SweepArgs a) {
    grid_dep_launch();
    __shared__ float4 stage[kStageSites * 4];       // [site][pair]: (c0, s0, c1, s1)
    __shared__ float red[kTileWarps][4][6];
    grid_dep_wait();
    constexpr int G = 8;
    const Geom& g = a.g;
    const Tiles& tl = a.tl;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t t = a.t_fixed > 0 ? (uint32_t)a.t_fixed : a.ctl->t;
    const uint32_t ctr1 = t | (a.ctl->tag << 16);
    const size_t plane = (size_t)g.H * g.Wh;
    const int c = a.colour, co = c ^ 1;
    const float* stab = tl.stab + (size_t)co * plane;
    const float q_m = a.m.q, J = a.m.J;
    const int n_items = tl.n * a.groups;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int tile = item / a.groups, grp = item - tile * a.groups;
        const int e0 = tl.start[tile], e1 = tl.start[tile + 1];
        if (e0 >= e1) continue;
        const int tpb = tl.tpx * tl.tpy;
        const int b = tile / tpb;
        // Running flags of the lane group's eight realizations in this block.
        unsigned long long rb;
        if (a.running) {
            rb = *reinterpret_cast<const unsigned long long*>(a.running + (size_t)b * a.Rp + grp * G);
        } else {
            rb = 0;
            for (int k = 0; k < G; ++k)
                if (grp * G + k < a.R) rb |= 0xffull << (8 * k);
        }
        if (rb == 0) continue;
        const TileFrame tf = tile_frame(g, tl, a.sl.of_block, tile);
        const S* oth = static_cast<const S*>(a.ang) + (size_t)(grp * 2 + co) * plane * G;
        S* own = static_cast<S*>(a.ang) + (size_t)(grp * 2 + c) * plane * G;

        // Stage: (cos, sin) of q phi_j for every realization of each running
        // pair, at every other-colour site of the tile and its halo.
        const int n_st = tf.nrow * tf.ncol;
        const float inv_ncol = 1.0f / (float)tf.ncol;
        for (int i = threadIdx.x; i < n_st * 4; i += kTileThreads) {
            const int q = i & 3, s = i >> 2;
            if (((rb >> (16 * q)) & 0xffffull) == 0) continue;
            // row = floor(s / ncol) through the reciprocal: s < 2^9 and ncol <= 18,
            // so (s + 1/2) / ncol stays at least 1/36 away from an integer.
            const int r = (int)(((float)s + 0.5f) * inv_ncol);
            const int k = s - r * tf.ncol;
            const int y = tf.ty0 - 1 + r, h = tf.hx_lo + k;
            const int x = 2 * h + ((co ^ y) & 1);
            const bool ok = (unsigned)y < (unsigned)g.H && (unsigned)x < (unsigned)g.W &&
                            (x >= tf.tx0 || tf.l_ok) && (x < tf.tx1 || tf.r_ok) &&
                            (y >= tf.ty0 || tf.u_ok) && (y < tf.ty1 || tf.d_ok);
            const size_t hs = (size_t)y * g.Wh + h;
            float v = -1.0f;
            if (ok) v = stab[hs];
            float2 ang = make_float2(v, v);
            if (v != v) ang = Store<S>::load2(oth + hs * G + 2 * q);
            float s0, c0, s1, c1;
            __sincosf(q_m * ang.x, &s0, &c0);
            __sincosf(q_m * ang.y, &s1, &c1);
            stage[i] = !(v < 0.0f) ? make_float4(c0, s0, c1, s1) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();

        // Update: one thread per (gap entry, realization pair).
        const float beta = a.beta[b];
        const int sl = slice_of(a.sl, b);
        const int4 rc = slice_rect(a.sl, sl);
        const uint32_t key1 = slice_key1(a.sl, sl);
        float ao0 = 0.f, ao1 = 0.f, al0 = 0.f, al1 = 0.f, au0 = 0.f, au1 = 0.f;
        const int ne = e1 - e0;
        const int ncol = tf.ncol;
        for (int i = threadIdx.x; i < ne * 4; i += kTileThreads) {
            const int q = i & 3;
            const bool run0 = ((rb >> (16 * q)) & 0xffull) != 0;
            const bool run1 = ((rb >> (16 * q + 8)) & 0xffull) != 0;
            if (!(run0 || run1)) continue;
            const uint2 en = tl.list[e0 + (i >> 2)];
            const int y = en.x >> 16, x = en.x & 0xffff;
            const uint32_t f = en.y;
            const int r = y - tf.ty0 + 1;
            const int hc = (x >> 1) - tf.hx_lo;
            const int kl = ((x - 1) >> 1) - tf.hx_lo, kr = ((x + 1) >> 1) - tf.hx_lo;
            const float4 L = stage[(r * ncol + kl) * 4 + q];
            const float4 R = stage[(r * ncol + kr) * 4 + q];
            const float4 U = stage[((r - 1) * ncol + hc) * 4 + q];
            const float4 D = stage[((r + 1) * ncol + hc) * 4 + q];
            const float C0 = (L.x + R.x) + (U.x + D.x);
            const float S0 = (L.y + R.y) + (U.y + D.y);
            const float C1 = (L.z + R.z) + (U.z + D.z);
            const float S1 = (L.w + R.w) + (U.w + D.w);
            const uint32_t hs = (uint32_t)y * (uint32_t)g.Wh + (uint32_t)(x >> 1);
            S* po = own + (size_t)hs * G + 2 * q;
            const float2 ph = Store<S>::load2(po);
            const int rl = grp * G + 2 * q;
            uint32_t w[4];
            philox4x32_10_rk(local_index(rc, y, x), ctr1, (a.r_base + (uint32_t)rl) >> 1, 0u,
                             a.rng.rk0, key1, w);
            const float bt = a.beta_site ? a.beta_site[(size_t)y * g.W + x] : beta;
            float2 out = ph;
            if (run0) {
                const SiteNew n = site_update<S>(ph.x, C0, S0, u01(w[0]), u01(w[1]), bt, a.m);
                out.x = n.phi;
                add_energy_lu(n, f, C0, S0, L.x, L.y, U.x, U.y, J, ao0, al0, au0);
            }
            if (run1) {
                const SiteNew n = site_update<S>(ph.y, C1, S1, u01(w[2]), u01(w[3]), bt, a.m);
                out.y = n.phi;
                add_energy_lu(n, f, C1, S1, L.z, L.w, U.z, U.w, J, ao1, al1, au1);
            }
            Store<S>::store2(po, out);
        }

        // The tile's energy changes: FP32 sums over the lanes of one pair
        // (lanes q, q + 4, ...) and over the warps, then one FP64 atomic per
        // (block, realization) for the own, left and upper blocks.
        if (a.energy) {
            float v[6] = {ao0, ao1, al0, al1, au0, au1};
#pragma unroll
            for (int d = 4; d < 32; d <<= 1)
#pragma unroll
                for (int k = 0; k < 6; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], d);
            if (lane < 4)
#pragma unroll
                for (int k = 0; k < 6; ++k) red[warp][lane][k] = v[k];
            __syncthreads();
            if (threadIdx.x < 4) {
                const int q = threadIdx.x;
                float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int w = 0; w < kTileWarps; ++w)
#pragma unroll
                    for (int k = 0; k < 6; ++k) s[k] += red[w][q][k];
                double* ea = a.eacc + (size_t)b * a.Rp + grp * G + 2 * q;
                const size_t up = (size_t)g.nbx * a.Rp;
                if (s[0] != 0.0f) atomicAdd(ea, (double)s[0]);
                if (s[1] != 0.0f) atomicAdd(ea + 1, (double)s[1]);
                if (s[2] != 0.0f) atomicAdd(ea - a.Rp, (double)s[2]);
                if (s[3] != 0.0f) atomicAdd(ea - a.Rp + 1, (double)s[3]);
                if (s[4] != 0.0f) atomicAdd(ea - up, (double)s[4]);
                if (s[5] != 0.0f) atomicAdd(ea - up + 1, (double)s[5]);
            }
        }
        __syncthreads();   // the next item restages
    }
}

template <typename S> struct TagT { using type = S; };
template <typename F> void with_storage_t(int storage, F&& f) {
    if (storage == 1) f(TagT<__nv_bfloat16>{});
    else if (storage == 2) f(TagT<__half>{});
    else f(TagT<float>{});
}

inline int grid_for_t(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

}  // namespace

Tiles tile_shape(const Geom& g) {
    Tiles t{};
    t.th = g.lb < kTileRows ? g.lb : kTileRows;
    t.tw = g.lb < kTileCols ? g.lb : kTileCols;
    t.tpy = (g.lb + t.th - 1) / t.th;
    t.tpx = (g.lb + t.tw - 1) / t.tw;
    t.n = g.nblk * t.tpx * t.tpy;
    return t;
}

void launch_stage_table(const Geom& g, const uint8_t* mask, const float* dang, float* stab,
                        cudaStream_t s) {
    k_stage_table<<<grid_for_t(2 * (int64_t)g.H * g.Wh, 256), 256, 0, s>>>(g, mask, dang, stab);
}

void launch_tile_count(const Geom& g, const Tiles& tl, const int32_t* of_block,
                       const uint8_t* mask, int32_t* cnt0, int32_t* cnt1, cudaStream_t s) {
    const int64_t threads = (int64_t)tl.n * 32;
    k_tile_count<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(g, tl, of_block, mask, cnt0,
                                                                   cnt1);
}

void launch_tile_lists(const Geom& g, const Tiles& tl, const int32_t* of_block,
                       const uint8_t* mask, const int32_t* start0, const int32_t* start1,
                       uint2* list0, uint2* list1, cudaStream_t s) {
    const int64_t threads = (int64_t)tl.n * 32;
    k_tile_lists<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(g, tl, of_block, mask, start0,
                                                                   start1, list0, list1);
}

int tile_blocks_per_sm(int storage) {
    int n = 1;
    with_storage_t(storage, [&](auto tag) {
        using S = typename decltype(tag)::type;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_tile<S>, kTileThreads, 0);
    });
    return n > 0 ? n : 1;
}

void launch_sweep_tile(const SweepArgs& a, int storage, int grid, cudaStream_t s) {
    with_storage_t(storage, [&](auto tag) {
        using S = typename decltype(tag)::type;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(kTileThreads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, k_sweep_tile<S>, a) != cudaSuccess) {
            cudaGetLastError();
            k_sweep_tile<S><<<grid, kTileThreads, 0, s>>>(a);
        }
    });
}

}  // namespace mpr
