// Device code of one checkerboard half-step (Sec. 2.2.2) and of the energy
// pass, shared by the per-launch kernels (mpr_kernels.cu) and the persistent
// calibration kernel (mpr_persist.cu).
//
// A (block, lane group) item is one block of the grid for the G realizations
// of one lane group. The state interleaves G realizations per site; each
// lane updates its site in both realizations of one realization pair, from
// one Philox block: words 0, 1 for the even realization, 2, 3 for the odd.
//
// Block energies are kept incrementally: a Metropolis move changes the energy
// of the site's four bonds by dE and the reflection conserves it, so a site
// whose bonds all belong to its own block adds dE there. A site on the left or
// top edge of its block splits the change bond by bond, because its left / up
// bond belongs to the neighbouring block (a bond is owned by the block of its
// left / upper site). Frozen sites never move, so stopped (block, realization)
// pairs cost nothing.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "mpr_device.cuh"
#include "mpr_internal.h"

namespace mpr {

__device__ __forceinline__ void add_energy(const SiteNew& n, uint32_t f, float C, float S,
                                           const float* nc, const float* ns, float J, float& ao,
                                           float& al, float& au) {
    if (!(f & (EDGE_L | EDGE_U))) {
        ao += n.dE;
        return;
    }
    float cn, sn;
    final_cs(n, C, S, cn, sn);
    const float dc = cn - n.co, ds = sn - n.so;
    const float dl = -J * (dc * nc[0] + ds * ns[0]);
    const float dr = -J * (dc * nc[1] + ds * ns[1]);
    const float du = -J * (dc * nc[2] + ds * ns[2]);
    const float dd = -J * (dc * nc[3] + ds * ns[3]);
    ao += dr + dd;
    if (f & EDGE_L) al += dl; else ao += dl;
    if (f & EDGE_U) au += du; else ao += du;
}

// Interior sites: warp sum of the block's own change, FP32 atomics into eacc
// (the stop test folds eacc into the FP64 block energy once per sweep).
__device__ __forceinline__ void flush_own(const SweepArgs& a, int b, int rl, float ao0, float ao1) {
    if (!__any_sync(0xffffffffu, ao0 != 0.0f || ao1 != 0.0f)) return;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        ao0 += __shfl_xor_sync(0xffffffffu, ao0, s);
        ao1 += __shfl_xor_sync(0xffffffffu, ao1, s);
    }
    if ((threadIdx.x & 31) != 0) return;
    float* ea = a.eacc + (size_t)b * a.Rp + rl;
    if (ao0 != 0.0f) atomicAdd(ea, ao0);
    if (ao1 != 0.0f) atomicAdd(ea + 1, ao1);
}

// From-scratch energies: FP64 warp sums added to the block energies.
__device__ __forceinline__ void flush_energy64(const SweepArgs& a, int b, int rl, double ao0,
                                               double ao1, double al0, double al1, double au0,
                                               double au1) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        ao0 += __shfl_xor_sync(0xffffffffu, ao0, s);
        ao1 += __shfl_xor_sync(0xffffffffu, ao1, s);
        al0 += __shfl_xor_sync(0xffffffffu, al0, s);
        al1 += __shfl_xor_sync(0xffffffffu, al1, s);
        au0 += __shfl_xor_sync(0xffffffffu, au0, s);
        au1 += __shfl_xor_sync(0xffffffffu, au1, s);
    }
    if ((threadIdx.x & 31) != 0) return;
    double* ea = a.ecur + (size_t)b * a.Rp + rl;
    if (ao0 != 0.0) atomicAdd(ea, ao0);
    if (ao1 != 0.0) atomicAdd(ea + 1, ao1);
    if (al0 != 0.0) atomicAdd(ea - a.Rp, al0);
    if (al1 != 0.0) atomicAdd(ea - a.Rp + 1, al1);
    const size_t up = (size_t)a.g.nbx * a.Rp;
    if (au0 != 0.0) atomicAdd(ea - up, au0);
    if (au1 != 0.0) atomicAdd(ea - up + 1, au1);
}

// (cos, sin) of q * phi_j of the four neighbours in both realizations. The
// state holds sample angles too, so every neighbour is one 8-byte load and a
// sin/cos pair per realization; a neighbour outside the grid is masked out.
__device__ __forceinline__ void neighbour_field(const SweepArgs& a, const float2* __restrict__ oth,
                                                int NP, uint32_t hs, int x, uint32_t f, float* nc0,
                                                float* ns0, float* nc1, float* ns1) {
    const uint32_t o = (uint32_t)(x & 1);
    const uint32_t hn[4] = {hs + o - 1u, hs + o, hs - (uint32_t)a.g.Wh, hs + (uint32_t)a.g.Wh};
    float2 v[4];
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const bool ex = (f & (NB_L << d)) != 0;
        v[d] = ex ? oth[(size_t)hn[d] * NP] : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const float m = (f & (NB_L << d)) ? 1.0f : 0.0f;
        float s0, c0, s1, c1;
        __sincosf(a.m.q * v[d].x, &s0, &c0);
        __sincosf(a.m.q * v[d].y, &s1, &c1);
        nc0[d] = m * c0;
        ns0[d] = m * s0;
        nc1[d] = m * c1;
        ns1[d] = m * s1;
    }
}

__device__ __forceinline__ void pair_running(const SweepArgs& a, int b, int rl, bool& run0,
                                             bool& run1) {
    if (a.running) {
        run0 = a.running[(size_t)b * a.Rp + rl] != 0;
        run1 = a.running[(size_t)b * a.Rp + rl + 1] != 0;
    } else {
        run0 = rl < a.R;
        run1 = rl + 1 < a.R;
    }
}

// Interior sites of one item (the segment after the block's edge entries):
// every bond of such a site belongs to the block, so the block's energy
// changes by the Metropolis dE. wpi warps share the item (wi = this warp's
// index among them): warp wi handles realization pair q = wi mod G/2, and
// warps of the same pair split the entries 32 at a time.
template <int G>
__device__ __forceinline__ void sweep_interior_item(const SweepArgs& a, int item, int wi, int wpi,
                                                    uint32_t ctr1) {
    constexpr int NP = G / 2;
    const int lane = threadIdx.x & 31;
    const int q = wi % NP, cw = wi / NP, CW = wpi / NP;
    const size_t plane = (size_t)a.g.H * a.g.Wh;
    const int c = a.colour, co = c ^ 1;
    const int b = item / a.groups, grp = item - b * a.groups;
    const int e0 = a.split[b], e1 = a.start[b + 1];
    if (e0 >= e1) return;
    const int rl = grp * G + 2 * q;
    bool run0, run1;
    pair_running(a, b, rl, run0, run1);
    if (!(run0 || run1)) return;
    float2* own = reinterpret_cast<float2*>(a.ang + (size_t)(grp * 2 + c) * plane * G) + q;
    const float2* oth =
        reinterpret_cast<const float2*>(a.ang + (size_t)(grp * 2 + co) * plane * G) + q;
    const float beta = a.beta[b];
    const uint32_t rpair = (a.r_base + (uint32_t)rl) >> 1;
    float ao0 = 0.f, ao1 = 0.f;
    for (int e = e0 + cw * 32 + lane; e < e1; e += CW * 32) {
        const uint2 en = a.list[e];
        const int y = en.x >> 16, x = en.x & 0xffff;
        const uint32_t f = en.y;
        const uint32_t hs = (uint32_t)y * (uint32_t)a.g.Wh + (uint32_t)(x >> 1);
        uint32_t w[4];
        philox4x32_10((uint32_t)y * (uint32_t)a.g.W + (uint32_t)x, ctr1, rpair, 0u, a.rng.key0,
                      a.rng.key1, w);
        const float2 ph = own[(size_t)hs * NP];
        float nc0[4], ns0[4], nc1[4], ns1[4];
        neighbour_field(a, oth, NP, hs, x, f, nc0, ns0, nc1, ns1);
        const float C0 = (nc0[0] + nc0[1]) + (nc0[2] + nc0[3]);
        const float S0 = (ns0[0] + ns0[1]) + (ns0[2] + ns0[3]);
        const float C1 = (nc1[0] + nc1[1]) + (nc1[2] + nc1[3]);
        const float S1 = (ns1[0] + ns1[1]) + (ns1[2] + ns1[3]);
        float2 out = ph;
        if (run0) {
            const SiteNew n = site_update(ph.x, C0, S0, u01(w[0]), u01(w[1]), beta, a.m);
            out.x = n.phi;
            ao0 += n.dE;
        }
        if (run1) {
            const SiteNew n = site_update(ph.y, C1, S1, u01(w[2]), u01(w[3]), beta, a.m);
            out.y = n.phi;
            ao1 += n.dE;
        }
        own[(size_t)hs * NP] = out;
    }
    if (a.energy) flush_own(a, b, rl, ao0, ao1);
}

// Interior sites of one item with two list entries per lane in flight: the
// two entries' loads and arithmetic are independent, and both realizations
// of the pair are computed without branches (a stopped one keeps its angle),
// so the compiler can overlap the two memory round trips.
template <int G>
__device__ __forceinline__ void sweep_interior_item2(const SweepArgs& a, int item, int wi, int wpi,
                                                     uint32_t ctr1) {
    constexpr int NP = G / 2;
    const int lane = threadIdx.x & 31;
    const int q = wi % NP, cw = wi / NP, CW = wpi / NP;
    const size_t plane = (size_t)a.g.H * a.g.Wh;
    const int c = a.colour, co = c ^ 1;
    const int b = item / a.groups, grp = item - b * a.groups;
    const int e0 = a.split[b], e1 = a.start[b + 1];
    if (e0 >= e1) return;
    const int rl = grp * G + 2 * q;
    bool run0, run1;
    pair_running(a, b, rl, run0, run1);
    if (!(run0 || run1)) return;
    float2* own = reinterpret_cast<float2*>(a.ang + (size_t)(grp * 2 + c) * plane * G) + q;
    const float2* oth =
        reinterpret_cast<const float2*>(a.ang + (size_t)(grp * 2 + co) * plane * G) + q;
    const float beta = a.beta[b];
    const uint32_t rpair = (a.r_base + (uint32_t)rl) >> 1;
    float ao0 = 0.f, ao1 = 0.f;
    for (int base = e0 + cw * 64 + lane; base < e1; base += CW * 64) {
        uint2 en[2];
        bool val[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int e = base + 32 * j;
            val[j] = e < e1;
            en[j] = val[j] ? a.list[e] : make_uint2(0u, 0u);
        }
        uint32_t hs[2], w[2][4];
        int xs[2];
        float2 ph[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int y = en[j].x >> 16;
            xs[j] = en[j].x & 0xffff;
            hs[j] = (uint32_t)y * (uint32_t)a.g.Wh + (uint32_t)(xs[j] >> 1);
            ph[j] = val[j] ? own[(size_t)hs[j] * NP] : make_float2(0.0f, 0.0f);
            philox4x32_10((uint32_t)y * (uint32_t)a.g.W + (uint32_t)xs[j], ctr1, rpair, 0u,
                          a.rng.key0, a.rng.key1, w[j]);
        }
        float nc0[2][4], ns0[2][4], nc1[2][4], ns1[2][4];
#pragma unroll
        for (int j = 0; j < 2; ++j)
            neighbour_field(a, oth, NP, hs[j], xs[j], val[j] ? en[j].y : 0u, nc0[j], ns0[j], nc1[j],
                            ns1[j]);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float C0 = (nc0[j][0] + nc0[j][1]) + (nc0[j][2] + nc0[j][3]);
            const float S0 = (ns0[j][0] + ns0[j][1]) + (ns0[j][2] + ns0[j][3]);
            const float C1 = (nc1[j][0] + nc1[j][1]) + (nc1[j][2] + nc1[j][3]);
            const float S1 = (ns1[j][0] + ns1[j][1]) + (ns1[j][2] + ns1[j][3]);
            const SiteNew n0 = site_update(ph[j].x, C0, S0, u01(w[j][0]), u01(w[j][1]), beta, a.m);
            const SiteNew n1 = site_update(ph[j].y, C1, S1, u01(w[j][2]), u01(w[j][3]), beta, a.m);
            const bool m0 = run0 && val[j], m1 = run1 && val[j];
            ao0 += m0 ? n0.dE : 0.0f;
            ao1 += m1 ? n1.dE : 0.0f;
            if (val[j])
                own[(size_t)hs[j] * NP] = make_float2(m0 ? n0.phi : ph[j].x, m1 ? n1.phi : ph[j].y);
        }
    }
    if (a.energy) flush_own(a, b, rl, ao0, ao1);
}

// Edge sites of one item (left / top edge of the block). A block has few of
// them, so one warp takes the whole item: lane = entry slot * (G/2) + pair,
// i.e. 32/(G/2) entries times all pairs per pass, and one site's G
// realizations are read as one contiguous chunk.
template <int G>
__device__ __forceinline__ void sweep_edge_item(const SweepArgs& a, int item, uint32_t ctr1) {
    constexpr int NP = G / 2;
    constexpr int EPI = 32 / NP;
    const int lane = threadIdx.x & 31;
    const int q = lane % NP, el = lane / NP;
    const size_t plane = (size_t)a.g.H * a.g.Wh;
    const int c = a.colour, co = c ^ 1;
    const int b = item / a.groups, grp = item - b * a.groups;
    const int e0 = a.start[b], e1 = a.split[b];
    if (e0 >= e1) return;
    const int rl = grp * G + 2 * q;
    bool run0, run1;
    pair_running(a, b, rl, run0, run1);
    if (!__any_sync(0xffffffffu, run0 || run1)) return;
    float2* own = reinterpret_cast<float2*>(a.ang + (size_t)(grp * 2 + c) * plane * G) + q;
    const float2* oth =
        reinterpret_cast<const float2*>(a.ang + (size_t)(grp * 2 + co) * plane * G) + q;
    const float beta = a.beta[b];
    const uint32_t rpair = (a.r_base + (uint32_t)rl) >> 1;
    float ao0 = 0.f, ao1 = 0.f, al0 = 0.f, al1 = 0.f, au0 = 0.f, au1 = 0.f;
    for (int base = e0; base < e1; base += EPI) {
        const int e = base + el;
        if (e >= e1 || !(run0 || run1)) continue;
        const uint2 en = a.list[e];
        const int y = en.x >> 16, x = en.x & 0xffff;
        const uint32_t f = en.y;
        const uint32_t hs = (uint32_t)y * (uint32_t)a.g.Wh + (uint32_t)(x >> 1);
        uint32_t w[4];
        philox4x32_10((uint32_t)y * (uint32_t)a.g.W + (uint32_t)x, ctr1, rpair, 0u, a.rng.key0,
                      a.rng.key1, w);
        const float2 ph = own[(size_t)hs * NP];
        float nc0[4], ns0[4], nc1[4], ns1[4];
        neighbour_field(a, oth, NP, hs, x, f, nc0, ns0, nc1, ns1);
        const float C0 = (nc0[0] + nc0[1]) + (nc0[2] + nc0[3]);
        const float S0 = (ns0[0] + ns0[1]) + (ns0[2] + ns0[3]);
        const float C1 = (nc1[0] + nc1[1]) + (nc1[2] + nc1[3]);
        const float S1 = (ns1[0] + ns1[1]) + (ns1[2] + ns1[3]);
        float2 out = ph;
        if (run0) {
            const SiteNew n = site_update(ph.x, C0, S0, u01(w[0]), u01(w[1]), beta, a.m);
            out.x = n.phi;
            add_energy(n, f, C0, S0, nc0, ns0, a.m.J, ao0, al0, au0);
        }
        if (run1) {
            const SiteNew n = site_update(ph.y, C1, S1, u01(w[2]), u01(w[3]), beta, a.m);
            out.y = n.phi;
            add_energy(n, f, C1, S1, nc1, ns1, a.m.J, ao1, al1, au1);
        }
        own[(size_t)hs * NP] = out;
    }
    if (!a.energy) return;
    // Sum over the entry slots of each pair; the slot-0 lane of each pair adds
    // to the blocks.
#pragma unroll
    for (int s = NP; s < 32; s <<= 1) {
        ao0 += __shfl_xor_sync(0xffffffffu, ao0, s);
        ao1 += __shfl_xor_sync(0xffffffffu, ao1, s);
        al0 += __shfl_xor_sync(0xffffffffu, al0, s);
        al1 += __shfl_xor_sync(0xffffffffu, al1, s);
        au0 += __shfl_xor_sync(0xffffffffu, au0, s);
        au1 += __shfl_xor_sync(0xffffffffu, au1, s);
    }
    if (el != 0) return;
    float* ea = a.eacc + (size_t)b * a.Rp + rl;
    if (ao0 != 0.0f) atomicAdd(ea, ao0);
    if (ao1 != 0.0f) atomicAdd(ea + 1, ao1);
    if (al0 != 0.0f) atomicAdd(ea - a.Rp, al0);
    if (al1 != 0.0f) atomicAdd(ea - a.Rp + 1, al1);
    const size_t up = (size_t)a.g.nbx * a.Rp;
    if (au0 != 0.0f) atomicAdd(ea - up, au0);
    if (au1 != 0.0f) atomicAdd(ea - up + 1, au1);
}

// One half-step over the whole list of one colour, flat: one thread per
// (gap entry, realization pair), 32 / (G/2) entries per warp, one lane group
// per blockIdx.y (a CTA never mixes lane groups). For calibration, where every
// block runs and only one or a few chains exist, this puts every site's
// latency chain into one wave. The block-energy change is summed per CTA in
// shared memory (the list is block-major, so a CTA spans few blocks) and
// flushed with one atomic per (block, realization); changes that belong to
// another block (left / up bonds of edge sites) go straight to global memory.
constexpr int kFlatThreads = 256;
constexpr int kFlatBlocks = 64;     // local blocks summed in shared memory per CTA

template <int G>
__device__ __forceinline__ void sweep_flat(const SweepArgs& a, int64_t n_list, uint32_t ctr1) {
    constexpr int NP = G / 2;
    __shared__ float acc[kFlatBlocks * G];
    const int grp = blockIdx.y;
    const int64_t t0 = (int64_t)blockIdx.x * kFlatThreads;
    const int64_t t = t0 + threadIdx.x;
    const int64_t e = t / NP;
    const int q = (int)(t % NP);
    for (int i = threadIdx.x; i < kFlatBlocks * G; i += kFlatThreads) acc[i] = 0.0f;
    const int b0 = (int)(a.list[t0 / NP].y >> META_SHIFT);
    __syncthreads();
    if (e < n_list) {
        const size_t plane = (size_t)a.g.H * a.g.Wh;
        const int c = a.colour, co = c ^ 1;
        const uint2 en = a.list[e];
        const int b = (int)(en.y >> META_SHIFT);
        const int rl = grp * G + 2 * q;
        bool run0, run1;
        pair_running(a, b, rl, run0, run1);
        if (run0 || run1) {
            float2* own = reinterpret_cast<float2*>(a.ang + (size_t)(grp * 2 + c) * plane * G) + q;
            const float2* oth =
                reinterpret_cast<const float2*>(a.ang + (size_t)(grp * 2 + co) * plane * G) + q;
            const int y = en.x >> 16, x = en.x & 0xffff;
            const uint32_t f = en.y;
            const uint32_t hs = (uint32_t)y * (uint32_t)a.g.Wh + (uint32_t)(x >> 1);
            uint32_t w[4];
            philox4x32_10((uint32_t)y * (uint32_t)a.g.W + (uint32_t)x, ctr1,
                          (a.r_base + (uint32_t)rl) >> 1, 0u, a.rng.key0, a.rng.key1, w);
            const float2 ph = own[(size_t)hs * NP];
            float nc0[4], ns0[4], nc1[4], ns1[4];
            neighbour_field(a, oth, NP, hs, x, f, nc0, ns0, nc1, ns1);
            const float C0 = (nc0[0] + nc0[1]) + (nc0[2] + nc0[3]);
            const float S0 = (ns0[0] + ns0[1]) + (ns0[2] + ns0[3]);
            const float C1 = (nc1[0] + nc1[1]) + (nc1[2] + nc1[3]);
            const float S1 = (ns1[0] + ns1[1]) + (ns1[2] + ns1[3]);
            const float beta = a.beta[b];
            float2 out = ph;
            float ao0 = 0.f, ao1 = 0.f, al0 = 0.f, al1 = 0.f, au0 = 0.f, au1 = 0.f;
            if (run0) {
                const SiteNew n = site_update(ph.x, C0, S0, u01(w[0]), u01(w[1]), beta, a.m);
                out.x = n.phi;
                add_energy(n, f, C0, S0, nc0, ns0, a.m.J, ao0, al0, au0);
            }
            if (run1) {
                const SiteNew n = site_update(ph.y, C1, S1, u01(w[2]), u01(w[3]), beta, a.m);
                out.y = n.phi;
                add_energy(n, f, C1, S1, nc1, ns1, a.m.J, ao1, al1, au1);
            }
            own[(size_t)hs * NP] = out;
            if (a.energy) {
                const int loc = b - b0;
                if (loc < kFlatBlocks) {
                    if (ao0 != 0.0f) atomicAdd(&acc[loc * G + 2 * q], ao0);
                    if (ao1 != 0.0f) atomicAdd(&acc[loc * G + 2 * q + 1], ao1);
                } else {
                    float* ea = a.eacc + (size_t)b * a.Rp + rl;
                    if (ao0 != 0.0f) atomicAdd(ea, ao0);
                    if (ao1 != 0.0f) atomicAdd(ea + 1, ao1);
                }
                if (f & (EDGE_L | EDGE_U)) {
                    float* ea = a.eacc + (size_t)b * a.Rp + rl;
                    if (al0 != 0.0f) atomicAdd(ea - a.Rp, al0);
                    if (al1 != 0.0f) atomicAdd(ea - a.Rp + 1, al1);
                    const size_t up = (size_t)a.g.nbx * a.Rp;
                    if (au0 != 0.0f) atomicAdd(ea - up, au0);
                    if (au1 != 0.0f) atomicAdd(ea - up + 1, au1);
                }
            }
        }
    }
    if (!a.energy) return;
    __syncthreads();
    for (int i = threadIdx.x; i < kFlatBlocks * G; i += kFlatThreads) {
        const float v = acc[i];
        if (v != 0.0f) atomicAdd(&a.eacc[(size_t)(b0 + i / G) * a.Rp + grp * G + (i % G)], v);
    }
}

// Energies from scratch (no move) of one item: every bond that touches a gap
// site, once. A bond always joins a colour-0 and a colour-1 site; colour 1
// adds every bond of its gap sites, colour 0 the bonds of its gap sites to
// samples. Bonds between two samples are the constant E_s,b. Every lane of
// the item is counted (the pass ignores the running flags).
template <int G>
__device__ __forceinline__ void energy_item(const SweepArgs& a, int item, int wi, int wpi) {
    constexpr int NP = G / 2;
    const int lane = threadIdx.x & 31;
    const int q = wi % NP, cw = wi / NP, CW = wpi / NP;
    const size_t plane = (size_t)a.g.H * a.g.Wh;
    const int c = a.colour, co = c ^ 1;
    const int b = item / a.groups, grp = item - b * a.groups;
    const int rl = grp * G + 2 * q;
    const int e0 = a.start[b], e1 = a.start[b + 1];
    const float2* own =
        reinterpret_cast<const float2*>(a.ang + (size_t)(grp * 2 + c) * plane * G) + q;
    const float2* oth =
        reinterpret_cast<const float2*>(a.ang + (size_t)(grp * 2 + co) * plane * G) + q;
    double ao0 = 0.0, ao1 = 0.0, al0 = 0.0, al1 = 0.0, au0 = 0.0, au1 = 0.0;
    for (int e = e0 + cw * 32 + lane; e < e1; e += CW * 32) {
        const uint2 en = a.list[e];
        const int y = en.x >> 16, x = en.x & 0xffff;
        const uint32_t f = en.y;
        const uint32_t hs = (uint32_t)y * (uint32_t)a.g.Wh + (uint32_t)(x >> 1);
        const float2 ph = own[(size_t)hs * NP];
        float nc0[4], ns0[4], nc1[4], ns1[4];
        neighbour_field(a, oth, NP, hs, x, f, nc0, ns0, nc1, ns1);
        float s0, c0, s1, c1;
        __sincosf(a.m.q * ph.x, &s0, &c0);
        __sincosf(a.m.q * ph.y, &s1, &c1);
        const uint32_t take = (c == 1) ? 0xFu : (~(f >> 4) & 0xFu);
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            if (!((f & (NB_L << d)) && (take & (1u << d)))) continue;
            const float b0 = -a.m.J * (c0 * nc0[d] + s0 * ns0[d]);
            const float b1 = -a.m.J * (c1 * nc1[d] + s1 * ns1[d]);
            if (d == 0 && (f & EDGE_L)) { al0 += b0; al1 += b1; }
            else if (d == 2 && (f & EDGE_U)) { au0 += b0; au1 += b1; }
            else { ao0 += b0; ao1 += b1; }
        }
    }
    flush_energy64(a, b, rl, ao0, ao1, al0, al1, au0, au1);
}

// Median of the targeted blocks' T by a radix select over the (positive)
// float bit patterns, run by one CTA; k is the 0-based rank.
__device__ inline uint32_t select_kth(const float* __restrict__ T, const int32_t* __restrict__ Nsp,
                                      int nblk, uint32_t k, uint32_t* hist, uint32_t* s_digit,
                                      uint32_t* s_k) {
    uint32_t prefix = 0, pmask = 0;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
            if (Nsp[b] <= 0) continue;
            const uint32_t v = __float_as_uint(T[b]);
            if ((v & pmask) == prefix) atomicAdd(&hist[(v >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t kk = k, d = 0;
            while (d < 255 && kk >= hist[d]) { kk -= hist[d]; ++d; }
            *s_digit = d;
            *s_k = kk;
        }
        __syncthreads();
        prefix |= (*s_digit) << shift;
        pmask |= 255u << shift;
        k = *s_k;
        __syncthreads();
    }
    return prefix;
}

// Median (mean of the two middle values for an even count) of the targeted
// blocks' T, by one CTA; 0 when no block is targeted.
__device__ inline float median_targeted(const float* __restrict__ T, const int32_t* __restrict__ Nsp,
                                        int nblk) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t s_digit, s_k, s_n;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    uint32_t cnt = 0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) cnt += Nsp[b] > 0;
    atomicAdd(&s_n, cnt);
    __syncthreads();
    const uint32_t n = s_n;
    float med = 0.0f;
    if (n > 0) {
        const float lo = __uint_as_float(select_kth(T, Nsp, nblk, (n - 1) / 2, hist, &s_digit, &s_k));
        const float hi =
            (n & 1) ? lo : __uint_as_float(select_kth(T, Nsp, nblk, n / 2, hist, &s_digit, &s_k));
        med = 0.5f * (lo + hi);
    }
    return med;
}

}  // namespace mpr
