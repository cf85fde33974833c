// Device code of one checkerboard half-step (Sec. 2.2.2) and of the energy
// pass, shared by the per-launch kernels (mpr_kernels.cu) and the persistent
// calibration kernel (mpr_persist.cu).
//
// A (block, lane group) item is one block of the grid for the G realizations
// of one lane group; the realizations' worklist hands out its realization
// pairs one by one (units), the calibration's flat kernel every entry. The state interleaves G realizations per site; each
// lane updates its site in both realizations of one realization pair, from
// one Philox block: words 0, 1 for the even realization, 2, 3 for the odd.
//
// Block energies are kept incrementally. A move changes the energy of the
// site's four bonds by dE, and the reflection conserves it (up to the
// rounding of the stored angle, which the 16-bit forms account for), so the
// site's block gains dE. A site on the left or top edge of its block hands
// the change of its left / up bond to the neighbouring block that owns it (a
// bond is owned by the block of its left / upper site). Frozen sites never
// move, so stopped (block, realization) pairs cost nothing.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mpr_device.cuh"
#include "mpr_internal.h"

namespace mpr {

// Element type of the batch state: a realization pair is two adjacent
// elements, loaded and stored as one 8-byte (FP32) or 4-byte (FP16 / BF16)
// access; arithmetic is FP32 throughout. The sample angles the method
// conditions on are never rounded: the 16-bit forms read them from the FP32
// per-field table instead of the state.
template <typename S> struct Store;

template <> struct Store<float> {
    static constexpr bool kExact = true;
    __device__ static float2 load2(const float* p) { return *reinterpret_cast<const float2*>(p); }
    __device__ static void store2(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
    __device__ static float load1(const float* p) { return *p; }
    __device__ static void store1(float* p, float v) { *p = v; }
    __device__ static float round(float v) { return v; }
};

template <> struct Store<__half> {
    static constexpr bool kExact = false;
    __device__ static float2 load2(const __half* p) {
        return __half22float2(*reinterpret_cast<const __half2*>(p));
    }
    __device__ static void store2(__half* p, float2 v) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(v.x, v.y);
    }
    __device__ static float load1(const __half* p) { return __half2float(*p); }
    __device__ static void store1(__half* p, float v) { *p = __float2half_rn(v); }
    __device__ static float round(float v) { return __half2float(__float2half_rn(v)); }
};

template <> struct Store<__nv_bfloat16> {
    static constexpr bool kExact = false;
    __device__ static float2 load2(const __nv_bfloat16* p) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
    }
    __device__ static void store2(__nv_bfloat16* p, float2 v) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(v.x, v.y);
    }
    __device__ static float load1(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    __device__ static void store1(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
    __device__ static float round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
};

// Site update with the state's rounding applied: the proposal is rounded
// before its energy is taken, so the Metropolis test judges the angle that
// is stored; the reflected angle is rounded too, and for the 16-bit forms
// dE becomes the exact change from the old to the stored final angle, with
// (ca, sa) the final angle's cos / sin and refl cleared.
template <typename S>
__device__ __forceinline__ SiteNew site_update(float phi, float C, float Sn, float u0, float u1,
                                               float beta, const Model& m) {
    SiteNew n;
    __sincosf(m.q * phi, &n.so, &n.co);
    const float php = Store<S>::round(kTwoPi * u0);
    float sp, cp;
    __sincosf(m.q * php, &sp, &cp);
    const float dE = m.J * ((C * n.co + Sn * n.so) - (C * cp + Sn * sp));
    const bool acc = (dE <= 0.0f) || (u1 < __expf(-dE * beta));
    n.phi = acc ? php : phi;
    n.dE = acc ? dE : 0.0f;
    n.ca = acc ? cp : n.co;
    n.sa = acc ? sp : n.so;
    // Over-relaxation, without branches. The reflected angle (2 psi - q phi)/q
    // is >= 0 only if psi >= 0, i.e. S >= 0, so psi is taken from (|S|, C) and
    // the move is kept only when S >= 0 and the angle lies in [0, 2pi]
    // (C = S = 0 gives NaN and fails the test).
    const float psi = atan2_upper(fabsf(Sn), C);
    const float por = (2.0f * psi - m.q * n.phi) * m.inv_q;
    n.refl = m.overrelax && Sn >= 0.0f && por >= 0.0f && por <= kTwoPi;
    n.phi = n.refl ? Store<S>::round(por) : n.phi;
    if constexpr (!Store<S>::kExact) {
        float sf, cf;
        __sincosf(m.q * n.phi, &sf, &cf);
        n.ca = cf;
        n.sa = sf;
        n.refl = false;
        n.dE = m.J * ((C * n.co + Sn * n.so) - (C * cf + Sn * sf));
    }
    return n;
}

// A block's change in one half-step: the FP32 warp sum of the unit's moves
// is added to eacc with an FP64 atomic, so every sum across units, half-steps
// and (in the stop test and the calibration fold) sweeps is FP64. (The warp
// sum stays FP32: GB300's FP64 pipe is narrow, and FP64 shuffle sums per unit
// doubled the half-step's time.)
__device__ __forceinline__ void flush_pair(double* ea, float v0, float v1) {
    if (!__any_sync(0xffffffffu, v0 != 0.0f || v1 != 0.0f)) return;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, s);
        v1 += __shfl_xor_sync(0xffffffffu, v1, s);
    }
    if ((threadIdx.x & 31) != 0) return;
    if (v0 != 0.0f) atomicAdd(ea, (double)v0);
    if (v1 != 0.0f) atomicAdd(ea + 1, (double)v1);
}

// Bond-by-bond split of a move at a block edge: (lc, ls) and (uc, us) are the
// left and upper neighbours' (cos, sin) of q phi_j.
__device__ __forceinline__ void add_energy_lu(const SiteNew& n, uint32_t f, float C, float S,
                                              float lc, float ls, float uc, float us, float J,
                                              float& ao, float& al, float& au) {
    if (!(f & (EDGE_L | EDGE_U))) {
        ao += n.dE;
        return;
    }
    float cn, sn;
    final_cs(n, C, S, cn, sn);
    const float dc = cn - n.co, ds = sn - n.so;
    const float dl = -J * (dc * lc + ds * ls);
    const float du = -J * (dc * uc + ds * us);
    ao += n.dE;
    if (f & EDGE_L) { ao -= dl; al += dl; }
    if (f & EDGE_U) { ao -= du; au += du; }
}

// The same with the four neighbours' (cos, sin) in arrays (left, right, up,
// down), as the kernels that keep all four use it.
__device__ __forceinline__ void add_energy(const SiteNew& n, uint32_t f, float C, float S,
                                           const float* nc, const float* ns, float J, float& ao,
                                           float& al, float& au) {
    add_energy_lu(n, f, C, S, nc[0], ns[0], nc[2], ns[2], J, ao, al, au);
}

// Angles of the four neighbours of a site in both realizations of the pair.
// FP32 state: every neighbour is one 8-byte state load (the state holds the
// sample angles too). 16-bit state: a gap neighbour is read from the state,
// a sample neighbour from the FP32 per-field table `dang`, both loads
// predicated on the flags. A neighbour outside the grid reads as 0 and is
// masked out by the caller.
template <typename S>
__device__ __forceinline__ void neighbour_angles(const SweepArgs& a, const S* __restrict__ oth,
                                                 int G, uint32_t hs, int x, uint32_t f,
                                                 float2 v[4]) {
    const uint32_t o = (uint32_t)(x & 1);
    const uint32_t hn[4] = {hs + o - 1u, hs + o, hs - (uint32_t)a.g.Wh, hs + (uint32_t)a.g.Wh};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const bool ex = (f & (NB_L << d)) != 0;
        if constexpr (Store<S>::kExact) {
            v[d] = ex ? Store<S>::load2(oth + (size_t)hn[d] * G) : make_float2(0.0f, 0.0f);
        } else {
            const bool gap = (f & (GAP_L << d)) != 0;
            const float* dn = a.dang + (size_t)(a.colour ^ 1) * a.g.H * a.g.Wh;
            const float sv = (ex && !gap) ? dn[hn[d]] : 0.0f;
            v[d] = (ex && gap) ? Store<S>::load2(oth + (size_t)hn[d] * G) : make_float2(sv, sv);
        }
    }
}

// (cos, sin) of q * phi_j of the four neighbours, masked by existence.
template <typename S>
__device__ __forceinline__ void neighbour_field(const SweepArgs& a, const S* __restrict__ oth,
                                                int G, uint32_t hs, int x, uint32_t f, float* nc0,
                                                float* ns0, float* nc1, float* ns1) {
    float2 v[4];
    neighbour_angles<S>(a, oth, G, hs, x, f, v);
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
        const uchar2 r2 = *reinterpret_cast<const uchar2*>(a.running + (size_t)b * a.Rp + rl);
        run0 = r2.x != 0;
        run1 = r2.y != 0;
    } else {
        run0 = rl < a.R;
        run1 = rl + 1 < a.R;
    }
}

// All gap sites of colour c in one item. wpi warps share the item (wi = this
// warp's index among them): warp wi handles realization pair q = wi mod G/2,
// and the wpi / (G/2) warps of a pair split the entries 32 at a time. The
// next entry of a lane is loaded while the current one is updated. The
// block's list puts its edge entries first, so the branch that splits an
// edge move bond by bond diverges in the first 32 entries only. kCal: the
// calibration's chains, whose two lanes of a pair may sit at different
// temperatures (the trisection's two points, or the k-point section's lane r
// at point r mod n_pts), as in sweep_flat.
template <int G, typename S, bool kCal = false>
__device__ __forceinline__ void sweep_item(const SweepArgs& a, int item, int wi, int wpi,
                                           uint32_t ctr1) {
    constexpr int NP = G / 2;
    const int lane = threadIdx.x & 31;
    const int q = wi % NP, cw = wi / NP, CW = wpi / NP;
    const size_t plane = (size_t)a.g.H * a.g.Wh;
    const int c = a.colour, co = c ^ 1;
    const int b = item / a.groups, grp = item - b * a.groups;
    const int e0 = a.start[b], e1 = a.start[b + 1];
    if (e0 >= e1) return;
    const int rl = grp * G + 2 * q;
    bool run0, run1;
    pair_running(a, b, rl, run0, run1);
    if (!(run0 || run1)) return;
    S* own = static_cast<S*>(a.ang) + (size_t)(grp * 2 + c) * plane * G + 2 * q;
    const S* oth = static_cast<const S*>(a.ang) + (size_t)(grp * 2 + co) * plane * G + 2 * q;
    float beta = a.beta[b], beta_odd = beta;
    if constexpr (kCal) {
        if (a.beta_pts) {
            beta = a.beta_pts[(size_t)(rl % a.n_pts) * a.g.nblk + b];
            beta_odd = a.beta_pts[(size_t)((rl + 1) % a.n_pts) * a.g.nblk + b];
        } else if (a.beta_odd) {
            beta_odd = a.beta_odd[b];
        }
    }
    const float J = a.m.J;
    const uint32_t rpair = (a.r_base + (uint32_t)rl) >> 1;
    const int sl = slice_of(a.sl, b);
    const int4 rc = slice_rect(a.sl, sl);
    const uint32_t key1 = slice_key1(a.sl, sl);
    float ao0 = 0.f, ao1 = 0.f, al0 = 0.f, al1 = 0.f, au0 = 0.f, au1 = 0.f;
    const int step = CW * 32;
    int e = e0 + cw * 32 + lane;
    uint2 nx = e < e1 ? a.list[e] : make_uint2(0u, 0u);
    for (; e < e1; e += step) {
        const uint2 en = nx;
        if (e + step < e1) nx = a.list[e + step];
        const int y = en.x >> 16, x = en.x & 0xffff;
        const uint32_t f = en.y;
        const uint32_t hs = (uint32_t)y * (uint32_t)a.g.Wh + (uint32_t)(x >> 1);
        uint32_t w[4];
        philox4x32_10_rk(local_index(rc, y, x), ctr1, rpair, 0u, a.rng.rk0, key1, w);
        const float2 ph = Store<S>::load2(own + (size_t)hs * G);
        float nc0[4], ns0[4], nc1[4], ns1[4];
        neighbour_field<S>(a, oth, G, hs, x, f, nc0, ns0, nc1, ns1);
        const float C0 = (nc0[0] + nc0[1]) + (nc0[2] + nc0[3]);
        const float S0 = (ns0[0] + ns0[1]) + (ns0[2] + ns0[3]);
        const float C1 = (nc1[0] + nc1[1]) + (nc1[2] + nc1[3]);
        const float S1 = (ns1[0] + ns1[1]) + (ns1[2] + ns1[3]);
        const float bt = a.beta_site ? a.beta_site[(size_t)y * a.g.W + x] : beta;
        float2 out = ph;
        if (run0) {
            const SiteNew n = site_update<S>(ph.x, C0, S0, u01(w[0]), u01(w[1]), bt, a.m);
            out.x = n.phi;
            add_energy(n, f, C0, S0, nc0, ns0, J, ao0, al0, au0);
        }
        if (run1) {
            const SiteNew n = site_update<S>(ph.y, C1, S1, u01(w[2]), u01(w[3]),
                                             kCal ? beta_odd : bt, a.m);
            out.y = n.phi;
            add_energy(n, f, C1, S1, nc1, ns1, J, ao1, al1, au1);
        }
        Store<S>::store2(own + (size_t)hs * G, out);
    }
    if (!a.energy) return;
    double* ea = a.eacc + (size_t)b * a.Rp + rl;
    flush_pair(ea, ao0, ao1);
    flush_pair(ea - a.Rp, al0, al1);
    flush_pair(ea - (size_t)a.g.nbx * a.Rp, au0, au1);
}

// Energy flush of one half-warp's unit: the FP32 sum over its 16 lanes, added
// by its lane 0 with an FP64 atomic (act: the half has a running unit).
// Every lane of the warp calls it.
__device__ __forceinline__ void flush_pair_half(double* ea, float v0, float v1, bool act) {
    if (!__any_sync(0xffffffffu, v0 != 0.0f || v1 != 0.0f)) return;
#pragma unroll
    for (int s = 8; s > 0; s >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, s);
        v1 += __shfl_xor_sync(0xffffffffu, v1, s);
    }
    if ((threadIdx.x & 15) != 0 || !act) return;
    if (v0 != 0.0f) atomicAdd(ea, (double)v0);
    if (v1 != 0.0f) atomicAdd(ea + 1, (double)v1);
}

// Two units per warp: lanes 0-15 take one (block, realization pair) unit,
// lanes 16-31 another, each half 16 gap entries at a time. For blocks whose
// colour holds few entries (about 64 at l_b = 16 and half the sites missing)
// the last, partial pass wastes fewer lanes, and the warp's per-unit work
// (bounds, flags, energy sums) serves two units. have: this half has a unit
// (item, pair q within its lane group); every lane of the warp calls this.
template <int G, typename S>
__device__ __forceinline__ void sweep_item_half(const SweepArgs& a, int item, int q, bool have,
                                                uint32_t ctr1) {
    const int hl = threadIdx.x & 15;
    const size_t plane = (size_t)a.g.H * a.g.Wh;
    const int c = a.colour, co = c ^ 1;
    const int b = have ? item / a.groups : 0, grp = have ? item - b * a.groups : 0;
    int e0 = 0, e1 = 0;
    bool run0 = false, run1 = false;
    const int rl = grp * G + 2 * q;
    if (have) {
        e0 = a.start[b];
        e1 = a.start[b + 1];
        pair_running(a, b, rl, run0, run1);
    }
    const bool act = have && e0 < e1 && (run0 || run1);
    float ao0 = 0.f, ao1 = 0.f, al0 = 0.f, al1 = 0.f, au0 = 0.f, au1 = 0.f;
    if (act) {
        S* own = static_cast<S*>(a.ang) + (size_t)(grp * 2 + c) * plane * G + 2 * q;
        const S* oth = static_cast<const S*>(a.ang) + (size_t)(grp * 2 + co) * plane * G + 2 * q;
        const float beta = a.beta[b];
        const float J = a.m.J;
        const uint32_t rpair = (a.r_base + (uint32_t)rl) >> 1;
        const int sl = slice_of(a.sl, b);
        const int4 rc = slice_rect(a.sl, sl);
        const uint32_t key1 = slice_key1(a.sl, sl);
        int e = e0 + hl;
        uint2 nx = e < e1 ? a.list[e] : make_uint2(0u, 0u);
        for (; e < e1; e += 16) {
            const uint2 en = nx;
            if (e + 16 < e1) nx = a.list[e + 16];
            const int y = en.x >> 16, x = en.x & 0xffff;
            const uint32_t f = en.y;
            const uint32_t hs = (uint32_t)y * (uint32_t)a.g.Wh + (uint32_t)(x >> 1);
            uint32_t w[4];
            philox4x32_10_rk(local_index(rc, y, x), ctr1, rpair, 0u, a.rng.rk0, key1, w);
            const float2 ph = Store<S>::load2(own + (size_t)hs * G);
            float nc0[4], ns0[4], nc1[4], ns1[4];
            neighbour_field<S>(a, oth, G, hs, x, f, nc0, ns0, nc1, ns1);
            const float C0 = (nc0[0] + nc0[1]) + (nc0[2] + nc0[3]);
            const float S0 = (ns0[0] + ns0[1]) + (ns0[2] + ns0[3]);
            const float C1 = (nc1[0] + nc1[1]) + (nc1[2] + nc1[3]);
            const float S1 = (ns1[0] + ns1[1]) + (ns1[2] + ns1[3]);
            const float bt = a.beta_site ? a.beta_site[(size_t)y * a.g.W + x] : beta;
            float2 out = ph;
            if (run0) {
                const SiteNew n = site_update<S>(ph.x, C0, S0, u01(w[0]), u01(w[1]), bt, a.m);
                out.x = n.phi;
                add_energy(n, f, C0, S0, nc0, ns0, J, ao0, al0, au0);
            }
            if (run1) {
                const SiteNew n = site_update<S>(ph.y, C1, S1, u01(w[2]), u01(w[3]), bt, a.m);
                out.y = n.phi;
                add_energy(n, f, C1, S1, nc1, ns1, J, ao1, al1, au1);
            }
            Store<S>::store2(own + (size_t)hs * G, out);
        }
    }
    if (!a.energy) return;
    double* ea = a.eacc + (size_t)b * a.Rp + rl;
    flush_pair_half(ea, ao0, ao1, act);
    flush_pair_half(ea - a.Rp, al0, al1, act);
    flush_pair_half(ea - (size_t)a.g.nbx * a.Rp, au0, au1, act);
}

// One half-step over the whole list of one colour, flat: one thread per
// (gap entry, realization pair), 32 / (G/2) entries per warp, one lane group
// per blockIdx.y (a CTA never mixes lane groups). For calibration, where every
// block runs and only one or a few chains exist, this puts every site's
// latency chain into one wave. The block-energy change is summed per CTA in
// shared memory (the list is block-major, so a CTA spans few blocks) and
// flushed with one atomic per (block, realization); changes that belong to
// another block (left / up bonds of edge sites) go straight to global memory.
// The per-CTA sums are FP32; the global accumulation is FP64.
constexpr int kFlatThreads = 256;
constexpr int kFlatBlocks = 64;     // local blocks summed in shared memory per CTA

// Programmatic dependent launch: a launch may start while the previous
// kernel on the stream finishes. griddepcontrol.wait blocks until every
// prerequisite grid has completed and its writes are visible; every thread of
// such a kernel executes it (so its completion implies its predecessors').
// launch_dependents lets the next launch begin once every CTA of this one
// has issued it or exited.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The list entry, its Philox block and the temperatures do not depend on the
// previous half-step, so they are taken before the dependency wait and
// overlap the previous launch's tail.
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
    const bool live = e < n_list;
    const int rl = grp * G + 2 * q;
    uint2 en = make_uint2(0u, 0u);
    int b = b0;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    float beta = 0.0f, beta1 = 0.0f;
    if (live) {
        en = a.list[e];
        b = (int)(en.y >> META_SHIFT);
        const int y = en.x >> 16, x = en.x & 0xffff;
        const int sl = slice_of(a.sl, b);
        philox4x32_10_rk(local_index(slice_rect(a.sl, sl), y, x), ctr1,
                         (a.r_base + (uint32_t)rl) >> 1, 0u, a.rng.rk0, slice_key1(a.sl, sl), w);
        if (a.beta_pts) {
            beta = a.beta_pts[(size_t)(rl % a.n_pts) * a.g.nblk + b];
            beta1 = a.beta_pts[(size_t)((rl + 1) % a.n_pts) * a.g.nblk + b];
        } else {
            beta = a.beta[b];
            beta1 = a.beta_odd ? a.beta_odd[b] : beta;
        }
    }
    grid_dep_wait();
    __syncthreads();
    float ao0 = 0.f, ao1 = 0.f, al0 = 0.f, al1 = 0.f, au0 = 0.f, au1 = 0.f;
    uint32_t f = 0;
    if (live) {
        const size_t plane = (size_t)a.g.H * a.g.Wh;
        const int c = a.colour, co = c ^ 1;
        bool run0, run1;
        pair_running(a, b, rl, run0, run1);
        if (run0 || run1) {
            float2* own = reinterpret_cast<float2*>(static_cast<float*>(a.ang) + (size_t)(grp * 2 + c) * plane * G) + q;
            const float2* oth =
                reinterpret_cast<const float2*>(static_cast<const float*>(a.ang) + (size_t)(grp * 2 + co) * plane * G) + q;
            const int y = en.x >> 16, x = en.x & 0xffff;
            f = en.y;
            const uint32_t hs = (uint32_t)y * (uint32_t)a.g.Wh + (uint32_t)(x >> 1);
            const float2 ph = own[(size_t)hs * NP];
            float nc0[4], ns0[4], nc1[4], ns1[4];
            neighbour_field<float>(a, reinterpret_cast<const float*>(oth), G, hs, x, f, nc0, ns0,
                                   nc1, ns1);
            const float C0 = (nc0[0] + nc0[1]) + (nc0[2] + nc0[3]);
            const float S0 = (ns0[0] + ns0[1]) + (ns0[2] + ns0[3]);
            const float C1 = (nc1[0] + nc1[1]) + (nc1[2] + nc1[3]);
            const float S1 = (ns1[0] + ns1[1]) + (ns1[2] + ns1[3]);
            float2 out = ph;
            if (run0) {
                const SiteNew n = site_update<float>(ph.x, C0, S0, u01(w[0]), u01(w[1]), beta, a.m);
                out.x = n.phi;
                add_energy(n, f, C0, S0, nc0, ns0, a.m.J, ao0, al0, au0);
            }
            if (run1) {
                const SiteNew n = site_update<float>(ph.y, C1, S1, u01(w[2]), u01(w[3]), beta1, a.m);
                out.y = n.phi;
                add_energy(n, f, C1, S1, nc1, ns1, a.m.J, ao1, al1, au1);
            }
            own[(size_t)hs * NP] = out;
        }
    }
    if (!a.energy) return;
    // The block's share: one warp sum per realization lane when the warp's
    // entries all lie in one block (the usual case: the list is block-major),
    // else an atomic per lane; shared-memory sums for the CTA's first blocks.
    const int lane = threadIdx.x & 31;
    if (__all_sync(0xffffffffu, b == __shfl_sync(0xffffffffu, b, 0))) {
#pragma unroll
        for (int d = 16; d >= NP; d >>= 1) {
            ao0 += __shfl_xor_sync(0xffffffffu, ao0, d);
            ao1 += __shfl_xor_sync(0xffffffffu, ao1, d);
        }
        if (lane < NP) {
            const int loc = b - b0;
            if (loc < kFlatBlocks) {
                if (ao0 != 0.0f) atomicAdd(&acc[loc * G + 2 * lane], ao0);
                if (ao1 != 0.0f) atomicAdd(&acc[loc * G + 2 * lane + 1], ao1);
            } else {
                double* ea = a.eacc + (size_t)b * a.Rp + grp * G + 2 * lane;
                if (ao0 != 0.0f) atomicAdd(ea, (double)ao0);
                if (ao1 != 0.0f) atomicAdd(ea + 1, (double)ao1);
            }
        }
    } else if (live) {
        const int loc = b - b0;
        if (loc < kFlatBlocks) {
            if (ao0 != 0.0f) atomicAdd(&acc[loc * G + 2 * q], ao0);
            if (ao1 != 0.0f) atomicAdd(&acc[loc * G + 2 * q + 1], ao1);
        } else {
            double* ea = a.eacc + (size_t)b * a.Rp + rl;
            if (ao0 != 0.0f) atomicAdd(ea, (double)ao0);
            if (ao1 != 0.0f) atomicAdd(ea + 1, (double)ao1);
        }
    }
    // Left / up bonds of edge sites belong to the neighbouring blocks.
    if (f & (EDGE_L | EDGE_U)) {
        double* ea = a.eacc + (size_t)b * a.Rp + rl;
        if (al0 != 0.0f) atomicAdd(ea - a.Rp, (double)al0);
        if (al1 != 0.0f) atomicAdd(ea - a.Rp + 1, (double)al1);
        const size_t up = (size_t)a.g.nbx * a.Rp;
        if (au0 != 0.0f) atomicAdd(ea - up, (double)au0);
        if (au1 != 0.0f) atomicAdd(ea - up + 1, (double)au1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kFlatBlocks * G; i += kFlatThreads) {
        const float v = acc[i];
        if (v != 0.0f) atomicAdd(&a.eacc[(size_t)(b0 + i / G) * a.Rp + grp * G + (i % G)], (double)v);
    }
}

// Energies from scratch (no move) of one item: the bonds that touch a gap
// site of this colour and belong to no gap site of the other colour (colour
// 1 counts all bonds of its gap sites, colour 0 only those to sample
// neighbours). Each lane sums its few bonds in FP32; the warp sums and the
// block totals are FP64.
template <int G, typename S>
__device__ __forceinline__ void energy_item(const SweepArgs& a, int item, int wi, int wpi) {
    constexpr int NP = G / 2;
    const int lane = threadIdx.x & 31;
    const int q = wi % NP, cw = wi / NP, CW = wpi / NP;
    const size_t plane = (size_t)a.g.H * a.g.Wh;
    const int c = a.colour, co = c ^ 1;
    const int b = item / a.groups, grp = item - b * a.groups;
    const int rl = grp * G + 2 * q;
    const int e0 = a.start[b], e1 = a.start[b + 1];
    const S* own = static_cast<const S*>(a.ang) + (size_t)(grp * 2 + c) * plane * G + 2 * q;
    const S* oth = static_cast<const S*>(a.ang) + (size_t)(grp * 2 + co) * plane * G + 2 * q;
    float o0 = 0.f, o1 = 0.f, l0 = 0.f, l1 = 0.f, u0 = 0.f, u1 = 0.f;
    for (int e = e0 + cw * 32 + lane; e < e1; e += CW * 32) {
        const uint2 en = a.list[e];
        const int y = en.x >> 16, x = en.x & 0xffff;
        const uint32_t f = en.y;
        const uint32_t hs = (uint32_t)y * (uint32_t)a.g.Wh + (uint32_t)(x >> 1);
        const float2 ph = Store<S>::load2(own + (size_t)hs * G);
        float nc0[4], ns0[4], nc1[4], ns1[4];
        neighbour_field<S>(a, oth, G, hs, x, f, nc0, ns0, nc1, ns1);
        float s0, c0, s1, c1;
        __sincosf(a.m.q * ph.x, &s0, &c0);
        __sincosf(a.m.q * ph.y, &s1, &c1);
        const uint32_t take = (c == 1) ? 0xFu : (~(f >> 4) & 0xFu);
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            if (!((f & (NB_L << d)) && (take & (1u << d)))) continue;
            const float b0 = -a.m.J * (c0 * nc0[d] + s0 * ns0[d]);
            const float b1 = -a.m.J * (c1 * nc1[d] + s1 * ns1[d]);
            if (d == 0 && (f & EDGE_L)) { l0 += b0; l1 += b1; }
            else if (d == 2 && (f & EDGE_U)) { u0 += b0; u1 += b1; }
            else { o0 += b0; o1 += b1; }
        }
    }
    double v[6] = {o0, o1, l0, l1, u0, u1};
#pragma unroll
    for (int s = 16; s > 0; s >>= 1)
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], s);
    if (lane != 0) return;
    double* ea = a.ecur + (size_t)b * a.Rp + rl;
    const size_t up = (size_t)a.g.nbx * a.Rp;
    if (v[0] != 0.0) atomicAdd(ea, v[0]);
    if (v[1] != 0.0) atomicAdd(ea + 1, v[1]);
    if (v[2] != 0.0) atomicAdd(ea - a.Rp, v[2]);
    if (v[3] != 0.0) atomicAdd(ea - a.Rp + 1, v[3]);
    if (v[4] != 0.0) atomicAdd(ea - up, v[4]);
    if (v[5] != 0.0) atomicAdd(ea - up + 1, v[5]);
}

// The stop test after sweep t_sweep, on the items of the sweep's worklist
// (every running (block, realization) pair belongs to one of them), in two
// parts: the second needs the final per-realization count of running
// targeted blocks, which the first completes.
//
// Targeted part: E_b += the sweep's change (eacc, then cleared); e_b = E_b / N_b;
// a targeted block stops once sigma (e_b(t) - e_s,b) >= 0 (CROSS), or, under the
// WINDOW rule, at a test sweep t = n_fit + n_f + k n_f once the least-squares
// slope of e_b over sweeps t - n_fit + 1 .. t no longer has the sign sigma
// (its numerator sum_j (2 j - (n_fit - 1)) e_b(t - n_fit + 1 + j)). Entries
// i = i0, i0 + step, ... < n of (item, lane) pairs (n = items * G). Entries
// below `cap` are readable whatever n is (the worklist buffer's length times
// G; past n they hold stale items), so the first item is read without waiting
// for n; every value of an entry is then read at once, and only then tested.
// U entries per pass: a pass reads all of its entries' values before it tests
// any of them, so U loads of each kind are in flight per thread (the test is
// latency-bound: an entry's loads wait for the worklist word naming its
// block). Entries are independent (each (block, realization) appears once).
template <int U = 1>
__device__ __forceinline__ void stop_targeted_range(const StopArgs& s, uint32_t t_sweep,
                                                    const uint32_t* __restrict__ w, int64_t n,
                                                    int64_t cap, int64_t i0, int64_t step) {
    for (int64_t ib = i0; ib < n; ib += (int64_t)U * step) {
        uint32_t item[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = ib + (int64_t)u * step;
            item[u] = i < cap ? w[i / s.G] : 0u;
        }
        size_t k[U];
        int b[U], r[U], sg[U];
        int32_t nsp[U], ob[U];
        uint8_t run[U];
        double E[U], inb[U], es[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = ib + (int64_t)u * step;
            b[u] = (int)(item[u] / (uint32_t)s.groups);
            r[u] = (int)(item[u] % (uint32_t)s.groups) * s.G + (int)(i % s.G);
            k[u] = (size_t)b[u] * s.Rp + r[u];
            const bool v = i < n;
            run[u] = v ? s.running[k[u]] : (uint8_t)0;
            E[u] = v ? s.ecur[k[u]] + s.eacc[k[u]] : 0.0;
            inb[u] = v ? s.inb[b[u]] : 0.0;
            es[u] = v ? s.es[b[u]] : 0.0;
            nsp[u] = v ? s.Nsp[b[u]] : 0;
            ob[u] = v ? s.of_block[b[u]] : 0;
            sg[u] = v ? s.sigma[k[u]] : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!run[u]) continue;
            s.eacc[k[u]] = 0.0;
            s.ecur[k[u]] = E[u];
            const double e = E[u] * inb[u];
            s.e_last[k[u]] = e;
            bool reached;
            if (s.win.rule == 1) {
                const int nf = s.win.n_fit;
                s.win.hist[(size_t)(t_sweep % (uint32_t)nf) * s.win.stride + k[u]] = e;
                if (nsp[u] == 0) continue;
                const uint32_t first = (uint32_t)(nf + s.win.n_f);
                if (t_sweep < first || (t_sweep - first) % (uint32_t)s.win.n_f != 0) continue;
                double num = 0.0;
                for (int j = 0; j < nf; ++j) {
                    const uint32_t sw = t_sweep - (uint32_t)nf + 1u + (uint32_t)j;
                    num += (double)(2 * j - (nf - 1)) *
                           s.win.hist[(size_t)(sw % (uint32_t)nf) * s.win.stride + k[u]];
                }
                reached = (double)sg[u] * num <= 0.0;
            } else {
                if (nsp[u] == 0) continue;
                reached = sg[u] > 0 ? (e >= es[u]) : (sg[u] < 0 ? (e <= es[u]) : true);
            }
            if (reached) {
                s.running[k[u]] = 0;
                s.stop[k[u]] = (int32_t)t_sweep;
                atomicSub(&s.tcount[ob[u] * s.Rp + r[u]], 1);
            }
        }
    }
}

// Closing part: blocks without sample bonds stop when no targeted block of
// their realization runs; everything stops at n_max. Items with a lane still
// running are appended to `out` (counter *n_out, one atomic per warp, items in
// lane order). Items i = i0, i0 + step, ... < n of the worklist w (nullptr:
// every item); `cap` as for the targeted part. Returns this thread's count of
// lanes still running.
__device__ __forceinline__ unsigned stop_rest_range(const StopArgs& s, uint32_t t_sweep,
                                                    const uint32_t* __restrict__ w, int64_t n,
                                                    int64_t cap, uint32_t* __restrict__ out,
                                                    uint32_t* n_out, int64_t i0, int64_t step) {
    unsigned cnt = 0;
    uint32_t item = w ? (i0 < cap ? w[i0] : 0u) : (uint32_t)i0;
    for (int64_t i = i0; i < n; i += step) {
        if (i != i0) item = w ? w[i] : (uint32_t)i;
        const int b = (int)(item / (uint32_t)s.groups), grp = (int)(item % (uint32_t)s.groups);
        const int32_t ob = s.of_block[b], nsp = s.Nsp[b];
        const int32_t* tc = s.tcount + (size_t)(ob < 0 ? 0 : ob) * s.Rp;
        bool any = false;
        for (int g = 0; g < s.G; ++g) {
            const int r = grp * s.G + g;
            const size_t k = (size_t)b * s.Rp + r;
            if (!s.running[k]) continue;
            if ((nsp == 0 && tc[r] == 0) || (int)t_sweep >= s.n_max) {
                s.running[k] = 0;
                s.stop[k] = (int32_t)t_sweep;
            } else {
                ++cnt;
                any = true;
            }
        }
        const unsigned act = __activemask();
        const unsigned vote = __ballot_sync(act, any);
        if (vote) {
            const int lane = threadIdx.x & 31;
            const int leader = __ffs(vote) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(n_out, (uint32_t)__popc(vote));
            base = __shfl_sync(act, base, leader);
            if (any) out[base + __popc(vote & ((1u << lane) - 1u))] = item;
        }
    }
    return cnt;
}

// ------------------------------------------------- grid-wide barrier --
// For cooperative launches (the persistent calibration and the simulation's
// stop tail). The barrier never waits forever: a CTA that has waited `limit`
// polls sets the error flag and returns false, and every CTA that sees the
// flag returns false too; the host then reports MPR_ETIMEOUT. A test hook
// (`extra`) makes the barrier wait for arrivals that never come, to exercise
// that path.
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Barrier over all CTAs of the launch. `gen` is the generation this CTA last
// passed (kept by thread 0). The last CTA to arrive runs last() (thread 0)
// before it releases the others, so its writes are visible to every CTA
// after the barrier. Returns false if the wait gave up here or elsewhere.
template <typename F>
__device__ bool grid_sync_then(GridBarrier* bar, unsigned int& gen, unsigned long long limit,
                               F&& last) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = ld_acquire(&bar->err) == 0;
        if (ok) {
            const unsigned int target = gen + 1;
            const unsigned int expect = gridDim.x + bar->extra;
            __threadfence();
            const unsigned int arrived = atomicAdd(&bar->arrive, 1u) + 1u;
            if (arrived == expect) {
                __threadfence();
                last();
                atomicExch(&bar->arrive, 0u);
                __threadfence();
                atomicExch(&bar->gen, target);
            } else {
                unsigned long long spins = 0;
                while (ld_acquire(&bar->gen) != target) {
                    if (ld_acquire(&bar->err) != 0) {
                        ok = 0;
                        break;
                    }
                    if (++spins > limit) {
                        atomicExch(&bar->err, 1u);
                        ok = 0;
                        break;
                    }
                    __nanosleep(100);
                }
            }
            __threadfence();
            gen = target;
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ bool grid_sync(GridBarrier* bar, unsigned int& gen,
                                          unsigned long long limit) {
    return grid_sync_then(bar, gen, limit, [] {});
}

// Median of the targeted blocks' T by a radix select over the (positive)
// float bit patterns, run by one CTA over the blocks of one slice (the block
// rectangle bk = (by0, bx0, nby_s, nbx_s) of a canvas nbx blocks wide); k is
// the 0-based rank.
__device__ inline uint32_t select_kth(const float* __restrict__ T, const int32_t* __restrict__ Nsp,
                                      int4 bk, int nbx, uint32_t k, uint32_t* hist,
                                      uint32_t* s_digit, uint32_t* s_k) {
    const int nb = bk.z * bk.w;
    uint32_t prefix = 0, pmask = 0;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        for (int j = threadIdx.x; j < nb; j += blockDim.x) {
            const int b = (bk.x + j / bk.w) * nbx + bk.y + j % bk.w;
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
// blocks' T within one slice, by one CTA; 0 when no block is targeted.
__device__ inline float median_targeted(const float* __restrict__ T, const int32_t* __restrict__ Nsp,
                                        int4 bk, int nbx) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t s_digit, s_k, s_n;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    const int nb = bk.z * bk.w;
    uint32_t cnt = 0;
    for (int j = threadIdx.x; j < nb; j += blockDim.x)
        cnt += Nsp[(bk.x + j / bk.w) * nbx + bk.y + j % bk.w] > 0;
    atomicAdd(&s_n, cnt);
    __syncthreads();
    const uint32_t n = s_n;
    float med = 0.0f;
    if (n > 0) {
        const float lo =
            __uint_as_float(select_kth(T, Nsp, bk, nbx, (n - 1) / 2, hist, &s_digit, &s_k));
        const float hi = (n & 1) ? lo
                                 : __uint_as_float(select_kth(T, Nsp, bk, nbx, n / 2, hist,
                                                              &s_digit, &s_k));
        med = 0.5f * (lo + hi);
    }
    return med;
}

}  // namespace mpr
