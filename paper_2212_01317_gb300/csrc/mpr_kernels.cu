// sm_103a kernels of the SV-MPR hot path (Lach & Zukovic, arXiv 2212.01317).
//
//   setup    Sec. 2.1 transform, Eq. 2 per block (Sec. 2.2.2), gap lists
//   init     Sec. 3.3.3 block-mean start
//   sweep    Sec. 2.2.2 checkerboard half-step: Metropolis + over-relaxation
//            of the gap sites of one colour, fused with the bond-energy sums
//            that feed the local-equilibrium stop (Sec. 3.4)
//   stop     per (block, realization) stop decisions
//   calib    per-block bisection of T by energy matching (Sec. 2.1, 2.2.2)
//   predict  conditional mean and back-transform (Sec. 2.1, 3.2), Eqs. 3-4
#include <cuda_runtime.h>

#include <cstdint>

#include "mpr_device.cuh"
#include "mpr_internal.h"
#include "mpr_launch.h"

namespace mpr {

namespace {

__device__ __forceinline__ size_t hidx(const Geom& g, int c, int y, int x) {
    return ((size_t)c * g.H + y) * g.Wh + (x >> 1);
}

// Order-preserving map of a float onto uint32 (for atomic min/max).
__device__ __forceinline__ uint32_t f2ord(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

}  // namespace

float ord2f(uint32_t u) {
    uint32_t v = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    __builtin_memcpy(&f, &v, 4);
    return f;
}

// ---------------------------------------------------------------- setup --
// z_min / z_max over the samples (Sec. 2.1: only the samples are known).
__global__ void k_minmax(const float* __restrict__ values, const uint8_t* __restrict__ mask,
                         int64_t n, uint32_t* __restrict__ mm) {
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (mask[i]) continue;
        const uint32_t o = f2ord(values[i]);
        lo = min(lo, o);
        hi = max(hi, o);
    }
    for (int d = 16; d > 0; d >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&mm[0], lo);
        atomicMax(&mm[1], hi);
    }
}

// Sample angles and their (cos, sin) of q*phi, per checkerboard colour.
__global__ void k_layout(Geom g, const float* __restrict__ values, const uint8_t* __restrict__ mask,
                         double zmin, double zmax, int degenerate, float q,
                         float* __restrict__ dang, float2* __restrict__ dcs) {
    const int64_t n = (int64_t)g.H * g.W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / g.W), x = (int)(i % g.W);
        const int c = (x + y) & 1;
        const size_t h = hidx(g, c, y, x);
        if (mask[i]) {
            dang[h] = 0.0f;
            dcs[h] = make_float2(0.0f, 0.0f);
            continue;
        }
        const double phi = degenerate ? 0.0
                                      : 6.283185307179586476925 * ((double)values[i] - zmin) /
                                            (zmax - zmin);
        const float pf = (float)phi;
        dang[h] = pf;
        double s, co;
        sincos((double)q * phi, &s, &co);
        dcs[h] = make_float2((float)co, (float)s);
    }
}

// One warp per block: Eq. 2 over the owned sample-sample bonds (FP64), bond
// counts, sample mean angle, gap counts per colour.
__global__ void k_block_stats(Geom g, const float* __restrict__ values,
                              const uint8_t* __restrict__ mask, double zmin, double zmax,
                              int degenerate, double q, double J, double* __restrict__ Es,
                              int32_t* __restrict__ Nsp, int32_t* __restrict__ Nb,
                              double* __restrict__ ssum, int32_t* __restrict__ nsamp,
                              int32_t* __restrict__ ngap0, int32_t* __restrict__ ngap1) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= g.nblk) return;
    const int by = warp / g.nbx, bx = warp % g.nbx;
    const int y0 = by * g.lb, x0 = bx * g.lb;
    const int y1 = min(g.H, y0 + g.lb), x1 = min(g.W, x0 + g.lb);
    const int bw = x1 - x0, nsite = (y1 - y0) * bw;
    const double scale = degenerate ? 0.0 : 6.283185307179586476925 / (zmax - zmin);
    double es = 0.0, sm = 0.0;
    int nsp = 0, nb = 0, ns = 0, g0 = 0, g1 = 0;
    for (int j = lane; j < nsite; j += 32) {
        const int y = y0 + j / bw, x = x0 + j % bw;
        const int64_t i = (int64_t)y * g.W + x;
        const bool gap = mask[i] != 0;
        const double pi = gap ? 0.0 : ((double)values[i] - zmin) * scale;
        if (gap) {
            if (((x + y) & 1) == 0) ++g0; else ++g1;
        } else {
            sm += pi;
            ++ns;
        }
        if (x + 1 < g.W) {
            ++nb;
            if (!gap && !mask[i + 1]) {
                const double pj = ((double)values[i + 1] - zmin) * scale;
                es += -J * cos(q * (pi - pj));
                ++nsp;
            }
        }
        if (y + 1 < g.H) {
            ++nb;
            if (!gap && !mask[i + g.W]) {
                const double pj = ((double)values[i + g.W] - zmin) * scale;
                es += -J * cos(q * (pi - pj));
                ++nsp;
            }
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        es += __shfl_xor_sync(0xffffffffu, es, d);
        sm += __shfl_xor_sync(0xffffffffu, sm, d);
        nsp += __shfl_xor_sync(0xffffffffu, nsp, d);
        nb += __shfl_xor_sync(0xffffffffu, nb, d);
        ns += __shfl_xor_sync(0xffffffffu, ns, d);
        g0 += __shfl_xor_sync(0xffffffffu, g0, d);
        g1 += __shfl_xor_sync(0xffffffffu, g1, d);
    }
    if (lane == 0) {
        Es[warp] = es;
        Nsp[warp] = nsp;
        Nb[warp] = nb;
        ssum[warp] = sm;
        nsamp[warp] = ns;
        ngap0[warp] = g0;
        ngap1[warp] = g1;
    }
}

// Exclusive scan of n counts into out[0..n] by one CTA of 1024 threads.
__global__ void k_scan_counts(const int32_t* __restrict__ cnt, int n, int32_t* __restrict__ out) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int per = (n + 1023) / 1024;
    const int a = min(n, t * per), b = min(n, a + per);
    int64_t s = 0;
    for (int i = a; i < b; ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        int64_t v = t >= d ? part[t - d] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - s;
    for (int i = a; i < b; ++i) {
        out[i] = (int32_t)run;
        run += cnt[i];
    }
    if (t == 1023) out[n] = (int32_t)part[1023];
}

// One warp per block: write the gap entries of both colours into the block's
// list segments, ballot-compacted: first the sites whose left or up bond
// belongs to a neighbouring block (block edge), then the others, each group
// in row-major order. Keeping the edge sites together lets most warps of the
// sweep skip the per-bond energy split.
__global__ void k_build_lists(Geom g, const uint8_t* __restrict__ mask,
                              const int32_t* __restrict__ start0, const int32_t* __restrict__ start1,
                              uint2* __restrict__ list0, uint2* __restrict__ list1,
                              int32_t* __restrict__ split0, int32_t* __restrict__ split1) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= g.nblk) return;
    const int b = warp;
    const int by = b / g.nbx, bx = b % g.nbx;
    const int y0 = by * g.lb, x0 = bx * g.lb;
    const int y1 = min(g.H, y0 + g.lb), x1 = min(g.W, x0 + g.lb);
    const int bw = x1 - x0, nsite = (y1 - y0) * bw;
    int o0 = start0[b], o1 = start1[b];
    for (int pass = 0; pass < 2; ++pass) {
        for (int j0 = 0; j0 < nsite; j0 += 32) {
            const int j = j0 + lane;
            bool take = false;
            int y = 0, x = 0, c = 0;
            if (j < nsite) {
                y = y0 + j / bw;
                x = x0 + j % bw;
                const bool edge = (x > 0 && x == x0) || (y > 0 && y == y0);
                take = mask[(int64_t)y * g.W + x] != 0 && edge == (pass == 0);
                c = (x + y) & 1;
            }
            const unsigned m0 = __ballot_sync(0xffffffffu, take && c == 0);
            const unsigned m1 = __ballot_sync(0xffffffffu, take && c == 1);
            if (take) {
                const int64_t i = (int64_t)y * g.W + x;
                uint32_t f = 0;
                if (x > 0) { f |= NB_L; if (mask[i - 1]) f |= GAP_L; }
                if (x + 1 < g.W) { f |= NB_R; if (mask[i + 1]) f |= GAP_R; }
                if (y > 0) { f |= NB_U; if (mask[i - g.W]) f |= GAP_U; }
                if (y + 1 < g.H) { f |= NB_D; if (mask[i + g.W]) f |= GAP_D; }
                if (x > 0 && x == x0) f |= EDGE_L;
                if (y > 0 && y == y0) f |= EDGE_U;
                const uint2 e = make_uint2(((uint32_t)y << 16) | (uint32_t)x,
                                           ((uint32_t)b << META_SHIFT) | f);
                const unsigned below = (1u << lane) - 1u;
                if (c == 0) list0[o0 + __popc(m0 & below)] = e;
                else list1[o1 + __popc(m1 & below)] = e;
            }
            o0 += __popc(m0);
            o1 += __popc(m1);
        }
        if (pass == 0 && lane == 0) {
            split0[b] = o0;   // end of the block's edge entries
            split1[b] = o1;
        }
    }
}

// ------------------------------------------------------------------ init --
// Sec. 3.3.3: every gap site starts from the sample mean angle of its block
// (global sample mean when the block has no sample); random start (plain
// MPR) draws 2*pi*u from the reserved tag 0xFFFF.
__global__ void k_init(Geom g, const uint2* __restrict__ list, int64_t n_list, int colour,
                       const float* __restrict__ init_angle, float* __restrict__ ang, int G,
                       int Rp, int random, Rng rng, uint32_t r_even) {
    const int64_t total = n_list * Rp;
    const size_t plane = (size_t)g.H * g.Wh;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = t / Rp;
        const int r = (int)(t % Rp);
        const uint2 en = list[e];
        const int y = en.x >> 16, x = en.x & 0xffff;
        const int b = en.y >> META_SHIFT;
        float v = init_angle[b];
        if (random) {
            const uint32_t gr = r_even + (uint32_t)r;
            uint32_t w[4];
            philox4x32_10((uint32_t)((int64_t)y * g.W + x), 0u | (0xFFFFu << 16), gr >> 1, 0u,
                          rng.key0, rng.key1, w);
            v = kTwoPi * u01(w[(gr & 1u) * 2u]);
        }
        const int grp = r / G, lane = r % G;
        ang[(((size_t)(grp * 2 + colour) * plane) + (size_t)y * g.Wh + (x >> 1)) * G + lane] = v;
    }
}

// Sample angles copied into every lane of the batch state, so that a
// neighbour read is the same load whether the neighbour is a gap or a sample.
__global__ void k_fill_samples(Geom g, const uint8_t* __restrict__ mask,
                               const float* __restrict__ dang, float* __restrict__ ang, int G,
                               int groups) {
    const int64_t n = (int64_t)g.H * g.W;
    const size_t plane = (size_t)g.H * g.Wh;
    const int64_t total = n * groups;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t % n;
        const int grp = (int)(t / n);
        if (mask[i]) continue;
        const int y = (int)(i / g.W), x = (int)(i % g.W);
        const int c = (x + y) & 1;
        const size_t hs = (size_t)y * g.Wh + (x >> 1);
        const float v = dang[(size_t)c * plane + hs];
        float* dst = ang + ((size_t)(grp * 2 + c) * plane + hs) * G;
        for (int l = 0; l < G; ++l) dst[l] = v;
    }
}

// ----------------------------------------------------------------- sweep --
// One checkerboard half-step (Sec. 2.2.2) over the running (block, lane
// group) items of a batch. The state interleaves G realizations per site; a
// CTA of four warps takes one item, warp w handles the realization pair
// (group * G + 2q, + 1), q = w mod G/2, and its 32 lanes walk the block's
// list of gap sites 32 at a time (warps sharing a pair split the list). Each
// lane updates its site in both realizations of the pair from one Philox
// block: words 0, 1 for the even realization, 2, 3 for the odd one.
//
// Block energies are kept incrementally: a Metropolis move changes the
// energy of the site's four bonds by dE and the reflection conserves it, so a
// site whose bonds all belong to its own block adds dE there. A site on the
// left or top edge of its block splits the change bond by bond, because its
// left / up bond belongs to the neighbouring block (a bond is owned by the
// block of its left / upper site). Frozen sites never move, so stopped
// (block, realization) pairs cost nothing.
namespace {

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

// Interior sites: only the block's own change.
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

// The same for the from-scratch energies, in FP64 into the block energies.
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

}  // namespace

// Interior sites of each block (the segment after its edge entries): every
// bond of the site belongs to the block, so the block's energy changes by the
// Metropolis dE (the reflection conserves it).
template <int G>
__global__ void __launch_bounds__(128) k_sweep(SweepArgs a) {
    constexpr int NP = G / 2;        // realization pairs per lane group
    constexpr int CW = 4 / NP;       // warps sharing one pair
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp % NP, cw = warp / NP;
    const uint32_t ctr1 = a.ctl->t | (a.ctl->tag << 16);
    const int n_items = a.work ? (int)a.ctl->n_work : a.g.nblk * a.groups;
    const size_t plane = (size_t)a.g.H * a.g.Wh;
    const int c = a.colour, co = c ^ 1;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int item = a.work ? (int)a.work[it] : it;
        const int b = item / a.groups, grp = item - b * a.groups;
        const int e0 = a.split[b], e1 = a.start[b + 1];
        if (e0 >= e1) continue;
        const int rl = grp * G + 2 * q;
        bool run0, run1;
        if (a.running) {
            run0 = a.running[(size_t)b * a.Rp + rl] != 0;
            run1 = a.running[(size_t)b * a.Rp + rl + 1] != 0;
        } else {
            run0 = rl < a.R;
            run1 = rl + 1 < a.R;
        }
        if (!(run0 || run1)) continue;
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
            philox4x32_10((uint32_t)y * (uint32_t)a.g.W + (uint32_t)x, ctr1, rpair, 0u,
                          a.rng.key0, a.rng.key1, w);
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
}

// Edge sites of each block (left / top edge: the left / up bond belongs to
// the neighbouring block, so the energy change is split bond by bond). A
// block has few of them, so one warp takes a whole (block, lane group) item:
// lane = entry slot * (G/2) + pair, i.e. 32/(G/2) entries times all pairs per
// pass, and one site's G realizations are read as one contiguous chunk.
template <int G>
__global__ void __launch_bounds__(128) k_sweep_edge(SweepArgs a) {
    constexpr int NP = G / 2;
    constexpr int EPI = 32 / NP;     // entries per warp pass
    const int lane = threadIdx.x & 31;
    const int q = lane % NP, el = lane / NP;
    const int wpb = blockDim.x >> 5;
    const int nwarps = gridDim.x * wpb;
    const uint32_t ctr1 = a.ctl->t | (a.ctl->tag << 16);
    const int n_items = a.work ? (int)a.ctl->n_work : a.g.nblk * a.groups;
    const size_t plane = (size_t)a.g.H * a.g.Wh;
    const int c = a.colour, co = c ^ 1;
    for (int it = blockIdx.x * wpb + (threadIdx.x >> 5); it < n_items; it += nwarps) {
        const int item = a.work ? (int)a.work[it] : it;
        const int b = item / a.groups, grp = item - b * a.groups;
        const int e0 = a.start[b], e1 = a.split[b];
        if (e0 >= e1) continue;
        const int rl = grp * G + 2 * q;
        bool run0, run1;
        if (a.running) {
            run0 = a.running[(size_t)b * a.Rp + rl] != 0;
            run1 = a.running[(size_t)b * a.Rp + rl + 1] != 0;
        } else {
            run0 = rl < a.R;
            run1 = rl + 1 < a.R;
        }
        if (!__any_sync(0xffffffffu, run0 || run1)) continue;
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
            philox4x32_10((uint32_t)y * (uint32_t)a.g.W + (uint32_t)x, ctr1, rpair, 0u,
                          a.rng.key0, a.rng.key1, w);
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
        if (!a.energy) continue;
        // Sum over the entry slots of each pair, then the slot-0 lane of each
        // pair adds to the blocks.
#pragma unroll
        for (int s = NP; s < 32; s <<= 1) {
            ao0 += __shfl_xor_sync(0xffffffffu, ao0, s);
            ao1 += __shfl_xor_sync(0xffffffffu, ao1, s);
            al0 += __shfl_xor_sync(0xffffffffu, al0, s);
            al1 += __shfl_xor_sync(0xffffffffu, al1, s);
            au0 += __shfl_xor_sync(0xffffffffu, au0, s);
            au1 += __shfl_xor_sync(0xffffffffu, au1, s);
        }
        if (el != 0) continue;
        float* ea = a.eacc + (size_t)b * a.Rp + rl;
        if (ao0 != 0.0f) atomicAdd(ea, ao0);
        if (ao1 != 0.0f) atomicAdd(ea + 1, ao1);
        if (al0 != 0.0f) atomicAdd(ea - a.Rp, al0);
        if (al1 != 0.0f) atomicAdd(ea - a.Rp + 1, al1);
        const size_t up = (size_t)a.g.nbx * a.Rp;
        if (au0 != 0.0f) atomicAdd(ea - up, au0);
        if (au1 != 0.0f) atomicAdd(ea - up + 1, au1);
    }
}

// Energies from scratch (no move): every bond that touches a gap site, once.
// A bond always joins a colour-0 and a colour-1 site; colour 1 adds every
// bond of its gap sites, colour 0 the bonds of its gap sites to samples.
// Bonds between two samples are the constant E_s,b.
template <int G>
__global__ void __launch_bounds__(128) k_energy(SweepArgs a) {
    constexpr int NP = G / 2;
    constexpr int CW = 4 / NP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp % NP, cw = warp / NP;
    const int n_items = a.g.nblk * a.groups;
    const size_t plane = (size_t)a.g.H * a.g.Wh;
    const int c = a.colour, co = c ^ 1;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int b = it / a.groups, grp = it - b * a.groups;
        const int rl = grp * G + 2 * q;
        bool run0, run1;
        if (a.running) {
            run0 = a.running[(size_t)b * a.Rp + rl] != 0;
            run1 = a.running[(size_t)b * a.Rp + rl + 1] != 0;
        } else {
            run0 = rl < a.R;
            run1 = rl + 1 < a.R;
        }
        if (!(run0 || run1)) continue;
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
            const size_t hs = (size_t)y * a.g.Wh + (x >> 1);
            const float2 ph = own[hs * NP];
            float nc0[4], ns0[4], nc1[4], ns1[4];
            neighbour_field(a, oth, NP, (uint32_t)hs, x, f, nc0, ns0, nc1, ns1);
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
}

template __global__ void k_sweep<2>(SweepArgs);
template __global__ void k_sweep<8>(SweepArgs);
template __global__ void k_sweep_edge<2>(SweepArgs);
template __global__ void k_sweep_edge<8>(SweepArgs);
template __global__ void k_energy<2>(SweepArgs);
template __global__ void k_energy<8>(SweepArgs);

// Advances the sweep index and hands the worklist built by the last stop
// test to the sweep that starts.
__global__ void k_tick(Control* ctl) {
    ctl->t += 1;
    ctl->n_work = ctl->n_work_next;
    ctl->n_work_next = 0;
    ctl->n_running = 0;
}

// ------------------------------------------------------------------ stop --
// es[b] = E_s,b / N_SP,b (0 without sample bonds) and inb[b] = 1 / N_b (0 for
// a block that owns no bond) are computed once at create, in FP64.

// E_b <- E_s,b for every (block, lane): the constant sample-sample part; the
// energy pass then adds the bonds that touch a gap site.
__global__ void k_ecur_reset(int nblk, int Rp, const double* __restrict__ Es,
                             double* __restrict__ ecur, float* __restrict__ eacc) {
    const int64_t n = (int64_t)nblk * Rp;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        ecur[t] = Es[t / Rp];
        eacc[t] = 0.0f;
    }
}

// t = 0: sigma = sign(e_s,b - e_b(0)), blocks without gap sites stop at 0;
// counts the running targeted blocks of every realization. `running` holds 1
// for the batch's lanes on entry.
__global__ void k_stop_init(int nblk, int Rp, const double* __restrict__ es,
                            const double* __restrict__ inb, const int32_t* __restrict__ Nsp,
                            const int32_t* __restrict__ ngap, const double* __restrict__ ecur,
                            int8_t* __restrict__ sigma, uint8_t* __restrict__ running,
                            int32_t* __restrict__ stop, int32_t* __restrict__ tcount,
                            double* __restrict__ e_last) {
    const int64_t n = (int64_t)nblk * Rp;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / Rp), r = (int)(t % Rp);
        const bool valid = running[t] != 0;
        const double e0 = ecur[t] * inb[b];
        e_last[t] = e0;
        int8_t sg = 0;
        if (Nsp[b] > 0 && inb[b] > 0.0) sg = (int8_t)((es[b] > e0) - (es[b] < e0));
        sigma[t] = sg;
        const bool run = valid && ngap[b] > 0;
        running[t] = run;
        stop[t] = run ? -1 : 0;
        if (run && Nsp[b] > 0) atomicAdd(&tcount[r], 1);
    }
}

// After sweep t: E_b += the sweep's change; targeted blocks stop once
// sigma (e_b(t) - e_s,b) >= 0. e_last keeps e_b(t) for inspection.
__global__ void k_stop_targeted(int nblk, int Rp, const Control* __restrict__ ctl,
                                const double* __restrict__ es, const double* __restrict__ inb,
                                const int32_t* __restrict__ Nsp, float* __restrict__ eacc,
                                double* __restrict__ ecur, const int8_t* __restrict__ sigma,
                                uint8_t* __restrict__ running, int32_t* __restrict__ stop,
                                int32_t* __restrict__ tcount, double* __restrict__ e_last) {
    const int64_t n = (int64_t)nblk * Rp;
    const int t_sweep = (int)ctl->t;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const float acc = eacc[t];
        if (acc != 0.0f) eacc[t] = 0.0f;
        if (!running[t]) continue;
        const int b = (int)(t / Rp), r = (int)(t % Rp);
        const double E = ecur[t] + (double)acc;
        ecur[t] = E;
        const double e = E * inb[b];
        e_last[t] = e;
        if (Nsp[b] == 0) continue;
        const int sg = sigma[t];
        const bool reached = sg > 0 ? (e >= es[b]) : (sg < 0 ? (e <= es[b]) : true);
        if (reached) {
            running[t] = 0;
            stop[t] = t_sweep;
            atomicSub(&tcount[r], 1);
        }
    }
}

// Blocks without sample bonds stop when no targeted block of their
// realization runs; every block stops at n_max. One thread per (block, lane
// group) item: items with a running lane go on the next sweep's worklist.
__global__ void k_stop_rest(int nblk, int groups, int G, int Rp, int n_max,
                            Control* __restrict__ ctl, const int32_t* __restrict__ Nsp,
                            uint8_t* __restrict__ running, int32_t* __restrict__ stop,
                            const int32_t* __restrict__ tcount, uint32_t* __restrict__ work) {
    const int64_t n = (int64_t)nblk * groups;
    const int t_sweep = (int)ctl->t;
    unsigned cnt = 0;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < n;
         it += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(it / groups), grp = (int)(it % groups);
        bool any = false;
        for (int g = 0; g < G; ++g) {
            const int r = grp * G + g;
            const size_t k = (size_t)b * Rp + r;
            if (!running[k]) continue;
            if ((Nsp[b] == 0 && tcount[r] == 0) || t_sweep >= n_max) {
                running[k] = 0;
                stop[k] = t_sweep;
            } else {
                ++cnt;
                any = true;
            }
        }
        if (any) work[atomicAdd(&ctl->n_work_next, 1u)] = (uint32_t)it;
    }
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&ctl->n_running, (unsigned long long)cnt);
}

// Site updates run by the batch: sum over (b, r) of stop sweep x gap sites.
__global__ void k_count_updates(int nblk, int Rp, const int32_t* __restrict__ stop,
                                const int32_t* __restrict__ ngap,
                                unsigned long long* __restrict__ total) {
    const int64_t n = (int64_t)nblk * Rp;
    unsigned long long s = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / Rp);
        if (stop[t] > 0) s += (unsigned long long)stop[t] * (unsigned long long)ngap[b];
    }
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(total, s);
}

// ----------------------------------------------------------- calibration --
__global__ void k_cal_init(int nblk, float t_lo, float t_hi, float* __restrict__ lo,
                           float* __restrict__ hi, double* __restrict__ ebar, Control* ctl) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        lo[b] = t_lo;
        hi[b] = t_hi;
        ebar[b] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->k = 0;
}

// Targeted blocks take their bracket midpoint (others: k_cal_fill); starts
// iteration ctl->k: random-stream tag 1 + k, sweep counter 0.
__global__ void k_cal_mid(int nblk, const int32_t* __restrict__ Nsp, const float* __restrict__ lo,
                          const float* __restrict__ hi, float* __restrict__ T, Control* ctl) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x)
        T[b] = Nsp[b] > 0 ? 0.5f * (lo[b] + hi[b]) : 0.0f;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->tag = 1u + ctl->k;
        ctl->t = 0;
    }
}

// Median of the targeted blocks' T by a single-CTA radix select on the
// (positive) float bit patterns; even counts average the two middle values.
__device__ uint32_t select_kth(const float* __restrict__ T, const int32_t* __restrict__ Nsp,
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

__global__ void k_cal_fill(int nblk, const int32_t* __restrict__ Nsp, float* __restrict__ T,
                           float* __restrict__ beta) {
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
        const float hi = (n & 1) ? lo
                                 : __uint_as_float(select_kth(T, Nsp, nblk, n / 2, hist, &s_digit, &s_k));
        med = 0.5f * (lo + hi);
    }
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        float tb = T[b];
        if (Nsp[b] <= 0) {
            tb = med;
            T[b] = med;
        }
        beta[b] = tb > 0.0f ? 1.0f / tb : 0.0f;
    }
}

// After calibration sweep t: fold the sweep's change into E_b; past n_eq
// sweeps add e_b of every chain to the running sum.
__global__ void k_cal_step(int nblk, int Rp, int chains, int n_eq, const Control* __restrict__ ctl,
                           const double* __restrict__ inb, float* __restrict__ eacc,
                           double* __restrict__ ecur, double* __restrict__ ebar) {
    const bool measure = (int)ctl->t > n_eq;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < chains; ++r) {
            const size_t k = (size_t)b * Rp + r;
            const double E = ecur[k] + (double)eacc[k];
            ecur[k] = E;
            eacc[k] = 0.0f;
            s += E * inb[b];
        }
        if (measure) ebar[b] += s;
    }
}

// Bisection step: <e_b> increases with T, so keep the half containing e_s,b.
// Inside the calibration graph, one thread also decides whether the loop over
// iterations goes on (cond != 0: graph conditional handle of the loop).
__global__ void k_cal_update(int nblk, double inv_count, const double* __restrict__ es,
                             const int32_t* __restrict__ Nsp, const float* __restrict__ T,
                             float* __restrict__ lo, float* __restrict__ hi,
                             double* __restrict__ ebar, Control* ctl, int n_bisect,
                             cudaGraphConditionalHandle cond) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        const double e = ebar[b] * inv_count;
        ebar[b] = 0.0;
        if (Nsp[b] <= 0) continue;
        if (e < es[b]) lo[b] = T[b]; else hi[b] = T[b];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t k = ctl->k + 1;
        ctl->k = k;
        if (cond) cudaGraphSetConditional(cond, k < (uint32_t)n_bisect ? 1u : 0u);
    }
}

// --------------------------------------------------------------- predict --
// Adds the batch's final angles of every gap site to the running sums.
__global__ void k_accumulate(Geom g, const uint2* __restrict__ list, int64_t n_list, int colour,
                             const float* __restrict__ ang, int G, int groups, int r_off, int R,
                             double* __restrict__ sum) {
    const size_t plane = (size_t)g.H * g.Wh;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_list;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint2 en = list[e];
        const int y = en.x >> 16, x = en.x & 0xffff;
        const size_t hs = (size_t)y * g.Wh + (x >> 1);
        double s = 0.0;
        for (int r = r_off; r < r_off + R; ++r) {
            const int grp = r / G, lane = r % G;
            s += (double)ang[((size_t)(grp * 2 + colour) * plane + hs) * G + lane];
        }
        sum[(size_t)colour * plane + hs] += s;
    }
}

// Sec. 2.1 back-transform of the conditional mean; samples copied bit for bit.
__global__ void k_predict(Geom g, const float* __restrict__ values,
                          const uint8_t* __restrict__ mask, const double* __restrict__ sum,
                          double inv_r, double zmin, double zmax, float* __restrict__ out,
                          const float* __restrict__ truth, double* __restrict__ err) {
    const int64_t n = (int64_t)g.H * g.W;
    double ea = 0.0, e2 = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!mask[i]) {
            out[i] = values[i];
            continue;
        }
        const int y = (int)(i / g.W), x = (int)(i % g.W);
        const double mphi = sum[hidx(g, (x + y) & 1, y, x)] * inv_r;
        const float z = (float)(zmin + (zmax - zmin) * mphi / 6.283185307179586476925);
        out[i] = z;
        if (truth) {
            const double e = (double)truth[i] - (double)z;
            ea += fabs(e);
            e2 += e * e;
        }
    }
    if (truth) {
        for (int d = 16; d > 0; d >>= 1) {
            ea += __shfl_xor_sync(0xffffffffu, ea, d);
            e2 += __shfl_xor_sync(0xffffffffu, e2, d);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&err[0], ea);
            atomicAdd(&err[1], e2);
        }
    }
}

// ------------------------------------------------------- state access --
__global__ void k_get_state(Geom g, const uint8_t* __restrict__ mask, const float* __restrict__ dang,
                            const float* __restrict__ ang, int G, int r, float* __restrict__ out) {
    const int64_t n = (int64_t)g.H * g.W;
    const size_t plane = (size_t)g.H * g.Wh;
    const int grp = r / G, lane = r % G;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / g.W), x = (int)(i % g.W);
        const int c = (x + y) & 1;
        const size_t hs = (size_t)y * g.Wh + (x >> 1);
        out[i] = mask[i] ? ang[((size_t)(grp * 2 + c) * plane + hs) * G + lane]
                         : dang[(size_t)c * plane + hs];
    }
}

__global__ void k_set_state(Geom g, const uint8_t* __restrict__ mask, float* __restrict__ ang,
                            int G, int r, const float* __restrict__ in) {
    const int64_t n = (int64_t)g.H * g.W;
    const size_t plane = (size_t)g.H * g.Wh;
    const int grp = r / G, lane = r % G;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!mask[i]) continue;
        const int y = (int)(i / g.W), x = (int)(i % g.W);
        const int c = (x + y) & 1;
        const size_t hs = (size_t)y * g.Wh + (x >> 1);
        ang[((size_t)(grp * 2 + c) * plane + hs) * G + lane] = in[i];
    }
}

// E_b from scratch in FP64 (one warp per block): Eq. 1 over the owned bonds.
__global__ void k_block_energy(Geom g, const uint8_t* __restrict__ mask,
                               const float* __restrict__ dang, const float* __restrict__ ang, int G,
                               int r, double q, double J, double* __restrict__ E) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= g.nblk) return;
    const size_t plane = (size_t)g.H * g.Wh;
    const int grp = r / G, ln = r % G;
    auto angle = [&](int y, int x) -> double {
        const int c = (x + y) & 1;
        const size_t hs = (size_t)y * g.Wh + (x >> 1);
        return mask[(int64_t)y * g.W + x] ? (double)ang[((size_t)(grp * 2 + c) * plane + hs) * G + ln]
                                          : (double)dang[(size_t)c * plane + hs];
    };
    const int by = warp / g.nbx, bx = warp % g.nbx;
    const int y0 = by * g.lb, x0 = bx * g.lb;
    const int y1 = min(g.H, y0 + g.lb), x1 = min(g.W, x0 + g.lb);
    const int bw = x1 - x0, nsite = (y1 - y0) * bw;
    double s = 0.0;
    for (int j = lane; j < nsite; j += 32) {
        const int y = y0 + j / bw, x = x0 + j % bw;
        const double pi = angle(y, x);
        if (x + 1 < g.W) s += -J * cos(q * (pi - angle(y, x + 1)));
        if (y + 1 < g.H) s += -J * cos(q * (pi - angle(y + 1, x)));
    }
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) E[warp] = s;
}

// ---------------------------------------------------------- launchers --
namespace {
inline int grid_for(int64_t n, int threads, int max_blocks = 152 * 16) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    return (int)b;
}
}  // namespace

void launch_minmax(const float* values, const uint8_t* mask, int64_t n, uint32_t* mm,
                   cudaStream_t s) {
    k_minmax<<<grid_for(n, 256), 256, 0, s>>>(values, mask, n, mm);
}

void launch_layout(const Geom& g, const float* values, const uint8_t* mask, double zmin,
                   double zmax, int degenerate, float q, float* dang, float2* dcs, cudaStream_t s) {
    k_layout<<<grid_for((int64_t)g.H * g.W, 256), 256, 0, s>>>(g, values, mask, zmin, zmax,
                                                              degenerate, q, dang, dcs);
}

void launch_block_stats(const Geom& g, const float* values, const uint8_t* mask, double zmin,
                        double zmax, int degenerate, double q, double J, double* Es, int32_t* Nsp,
                        int32_t* Nb, double* ssum, int32_t* nsamp, int32_t* ngap0, int32_t* ngap1,
                        cudaStream_t s) {
    const int threads = 256;
    const int blocks = (int)(((int64_t)g.nblk * 32 + threads - 1) / threads);
    k_block_stats<<<blocks, threads, 0, s>>>(g, values, mask, zmin, zmax, degenerate, q, J, Es,
                                             Nsp, Nb, ssum, nsamp, ngap0, ngap1);
}

void launch_scan(const int32_t* cnt, int n, int32_t* out, cudaStream_t s) {
    k_scan_counts<<<1, 1024, 0, s>>>(cnt, n, out);
}

void launch_build_lists(const Geom& g, const uint8_t* mask, const int32_t* start0,
                        const int32_t* start1, uint2* list0, uint2* list1, int32_t* split0,
                        int32_t* split1, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (int)(((int64_t)g.nblk * 32 + threads - 1) / threads);
    k_build_lists<<<blocks, threads, 0, s>>>(g, mask, start0, start1, list0, list1, split0, split1);
}

void launch_init(const Geom& g, const uint2* list, int64_t n_list, int colour,
                 const float* init_angle, float* ang, int G, int Rp, int random, Rng rng,
                 uint32_t r_even, cudaStream_t s) {
    if (n_list == 0) return;
    k_init<<<grid_for(n_list * Rp, 256), 256, 0, s>>>(g, list, n_list, colour, init_angle, ang, G,
                                                     Rp, random, rng, r_even);
}

void launch_fill_samples(const Geom& g, const uint8_t* mask, const float* dang, float* ang, int G,
                         int groups, cudaStream_t s) {
    k_fill_samples<<<grid_for((int64_t)g.H * g.W * groups, 256), 256, 0, s>>>(g, mask, dang, ang, G,
                                                                             groups);
}

void launch_sweep(const SweepArgs& a, int G, int grid, bool edge, cudaStream_t s) {
    if (G == 2) {
        if (edge) k_sweep_edge<2><<<grid, 128, 0, s>>>(a);
        else k_sweep<2><<<grid, 128, 0, s>>>(a);
    } else {
        if (edge) k_sweep_edge<8><<<grid, 128, 0, s>>>(a);
        else k_sweep<8><<<grid, 128, 0, s>>>(a);
    }
}

void launch_energy(const SweepArgs& a, int G, int grid, cudaStream_t s) {
    if (G == 2) k_energy<2><<<grid, 128, 0, s>>>(a);
    else k_energy<8><<<grid, 128, 0, s>>>(a);
}

int sweep_blocks_per_sm(int G) {
    int n = 0;
    if (G == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<2>, 128, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<8>, 128, 0);
    return n > 0 ? n : 1;
}

void launch_tick(Control* ctl, cudaStream_t s) { k_tick<<<1, 1, 0, s>>>(ctl); }

void launch_ecur_reset(int nblk, int Rp, const double* Es, double* ecur, float* eacc,
                       cudaStream_t s) {
    k_ecur_reset<<<grid_for((int64_t)nblk * Rp, 256), 256, 0, s>>>(nblk, Rp, Es, ecur, eacc);
}

void launch_stop_init(int nblk, int Rp, const double* es, const double* inb, const int32_t* Nsp,
                      const int32_t* ngap, const double* ecur, int8_t* sigma, uint8_t* running,
                      int32_t* stop, int32_t* tcount, double* e_last, cudaStream_t s) {
    k_stop_init<<<grid_for((int64_t)nblk * Rp, 256), 256, 0, s>>>(
        nblk, Rp, es, inb, Nsp, ngap, ecur, sigma, running, stop, tcount, e_last);
}

void launch_stop_targeted(int nblk, int Rp, const Control* ctl, const double* es,
                          const double* inb, const int32_t* Nsp, float* eacc, double* ecur,
                          const int8_t* sigma, uint8_t* running, int32_t* stop, int32_t* tcount,
                          double* e_last, cudaStream_t s) {
    k_stop_targeted<<<grid_for((int64_t)nblk * Rp, 256), 256, 0, s>>>(
        nblk, Rp, ctl, es, inb, Nsp, eacc, ecur, sigma, running, stop, tcount, e_last);
}

void launch_stop_rest(int nblk, int groups, int G, int Rp, int n_max, Control* ctl,
                      const int32_t* Nsp, uint8_t* running, int32_t* stop, const int32_t* tcount,
                      uint32_t* work, cudaStream_t s) {
    k_stop_rest<<<grid_for((int64_t)nblk * groups, 256), 256, 0, s>>>(
        nblk, groups, G, Rp, n_max, ctl, Nsp, running, stop, tcount, work);
}

void launch_count_updates(int nblk, int Rp, const int32_t* stop, const int32_t* ngap,
                          unsigned long long* total, cudaStream_t s) {
    k_count_updates<<<grid_for((int64_t)nblk * Rp, 256), 256, 0, s>>>(nblk, Rp, stop, ngap, total);
}

void launch_cal_init(int nblk, float t_lo, float t_hi, float* lo, float* hi, double* ebar,
                     Control* ctl, cudaStream_t s) {
    k_cal_init<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, t_lo, t_hi, lo, hi, ebar, ctl);
}

void launch_cal_mid(int nblk, const int32_t* Nsp, const float* lo, const float* hi, float* T,
                    Control* ctl, cudaStream_t s) {
    k_cal_mid<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, Nsp, lo, hi, T, ctl);
}

void launch_cal_fill(int nblk, const int32_t* Nsp, float* T, float* beta, cudaStream_t s) {
    k_cal_fill<<<1, 1024, 0, s>>>(nblk, Nsp, T, beta);
}

void launch_cal_step(int nblk, int Rp, int chains, int n_eq, const Control* ctl,
                     const double* inb, float* eacc, double* ecur, double* ebar, cudaStream_t s) {
    k_cal_step<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, Rp, chains, n_eq, ctl, inb, eacc, ecur,
                                                  ebar);
}

void launch_cal_update(int nblk, double inv_count, const double* es, const int32_t* Nsp,
                       const float* T, float* lo, float* hi, double* ebar, Control* ctl,
                       int n_bisect, cudaGraphConditionalHandle cond, cudaStream_t s) {
    k_cal_update<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, inv_count, es, Nsp, T, lo, hi, ebar,
                                                    ctl, n_bisect, cond);
}

void launch_accumulate(const Geom& g, const uint2* list, int64_t n_list, int colour,
                       const float* ang, int G, int groups, int r_off, int R, double* sum,
                       cudaStream_t s) {
    if (n_list == 0) return;
    k_accumulate<<<grid_for(n_list, 256), 256, 0, s>>>(g, list, n_list, colour, ang, G, groups,
                                                      r_off, R, sum);
}

void launch_predict(const Geom& g, const float* values, const uint8_t* mask, const double* sum,
                    double inv_r, double zmin, double zmax, float* out, const float* truth,
                    double* err, cudaStream_t s) {
    k_predict<<<grid_for((int64_t)g.H * g.W, 256), 256, 0, s>>>(g, values, mask, sum, inv_r, zmin,
                                                               zmax, out, truth, err);
}

void launch_get_state(const Geom& g, const uint8_t* mask, const float* dang, const float* ang,
                      int G, int r, float* out, cudaStream_t s) {
    k_get_state<<<grid_for((int64_t)g.H * g.W, 256), 256, 0, s>>>(g, mask, dang, ang, G, r, out);
}

void launch_set_state(const Geom& g, const uint8_t* mask, float* ang, int G, int r,
                      const float* in, cudaStream_t s) {
    k_set_state<<<grid_for((int64_t)g.H * g.W, 256), 256, 0, s>>>(g, mask, ang, G, r, in);
}

void launch_block_energy(const Geom& g, const uint8_t* mask, const float* dang, const float* ang,
                         int G, int r, double q, double J, double* E, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (int)(((int64_t)g.nblk * 32 + threads - 1) / threads);
    k_block_energy<<<blocks, threads, 0, s>>>(g, mask, dang, ang, G, r, q, J, E);
}

}  // namespace mpr
