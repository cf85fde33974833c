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

// One warp per block: write the gap entries of both colours in row-major
// order into the block's list segments (ballot-based stable compaction).
__global__ void k_build_lists(Geom g, const uint8_t* __restrict__ mask,
                              const int32_t* __restrict__ start0, const int32_t* __restrict__ start1,
                              uint2* __restrict__ list0, uint2* __restrict__ list1) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= g.nblk) return;
    const int b = warp;
    const int by = b / g.nbx, bx = b % g.nbx;
    const int y0 = by * g.lb, x0 = bx * g.lb;
    const int y1 = min(g.H, y0 + g.lb), x1 = min(g.W, x0 + g.lb);
    const int bw = x1 - x0, nsite = (y1 - y0) * bw;
    int o0 = start0[b], o1 = start1[b];
    for (int j0 = 0; j0 < nsite; j0 += 32) {
        const int j = j0 + lane;
        bool gap = false;
        int y = 0, x = 0, c = 0;
        if (j < nsite) {
            y = y0 + j / bw;
            x = x0 + j % bw;
            gap = mask[(int64_t)y * g.W + x] != 0;
            c = (x + y) & 1;
        }
        const unsigned m0 = __ballot_sync(0xffffffffu, gap && c == 0);
        const unsigned m1 = __ballot_sync(0xffffffffu, gap && c == 1);
        if (gap) {
            const int64_t i = (int64_t)y * g.W + x;
            uint32_t f = 0;
            if (x > 0) { f |= NB_L; if (mask[i - 1]) f |= GAP_L; }
            if (x + 1 < g.W) { f |= NB_R; if (mask[i + 1]) f |= GAP_R; }
            if (y > 0) { f |= NB_U; if (mask[i - g.W]) f |= GAP_U; }
            if (y + 1 < g.H) { f |= NB_D; if (mask[i + g.W]) f |= GAP_D; }
            if (x > 0 && x % g.lb == 0) f |= EDGE_L;
            if (y > 0 && y % g.lb == 0) f |= EDGE_U;
            const uint2 e = make_uint2(((uint32_t)y << 16) | (uint32_t)x,
                                       ((uint32_t)b << META_SHIFT) | f);
            const unsigned below = (1u << lane) - 1u;
            if (c == 0) list0[o0 + __popc(m0 & below)] = e;
            else list1[o1 + __popc(m1 & below)] = e;
        }
        o0 += __popc(m0);
        o1 += __popc(m1);
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

// ----------------------------------------------------------------- sweep --
// One checkerboard half-step. A warp owns one (block, lane-group) work item
// and walks the block's list of gap sites of the colour; lane = slot * G +
// realization lane. With G >= 2 each lane pair (realizations 2m, 2m+1)
// shares Philox blocks: the even lane draws for site A, the odd lane for
// site B, and the two swap the halves they do not own.
//
// Bond energies for the stop test are summed here. A bond always joins a
// colour-0 and a colour-1 site; the colour-1 half-step adds every bond of its
// gap sites (their colour-0 partners are final for the sweep); the colour-0
// half-step adds the bonds of its gap sites to sample neighbours (those
// partners never move). Bonds between two samples are the constant E_s,b.
// A bond is owned by the block of its left / upper site.
template <int G>
__global__ void __launch_bounds__(256) k_halfstep(SweepArgs a) {
    constexpr int S = 32 / G;                 // list slots per warp pass
    constexpr int PER = (G >= 2) ? 2 : 1;     // entries per slot per pass
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const int slot = lane / G;
    const int warps = gridDim.x * (blockDim.x >> 5);
    const int n_items = a.g.nblk * a.groups;
    const int c = a.colour, co = c ^ 1;
    const size_t plane = (size_t)a.g.H * a.g.Wh;
    const uint32_t ctr1 = a.t | (a.tag << 16);

    for (int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < n_items;
         item += warps) {
        const int b = item / a.groups;
        const int grp = item - b * a.groups;
        const int e0 = a.start[b], e1 = a.start[b + 1];
        if (e0 == e1) continue;
        const int rl = grp * G + gl;                     // lane realization in the batch
        bool run_own = true, run_l = false, run_u = false;
        if (a.running) {
            run_own = a.running[(size_t)b * a.Rp + rl] != 0;
            if (a.energy) {
                const int bx = b % a.g.nbx;
                run_l = bx > 0 && a.running[(size_t)(b - 1) * a.Rp + rl] != 0;
                run_u = b >= a.g.nbx && a.running[(size_t)(b - a.g.nbx) * a.Rp + rl] != 0;
            }
        } else {
            run_own = rl < a.R;
            run_l = run_own && a.energy && (b % a.g.nbx) > 0;
            run_u = run_own && a.energy && b >= a.g.nbx;
        }
        if (!__any_sync(0xffffffffu, run_own || run_l || run_u)) continue;
        const bool move = a.update && run_own;
        float* own = a.ang + (size_t)(grp * 2 + c) * plane * G;
        const float* oth = a.ang + (size_t)(grp * 2 + co) * plane * G;
        const float2* dco = a.dcs + (size_t)co * plane;
        const float beta = a.beta[b];
        const uint32_t rg = a.r_base + (uint32_t)rl;   // global realization index
        double d_own = 0.0;
        float f_own = 0.0f, f_l = 0.0f, f_u = 0.0f;
        int fold = 0;

        for (int base = e0; base < e1; base += S * PER) {
            uint2 ent[PER];
            bool val[PER];
#pragma unroll
            for (int p = 0; p < PER; ++p) {
                const int e = base + slot * PER + p;
                val[p] = e < e1;
                ent[p] = val[p] ? a.list[e] : make_uint2(0u, 0u);
            }
            // Random numbers: words (2(r&1), 2(r&1)+1) of the block for
            // counter (site, t | tag << 16, r >> 1, 0).
            float u0[PER], u1[PER];
            if (a.update) {
                if constexpr (G >= 2) {
                    const bool odd = (gl & 1) != 0;
                    const uint2 mine = odd ? ent[1] : ent[0];
                    const uint32_t site = (mine.x >> 16) * (uint32_t)a.g.W + (mine.x & 0xffffu);
                    uint32_t w[4];
                    philox4x32_10(site, ctr1, rg >> 1, 0u, a.rng.key0, a.rng.key1, w);
                    const uint32_t sx = odd ? w[0] : w[2];
                    const uint32_t sy = odd ? w[1] : w[3];
                    const uint32_t rx = __shfl_xor_sync(0xffffffffu, sx, 1);
                    const uint32_t ry = __shfl_xor_sync(0xffffffffu, sy, 1);
                    // even: A = (w0, w1) own, B = (rx, ry); odd: A = (rx, ry), B = (w2, w3)
                    u0[0] = u01(odd ? rx : w[0]);
                    u1[0] = u01(odd ? ry : w[1]);
                    u0[1] = u01(odd ? w[2] : rx);
                    u1[1] = u01(odd ? w[3] : ry);
                } else {
                    const uint32_t site = (ent[0].x >> 16) * (uint32_t)a.g.W + (ent[0].x & 0xffffu);
                    uint32_t w[4];
                    philox4x32_10(site, ctr1, rg >> 1, 0u, a.rng.key0, a.rng.key1, w);
                    const int o = (rg & 1u) * 2;
                    u0[0] = u01(o ? w[2] : w[0]);
                    u1[0] = u01(o ? w[3] : w[1]);
                }
            }
#pragma unroll
            for (int p = 0; p < PER; ++p) {
                if (!val[p]) continue;
                const int y = ent[p].x >> 16, x = ent[p].x & 0xffff;
                const uint32_t f = ent[p].y;
                const size_t hs = (size_t)y * a.g.Wh + (x >> 1);
                // Neighbour field and, per neighbour, (cos, sin) of q*phi_j.
                float nc[4], ns[4];
                const int ny[4] = {y, y, y - 1, y + 1};
                const int nx[4] = {x - 1, x + 1, x, x};
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    nc[d] = 0.0f;
                    ns[d] = 0.0f;
                    if (f & (NB_L << d)) {
                        const size_t hn = (size_t)ny[d] * a.g.Wh + (nx[d] >> 1);
                        if (f & (GAP_L << d)) {
                            const float pj = oth[hn * G + gl];
                            __sincosf(a.m.q * pj, &ns[d], &nc[d]);
                        } else {
                            const float2 cs = __ldg(&dco[hn]);
                            nc[d] = cs.x;
                            ns[d] = cs.y;
                        }
                    }
                }
                const float C = (nc[0] + nc[1]) + (nc[2] + nc[3]);
                const float Sg = (ns[0] + ns[1]) + (ns[2] + ns[3]);
                const float phi = own[hs * G + gl];
                float cn, sn;
                if (move) {
                    const SiteNew n = site_update(phi, C, Sg, u0[p], u1[p], beta, a.m);
                    own[hs * G + gl] = n.phi;
                    cn = n.c;
                    sn = n.s;
                } else {
                    __sincosf(a.m.q * phi, &sn, &cn);
                }
                if (a.energy) {
                    // colour 1: every bond; colour 0: bonds to sample neighbours.
                    const uint32_t take = (c == 1) ? 0xFu : (~(f >> 4) & 0xFu);
                    float eb[4];
#pragma unroll
                    for (int d = 0; d < 4; ++d)
                        eb[d] = ((f & (NB_L << d)) && (take & (1u << d)))
                                    ? -a.m.J * (cn * nc[d] + sn * ns[d])
                                    : 0.0f;
                    // right and down are always owned by b; left / up by b only
                    // inside the block.
                    f_own += eb[1] + eb[3];
                    if (f & EDGE_L) f_l += eb[0]; else f_own += eb[0];
                    if (f & EDGE_U) f_u += eb[2]; else f_own += eb[2];
                }
            }
            if (a.energy && ++fold == 8) {
                d_own += (double)f_own;
                f_own = 0.0f;
                fold = 0;
            }
        }
        if (a.energy) {
            d_own += (double)f_own;
            double d_l = (double)f_l, d_u = (double)f_u;
            // Sum over the slots that share a realization lane.
#pragma unroll
            for (int d = G; d < 32; d <<= 1) {
                d_own += __shfl_xor_sync(0xffffffffu, d_own, d);
                d_l += __shfl_xor_sync(0xffffffffu, d_l, d);
                d_u += __shfl_xor_sync(0xffffffffu, d_u, d);
            }
            if (slot == 0 && rl < a.Rp) {
                if (run_own) atomicAdd(&a.eacc[(size_t)b * a.Rp + rl], d_own);
                if (run_l && d_l != 0.0) atomicAdd(&a.eacc[(size_t)(b - 1) * a.Rp + rl], d_l);
                if (run_u && d_u != 0.0)
                    atomicAdd(&a.eacc[(size_t)(b - a.g.nbx) * a.Rp + rl], d_u);
            }
        }
    }
}

template __global__ void k_halfstep<1>(SweepArgs);
template __global__ void k_halfstep<8>(SweepArgs);
template __global__ void k_halfstep<32>(SweepArgs);

// ------------------------------------------------------------------ stop --
// t = 0: E_b(0) = E_s,b + eacc, sigma = sign(e_s,b - e_b(0)), blocks without
// gap sites stop at 0; counts the running targeted blocks per realization.
__global__ void k_stop_init(int nblk, int Rp, int R, int r_off, const double* __restrict__ Es,
                            const int32_t* __restrict__ Nsp, const int32_t* __restrict__ Nb,
                            const int32_t* __restrict__ ngap, double* __restrict__ eacc,
                            int8_t* __restrict__ sigma, uint8_t* __restrict__ running,
                            int32_t* __restrict__ stop, int32_t* __restrict__ tcount,
                            double* __restrict__ e_last) {
    const int64_t n = (int64_t)nblk * Rp;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / Rp), r = (int)(t % Rp);
        const bool valid = r >= r_off && r < r_off + R;
        const double E0 = Es[b] + eacc[t];
        eacc[t] = 0.0;
        e_last[t] = Nb[b] > 0 ? E0 / (double)Nb[b] : 0.0;
        int8_t sg = 0;
        if (Nsp[b] > 0 && Nb[b] > 0) {
            const double es = Es[b] / (double)Nsp[b];
            const double e0 = E0 / (double)Nb[b];
            sg = (int8_t)((es > e0) - (es < e0));
        }
        sigma[t] = sg;
        const bool run = valid && ngap[b] > 0;
        running[t] = run;
        stop[t] = valid ? (run ? -1 : 0) : 0;
        if (run && Nsp[b] > 0) atomicAdd(&tcount[r], 1);
    }
}

// After sweep t, targeted blocks: stop once sigma (e_b(t) - e_s,b) >= 0.
// e_last keeps e_b(t) of every running (block, realization) for inspection.
__global__ void k_stop_targeted(int nblk, int Rp, int t_sweep, const double* __restrict__ Es,
                                const int32_t* __restrict__ Nsp, const int32_t* __restrict__ Nb,
                                double* __restrict__ eacc, const int8_t* __restrict__ sigma,
                                uint8_t* __restrict__ running, int32_t* __restrict__ stop,
                                int32_t* __restrict__ tcount, double* __restrict__ e_last) {
    const int64_t n = (int64_t)nblk * Rp;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / Rp), r = (int)(t % Rp);
        const double acc = eacc[t];
        eacc[t] = 0.0;
        if (!running[t]) continue;
        const double e = Nb[b] > 0 ? (Es[b] + acc) / (double)Nb[b] : 0.0;
        e_last[t] = e;
        if (Nsp[b] == 0) continue;
        const double es = Es[b] / (double)Nsp[b];
        if ((double)sigma[t] * (e - es) >= 0.0) {
            running[t] = 0;
            stop[t] = t_sweep;
            atomicSub(&tcount[r], 1);
        }
    }
}

// Blocks without sample bonds stop when no targeted block of their
// realization runs; every block stops at n_max. Counts what still runs.
__global__ void k_stop_rest(int nblk, int Rp, int t_sweep, int n_max,
                            const int32_t* __restrict__ Nsp, uint8_t* __restrict__ running,
                            int32_t* __restrict__ stop, const int32_t* __restrict__ tcount,
                            unsigned long long* __restrict__ n_running) {
    const int64_t n = (int64_t)nblk * Rp;
    unsigned cnt = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (!running[t]) continue;
        const int b = (int)(t / Rp), r = (int)(t % Rp);
        if ((Nsp[b] == 0 && tcount[r] == 0) || t_sweep >= n_max) {
            running[t] = 0;
            stop[t] = t_sweep;
        } else {
            ++cnt;
        }
    }
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(n_running, (unsigned long long)cnt);
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
                           float* __restrict__ hi, double* __restrict__ ebar) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        lo[b] = t_lo;
        hi[b] = t_hi;
        ebar[b] = 0.0;
    }
}

// Targeted blocks take their bracket midpoint; others are set by k_cal_fill.
__global__ void k_cal_mid(int nblk, const int32_t* __restrict__ Nsp, const float* __restrict__ lo,
                          const float* __restrict__ hi, float* __restrict__ T) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x)
        T[b] = Nsp[b] > 0 ? 0.5f * (lo[b] + hi[b]) : 0.0f;
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
        const float a = __uint_as_float(select_kth(T, Nsp, nblk, (n - 1) / 2, hist, &s_digit, &s_k));
        const float b = (n & 1) ? a
                                : __uint_as_float(select_kth(T, Nsp, nblk, n / 2, hist, &s_digit, &s_k));
        med = 0.5f * (a + b);
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

// After a measured sweep: e_b summed over the chains of the batch.
__global__ void k_cal_measure(int nblk, int Rp, int chains, const double* __restrict__ Es,
                              const int32_t* __restrict__ Nb, double* __restrict__ eacc,
                              double* __restrict__ ebar) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < chains; ++r) {
            const double acc = eacc[(size_t)b * Rp + r];
            eacc[(size_t)b * Rp + r] = 0.0;
            if (Nb[b] > 0) s += (Es[b] + acc) / (double)Nb[b];
        }
        ebar[b] += s;
    }
}

// Bisection step: <e_b> increases with T, so keep the half containing e_s,b.
__global__ void k_cal_update(int nblk, double inv_count, const double* __restrict__ Es,
                             const int32_t* __restrict__ Nsp, const float* __restrict__ T,
                             float* __restrict__ lo, float* __restrict__ hi,
                             double* __restrict__ ebar, double* __restrict__ trace) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        const double e = ebar[b] * inv_count;
        ebar[b] = 0.0;
        if (trace) trace[b] = e;
        if (Nsp[b] <= 0) continue;
        const double es = Es[b] / (double)Nsp[b];
        if (e < es) lo[b] = T[b]; else hi[b] = T[b];
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
                        const int32_t* start1, uint2* list0, uint2* list1, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (int)(((int64_t)g.nblk * 32 + threads - 1) / threads);
    k_build_lists<<<blocks, threads, 0, s>>>(g, mask, start0, start1, list0, list1);
}

void launch_init(const Geom& g, const uint2* list, int64_t n_list, int colour,
                 const float* init_angle, float* ang, int G, int Rp, int random, Rng rng,
                 uint32_t r_even, cudaStream_t s) {
    if (n_list == 0) return;
    k_init<<<grid_for(n_list * Rp, 256), 256, 0, s>>>(g, list, n_list, colour, init_angle, ang, G,
                                                     Rp, random, rng, r_even);
}

void launch_halfstep(const SweepArgs& a, int G, int n_sm, cudaStream_t s) {
    const int threads = 256;
    const int64_t items = (int64_t)a.g.nblk * a.groups;
    const int64_t want = (items + 7) / 8;
    const int blocks = (int)(want < (int64_t)n_sm * 8 ? want : (int64_t)n_sm * 8);
    switch (G) {
        case 1: k_halfstep<1><<<blocks, threads, 0, s>>>(a); break;
        case 8: k_halfstep<8><<<blocks, threads, 0, s>>>(a); break;
        default: k_halfstep<32><<<blocks, threads, 0, s>>>(a); break;
    }
}

void launch_stop_init(int nblk, int Rp, int R, int r_off, const double* Es, const int32_t* Nsp,
                      const int32_t* Nb, const int32_t* ngap, double* eacc, int8_t* sigma,
                      uint8_t* running, int32_t* stop, int32_t* tcount, double* e_last,
                      cudaStream_t s) {
    k_stop_init<<<grid_for((int64_t)nblk * Rp, 256), 256, 0, s>>>(
        nblk, Rp, R, r_off, Es, Nsp, Nb, ngap, eacc, sigma, running, stop, tcount, e_last);
}

void launch_stop_targeted(int nblk, int Rp, int t, const double* Es, const int32_t* Nsp,
                          const int32_t* Nb, double* eacc, const int8_t* sigma, uint8_t* running,
                          int32_t* stop, int32_t* tcount, double* e_last, cudaStream_t s) {
    k_stop_targeted<<<grid_for((int64_t)nblk * Rp, 256), 256, 0, s>>>(
        nblk, Rp, t, Es, Nsp, Nb, eacc, sigma, running, stop, tcount, e_last);
}

void launch_stop_rest(int nblk, int Rp, int t, int n_max, const int32_t* Nsp, uint8_t* running,
                      int32_t* stop, const int32_t* tcount, unsigned long long* n_running,
                      cudaStream_t s) {
    k_stop_rest<<<grid_for((int64_t)nblk * Rp, 256), 256, 0, s>>>(nblk, Rp, t, n_max, Nsp,
                                                                  running, stop, tcount, n_running);
}

void launch_count_updates(int nblk, int Rp, const int32_t* stop, const int32_t* ngap,
                          unsigned long long* total, cudaStream_t s) {
    k_count_updates<<<grid_for((int64_t)nblk * Rp, 256), 256, 0, s>>>(nblk, Rp, stop, ngap, total);
}

void launch_cal_init(int nblk, float t_lo, float t_hi, float* lo, float* hi, double* ebar,
                     cudaStream_t s) {
    k_cal_init<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, t_lo, t_hi, lo, hi, ebar);
}

void launch_cal_mid(int nblk, const int32_t* Nsp, const float* lo, const float* hi, float* T,
                    cudaStream_t s) {
    k_cal_mid<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, Nsp, lo, hi, T);
}

void launch_cal_fill(int nblk, const int32_t* Nsp, float* T, float* beta, cudaStream_t s) {
    k_cal_fill<<<1, 1024, 0, s>>>(nblk, Nsp, T, beta);
}

void launch_cal_measure(int nblk, int Rp, int chains, const double* Es, const int32_t* Nb,
                        double* eacc, double* ebar, cudaStream_t s) {
    k_cal_measure<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, Rp, chains, Es, Nb, eacc, ebar);
}

void launch_cal_update(int nblk, double inv_count, const double* Es, const int32_t* Nsp,
                       const float* T, float* lo, float* hi, double* ebar, double* trace,
                       cudaStream_t s) {
    k_cal_update<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, inv_count, Es, Nsp, T, lo, hi, ebar,
                                                    trace);
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
