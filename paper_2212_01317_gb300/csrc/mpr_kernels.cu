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
#include "mpr_lists.cuh"
#include "mpr_stats.cuh"
#include "mpr_sweep.cuh"

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
// z_min / z_max over the samples of one field (mask != 0: gap), into mm[0..1].
__global__ void k_minmax_field(const float* __restrict__ values, const uint8_t* __restrict__ mask,
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

// z_min / z_max over the samples of every slice (Sec. 2.1: only the samples
// are known): mm[2 s], mm[2 s + 1] as order-preserving integers.
// One warp min / max per 32 sites when their samples share a slice (the
// usual case), else an atomic per sample.
__global__ void k_minmax(Geom g, const int32_t* __restrict__ of_block,
                         const float* __restrict__ values, const uint8_t* __restrict__ mask,
                         uint32_t* __restrict__ mm) {
    const int64_t n = (int64_t)g.H * g.W;
    const int64_t n_warps = (n + 31) / 32 * 32;   // every lane of a warp runs every iteration
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_warps;
         i += (int64_t)gridDim.x * blockDim.x) {
        int s = -1;
        uint32_t lo = 0xffffffffu, hi = 0u;
        if (i < n && !mask[i]) {
            const int y = (int)(i / g.W), x = (int)(i % g.W);
            s = of_block[(y / g.lb) * g.nbx + x / g.lb];
            lo = hi = f2ord(values[i]);
        }
        int smax = s;
        for (int d = 16; d > 0; d >>= 1) smax = max(smax, __shfl_xor_sync(0xffffffffu, smax, d));
        if (__all_sync(0xffffffffu, s < 0 || s == smax)) {
            if (smax < 0) continue;
            for (int d = 16; d > 0; d >>= 1) {
                lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
                hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
            }
            if ((threadIdx.x & 31) == 0) {
                atomicMin(&mm[2 * smax], lo);
                atomicMax(&mm[2 * smax + 1], hi);
            }
        } else if (s >= 0) {
            atomicMin(&mm[2 * s], lo);
            atomicMax(&mm[2 * s + 1], hi);
        }
    }
}

// Sample angles per checkerboard colour (Sec. 2.1 transform).
__global__ void k_layout(Geom g, Slices sl, const float* __restrict__ values,
                         const uint8_t* __restrict__ mask, float* __restrict__ dang) {
    const int64_t n = (int64_t)g.H * g.W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / g.W), x = (int)(i % g.W);
        const int c = (x + y) & 1;
        const size_t h = hidx(g, c, y, x);
        if (mask[i]) {
            dang[h] = 0.0f;
            continue;
        }
        const int s = sl.of_block[(y / g.lb) * g.nbx + x / g.lb];
        const double zmin = sl.zmin[s], zmax = sl.zmax[s];
        const double phi = sl.degenerate[s] ? 0.0
                                            : 6.283185307179586476925 * ((double)values[i] - zmin) /
                                                  (zmax - zmin);
        dang[h] = (float)phi;
    }
}

// One warp per block: Eq. 2 over the owned sample-sample bonds (FP64), bond
// counts, sample mean angle, gap counts per colour.
__global__ void k_block_stats(Geom g, Slices sl, const float* __restrict__ values,
                              const uint8_t* __restrict__ mask, double q, double J,
                              double* __restrict__ Es, int32_t* __restrict__ Nsp,
                              int32_t* __restrict__ Nb, double* __restrict__ ssum,
                              int32_t* __restrict__ nsamp, int32_t* __restrict__ ngap0,
                              int32_t* __restrict__ ngap1) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= g.nblk) return;
    const int by = warp / g.nbx, bx = warp % g.nbx;
    const int y0 = by * g.lb, x0 = bx * g.lb;
    const int y1 = min(g.H, y0 + g.lb), x1 = min(g.W, x0 + g.lb);
    const int s = sl.of_block[warp];
    const double zmin = s >= 0 ? sl.zmin[s] : 0.0, zmax = s >= 0 ? sl.zmax[s] : 1.0;
    const double scale = (s < 0 || sl.degenerate[s]) ? 0.0 : 6.283185307179586476925 / (zmax - zmin);
    // A bond to the right / down neighbour exists when that site is present
    // and in the same slice (blocks never straddle slices).
    const bool right_ok = x1 < g.W && bx + 1 < g.nbx && sl.of_block[warp + 1] == s;
    const bool down_ok = y1 < g.H && by + 1 < g.nby && sl.of_block[warp + g.nbx] == s;
    const BlockSums r = block_sums<true>(values, mask, g.W, y0, x0, y1, x1, right_ok, down_ok,
                                         zmin, scale, q, J, s >= 0);
    if (lane == 0) {
        Es[warp] = r.es;
        Nsp[warp] = r.nsp;
        Nb[warp] = r.nb;
        ssum[warp] = r.sm;
        nsamp[warp] = r.ns;
        ngap0[warp] = r.g0;
        ngap1[warp] = r.g1;
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
__global__ void k_build_lists(Geom g, const int32_t* __restrict__ of_block,
                              const uint8_t* __restrict__ mask,
                              const int32_t* __restrict__ start0, const int32_t* __restrict__ start1,
                              uint2* __restrict__ list0, uint2* __restrict__ list1,
                              int32_t* __restrict__ split0, int32_t* __restrict__ split1) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= g.nblk) return;
    // Neighbours across the block's left / right / upper / lower edge exist
    // only in the same slice; within the slice, absent sites have no bonds.
    const BlockFrame fr = block_frame(g, of_block, warp);
    const int bw = fr.x1 - fr.x0, nsite = (fr.y1 - fr.y0) * bw;
    int o0 = start0[fr.b], o1 = start1[fr.b];
    for (int pass = 0; pass < 2; ++pass) {
        for (int j0 = 0; j0 < nsite; j0 += 32) {
            const int j = j0 + lane;
            bool take = false;
            int y = 0, x = 0, c = 0;
            if (j < nsite) {
                y = fr.y0 + j / bw;
                x = fr.x0 + j % bw;
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
        if (pass == 0 && lane == 0) {
            split0[fr.b] = o0;   // end of the block's edge entries
            split1[fr.b] = o1;
        }
    }
}

// ------------------------------------------------------------------ init --
// Sec. 3.3.3: every gap site starts from the sample mean angle of its block
// (global sample mean when the block has no sample); random start (plain
// MPR) draws 2*pi*u from the reserved tag 0xFFFF.
template <typename S>
__global__ void k_init(Geom g, Slices sl, const uint2* __restrict__ list, int64_t n_list,
                       int colour, const float* __restrict__ init_angle, S* __restrict__ ang, int G,
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
            const int s = sl.of_block[b];
            uint32_t w[4];
            philox4x32_10(local_index(sl.rect[s], y, x), 0u | (0xFFFFu << 16), gr >> 1, 0u,
                          rng.key0, sl.key1[s], w);
            v = kTwoPi * u01(w[(gr & 1u) * 2u]);
        }
        const int grp = r / G, lane = r % G;
        Store<S>::store1(
            ang + (((size_t)(grp * 2 + colour) * plane) + (size_t)y * g.Wh + (x >> 1)) * G + lane, v);
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
// One half-step of the batch over the worklist of running units (or every
// unit). A unit is one realization pair of one block: u = b * npairs + p
// with npairs = Rp / 2 and pair p = group * (G/2) + q, so a pair whose two
// realizations have stopped costs nothing. WPU warps take a unit (1: one
// warp per pair; 2, 4: the pair's entries split between them, for the few
// units left at the end of a batch), 128 / (32 WPU) units per CTA.
template <int G, typename S, int WPU>
__global__ void __launch_bounds__(128, 8) k_sweep(SweepArgs a) {
    grid_dep_launch();
    grid_dep_wait();
    constexpr int NP = G / 2;
    const uint32_t t = a.t_fixed > 0 ? (uint32_t)a.t_fixed : a.ctl->t;
    const uint32_t ctr1 = t | (a.ctl->tag << 16);
    const uint32_t* work = a.work ? a.work + (size_t)(t & 1u) * a.work_stride : nullptr;
    const int npairs = a.groups * NP;
    constexpr int UPC = 4 / WPU;
    const int warp = threadIdx.x >> 5;
    const int slot = warp / WPU, cw = warp % WPU;
    const int it0 = blockIdx.x * UPC + slot;
    // The worklist buffer is work_stride entries long whatever the count, so
    // the first unit is read together with the count (stale past it).
    int u = work ? (it0 < (int)a.work_stride ? (int)work[it0] : 0) : it0;
    const int n_units = work ? (int)a.ctl->n_work[t & 1u] : a.g.nblk * npairs;
    for (int it = it0; it < n_units; it += gridDim.x * UPC) {
        if (it != it0) u = work ? (int)work[it] : it;
        const int b = u / npairs, p = u - b * npairs;
        const int grp = p / NP, q = p - grp * NP;
        sweep_item<G, S>(a, b * a.groups + grp, q + NP * cw, NP * WPU, ctr1);
    }
}

// The same half-step with two units per warp (sweep_item_half), eight per
// CTA: for short per-block entry lists.
template <int G, typename S>
__global__ void __launch_bounds__(128, 8) k_sweep_half(SweepArgs a) {
    grid_dep_launch();
    grid_dep_wait();
    constexpr int NP = G / 2;
    const uint32_t t = a.t_fixed > 0 ? (uint32_t)a.t_fixed : a.ctl->t;
    const uint32_t ctr1 = t | (a.ctl->tag << 16);
    const uint32_t* work = a.work ? a.work + (size_t)(t & 1u) * a.work_stride : nullptr;
    const int npairs = a.groups * NP;
    const int warp = threadIdx.x >> 5, half = (threadIdx.x >> 4) & 1;
    const int it0 = blockIdx.x * 8 + warp * 2 + half;
    int u = work ? (it0 < (int)a.work_stride ? (int)work[it0] : 0) : it0;
    const int n_units = work ? (int)a.ctl->n_work[t & 1u] : a.g.nblk * npairs;
    // The loop bound is the warp's (both halves share the energy shuffles).
    for (int base = blockIdx.x * 8 + warp * 2; base < n_units; base += gridDim.x * 8) {
        const int it = base + half;
        const bool have = it < n_units;
        if (it != it0) u = have ? (work ? (int)work[it] : it) : 0;
        const int b = u / npairs, p = u - b * npairs;
        const int grp = p / NP, q = p - grp * NP;
        sweep_item_half<G, S>(a, b * a.groups + grp, q, have, ctr1);
    }
}

// Fold of the previous sweep's block energies by CTA `cta` of f.ctas: E_b of
// every (block, chain lane) gains the sweep's change, and during the measured
// sweeps each point's mean e_b gains E_b / N_b. It touches eacc of the other
// parity and ecur, which the half-step does not. kThreads: the CTA size.
template <int kThreads>
__device__ __forceinline__ void fold_block_energies(const FoldArgs& f, int cta) {
    for (int b = cta * kThreads + (int)threadIdx.x; b < f.nblk; b += f.ctas * kThreads) {
        double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int r = 0; r < f.chains * f.points; ++r) {
            const size_t k = (size_t)b * f.Rp + r;
            const double E = f.ecur[k] + f.eacc[k];
            f.ecur[k] = E;
            f.eacc[k] = 0.0;
            s[r % f.points] += E * f.inb[b];
        }
        if (f.measure) {
            if (f.points > 2) {
                for (int p = 0; p < f.points; ++p) f.ebar_pts[(size_t)p * f.nblk + b] += s[p];
            } else {
                f.ebar[b] += s[0];
                if (f.points == 2) f.ebar_odd[b] += s[1];
            }
        }
    }
}

// The last f.ctas CTAs (of blockIdx.y = 0) fold the previous sweep's block
// energies instead (fold_block_energies). Eight CTAs per SM (32 registers, a few spilled) keep a
// 1024^2 field's colour (262 k threads) in one wave: the calibration took
// 13.2 ms per bench step at the compiler's 47 registers (five CTAs per SM),
// 12.7 ms at six CTAs per SM and 12.0 ms at eight.
template <int G>
__global__ void __launch_bounds__(kFlatThreads, 8) k_sweep_flat(SweepArgs a, int64_t n_list,
                                                            FoldArgs f) {
    grid_dep_launch();
    const int sweep_ctas = (int)gridDim.x - f.ctas;
    if ((int)blockIdx.x >= sweep_ctas) {
        grid_dep_wait();
        if (blockIdx.y != 0) return;
        fold_block_energies<kFlatThreads>(f, (int)blockIdx.x - sweep_ctas);
        return;
    }
    // The sweep index comes from the Control only when the launch does not
    // fix it, and the Control may be written by the previous kernel: wait for
    // it first then (the prologue overlap is for launches with a fixed index).
    if (a.t_fixed <= 0) grid_dep_wait();
    const uint32_t t = a.t_fixed > 0 ? (uint32_t)a.t_fixed : a.ctl->t;
    sweep_flat<G>(a, n_list, t | (a.ctl->tag << 16));
}

// The calibration's half-step in the warp form: one warp per (block, pair)
// unit over every unit (the chains never stop), each lane at its point's
// temperature, and f.ctas trailing CTAs that fold the previous sweep as in
// k_sweep_flat. For lists of many waves, where the flat kernel's per-thread
// setup (entry, random block, temperatures, block sums) weighs on every
// update; the flat form stays for lists of a few waves, which it covers in
// one latency chain.
template <int G>
__global__ void __launch_bounds__(128, 8) k_sweep_cal(SweepArgs a, FoldArgs f) {
    grid_dep_launch();
    grid_dep_wait();
    const int sweep_ctas = (int)gridDim.x - f.ctas;
    if ((int)blockIdx.x >= sweep_ctas) {
        fold_block_energies<128>(f, (int)blockIdx.x - sweep_ctas);
        return;
    }
    constexpr int NP = G / 2;
    const uint32_t t = a.t_fixed > 0 ? (uint32_t)a.t_fixed : a.ctl->t;
    const uint32_t ctr1 = t | (a.ctl->tag << 16);
    const int npairs = a.groups * NP;
    const int n_units = a.g.nblk * npairs;
    for (int u = blockIdx.x * 4 + (int)(threadIdx.x >> 5); u < n_units; u += sweep_ctas * 4) {
        const int b = u / npairs, p = u - b * npairs;
        const int grp = p / NP, q = p - grp * NP;
        sweep_item<G, float, true>(a, b * a.groups + grp, q, NP, ctr1);
    }
}

template <int G, typename S>
__global__ void __launch_bounds__(128) k_energy(SweepArgs a) {
    const int n_items = a.g.nblk * a.groups;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x)
        energy_item<G, S>(a, it, threadIdx.x >> 5, 4);
}

template __global__ void k_sweep_flat<2>(SweepArgs, int64_t, FoldArgs);
template __global__ void k_sweep_flat<8>(SweepArgs, int64_t, FoldArgs);
template __global__ void k_sweep_cal<2>(SweepArgs, FoldArgs);
template __global__ void k_sweep_cal<8>(SweepArgs, FoldArgs);

// ------------------------------------------------------------------ stop --
// es[b] = E_s,b / N_SP,b (0 without sample bonds) and inb[b] = 1 / N_b (0 for
// a block that owns no bond) are computed once at create, in FP64.

// E_b <- E_s,b for every (block, lane): the constant sample-sample part; the
// energy pass then adds the bonds that touch a gap site.
__global__ void k_ecur_reset(int nblk, int Rp, const double* __restrict__ Es,
                             double* __restrict__ ecur, double* __restrict__ eacc) {
    const int64_t n = (int64_t)nblk * Rp;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        ecur[t] = Es[t / Rp];
        eacc[t] = 0.0;
    }
}

// t = 0: sigma = sign(e_s,b - e_b(0)), blocks without gap sites stop at 0;
// counts the running targeted blocks of every realization. `running` holds 1
// for the batch's lanes on entry.
__global__ void k_stop_init(int nblk, int Rp, const int32_t* __restrict__ of_block,
                            const double* __restrict__ es,
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
        if (run && Nsp[b] > 0) atomicAdd(&tcount[of_block[b] * Rp + r], 1);
    }
}

// The stop test after sweep t in two kernels (stop_targeted_range, then
// stop_rest_range): the second needs the final per-realization count of
// running targeted blocks, which the first completes.
//
// k_stop_targeted: one thread per (item, lane) of the sweep's worklist.
// t_known >= 0: the sweep index (the host's loop knows it), else read from ctl.
__global__ void k_stop_targeted(StopArgs sa, Control* __restrict__ ctl,
                                const uint32_t* __restrict__ work, uint32_t work_stride,
                                int t_known) {
    grid_dep_launch();
    grid_dep_wait();
    const uint32_t t_sweep = t_known >= 0 ? (uint32_t)t_known : ctl->t;
    const uint32_t* w = work + (size_t)(t_sweep & 1u) * work_stride;
    const int64_t n = (int64_t)ctl->n_work[t_sweep & 1u] * sa.G;
    stop_targeted_range<4>(sa, t_sweep, w, n, (int64_t)work_stride * sa.G,
                        blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                        (int64_t)gridDim.x * blockDim.x);
}

// k_stop_rest: one thread per item of the worklist (`work` == nullptr: every
// item, as at t = 0); items with a lane still running go on the next sweep's
// worklist. The CTA that finishes last closes the sweep: t + 1, the next
// worklist's size, the running count, and a cleared counter for the list
// after it.
__global__ void k_stop_rest(StopArgs sa, cudaGraphConditionalHandle cond,
                            Control* __restrict__ ctl, const uint32_t* __restrict__ work,
                            uint32_t* __restrict__ work_all, uint32_t work_stride, int t_known) {
    grid_dep_launch();
    grid_dep_wait();
    const uint32_t t_sweep = t_known >= 0 ? (uint32_t)t_known : ctl->t;
    const uint32_t par = t_sweep & 1u, nxt = par ^ 1u;
    const uint32_t* w = work ? work + (size_t)par * work_stride : nullptr;
    uint32_t* out = work_all + (size_t)nxt * work_stride;
    const int64_t n = w ? (int64_t)ctl->n_work[par] : (int64_t)sa.nblk * sa.groups;
    const int n_max = sa.n_max;
    unsigned cnt = stop_rest_range(sa, t_sweep, w, n, (int64_t)work_stride, out,
                                   &ctl->n_work[nxt],
                                   blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                                   (int64_t)gridDim.x * blockDim.x);
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&ctl->n_running_acc, (unsigned long long)cnt);
    // Last CTA out closes the sweep (every other CTA's atomics are visible to
    // it after its ticket: each CTA fences before taking one).
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const unsigned long long left = atomicExch(&ctl->n_running_acc, 0ull);
        ctl->n_running = left;
        ctl->n_work[par] = 0;
        ctl->ticket = 0;
        ctl->t = t_sweep + 1;
        __threadfence();
        // Inside a graph's sweep loop: continue while pairs run and sweeps remain.
        if (cond) cudaGraphSetConditional(cond, (left > 0 && (int)t_sweep < n_max) ? 1u : 0u);
    }
}

// Site updates run by the batch: sum over (b, r) of stop sweep x gap sites.
// With ctl: the updates run so far, pairs still running (stop < 0) counted
// up to the last completed sweep (ctl->t - 1).
__global__ void k_count_updates(int nblk, int Rp, const int32_t* __restrict__ stop,
                                const int32_t* __restrict__ ngap, const Control* ctl,
                                unsigned long long* __restrict__ total) {
    const int64_t n = (int64_t)nblk * Rp;
    const int32_t t_done = ctl ? (int32_t)ctl->t - 1 : 0;
    unsigned long long s = 0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / Rp);
        const int32_t st = stop[t] < 0 ? t_done : stop[t];
        if (st > 0) s += (unsigned long long)st * (unsigned long long)ngap[b];
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

// Blocks without sample bonds take the median of their slice's targeted
// blocks' T (Sec. 2.2.2); every block gets beta = 1 / T. One CTA per slice.
__global__ void k_cal_fill(Slices sl, int nbx, const int32_t* __restrict__ Nsp,
                           float* __restrict__ T, float* __restrict__ beta) {
    const int4 bk = sl.blk[blockIdx.x];
    const int nb = bk.z * bk.w;
    // The median only serves blocks that do not calibrate: skip the select
    // when the slice has none.
    int fill = 0;
    for (int j = threadIdx.x; j < nb && !fill; j += blockDim.x)
        fill = Nsp[(bk.x + j / bk.w) * nbx + bk.y + j % bk.w] <= 0;
    const float med = __syncthreads_or(fill) ? median_targeted(T, Nsp, bk, nbx) : 0.0f;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        const int b = (bk.x + j / bk.w) * nbx + bk.y + j % bk.w;
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
__global__ void k_cal_step(int nblk, int Rp, int chains, int n_eq, int t_fixed,
                           const Control* __restrict__ ctl, const double* __restrict__ inb,
                           double* __restrict__ eacc, double* __restrict__ ecur,
                           double* __restrict__ ebar, int points, double* __restrict__ ebar_odd,
                           double* __restrict__ ebar_pts) {
    const bool measure = (t_fixed > 0 ? t_fixed : (int)ctl->t) > n_eq;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int r = 0; r < chains * points; ++r) {
            const size_t k = (size_t)b * Rp + r;
            const double E = ecur[k] + eacc[k];
            ecur[k] = E;
            eacc[k] = 0.0;
            s[r % points] += E * inb[b];
        }
        if (measure) {
            if (points > 2) {
                for (int p = 0; p < points; ++p) ebar_pts[(size_t)p * nblk + b] += s[p];
            } else {
                ebar[b] += s[0];
                if (points == 2) ebar_odd[b] += s[1];
            }
        }
    }
}

// k-point calibration (4 or 8 temperatures per block and iteration, lane r
// of the chains at point r mod points): T_p = lo + (p + 1) (hi - lo) / (points
// + 1), p = 0 .. points - 1, for every targeted block (untargeted: 0, the
// median fills them in).
__global__ void k_kpts_mid(int nblk, int points, const int32_t* __restrict__ Nsp,
                           const float* __restrict__ lo, const float* __restrict__ hi,
                           float* __restrict__ Tk, Control* ctl) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        const bool t = Nsp[b] > 0;
        const float w = (hi[b] - lo[b]) / (float)(points + 1);
        for (int p = 0; p < points; ++p)
            Tk[(size_t)p * nblk + b] = t ? lo[b] + (float)(p + 1) * w : 0.0f;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->tag = 1u + ctl->k;
        ctl->t = 0;
    }
}

// k-point step: the new bracket runs from the highest point whose mean e_b is
// below e_s,b to the lowest point whose mean is not (<e_b> grows with T); the
// points' span when noise makes those cross.
__global__ void k_kpts_update(int nblk, int points, double inv_count, const double* __restrict__ es,
                              const int32_t* __restrict__ Nsp, const float* __restrict__ Tk,
                              float* __restrict__ lo, float* __restrict__ hi,
                              double* __restrict__ ebar_pts, Control* ctl, int n_iter,
                              cudaGraphConditionalHandle cond) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        float nlo = lo[b], nhi = hi[b];
        const bool t = Nsp[b] > 0;
        for (int p = 0; p < points; ++p) {
            const size_t i = (size_t)p * nblk + b;
            const double e = ebar_pts[i] * inv_count;
            ebar_pts[i] = 0.0;
            if (!t) continue;
            const float tp = Tk[i];
            if (e < es[b]) { if (tp > nlo) nlo = tp; }
            else if (tp < nhi) nhi = tp;
        }
        if (!t) continue;
        if (nlo > nhi) {
            nlo = Tk[b];
            nhi = Tk[(size_t)(points - 1) * nblk + b];
        }
        lo[b] = nlo;
        hi[b] = nhi;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t k = ctl->k + 1;
        ctl->k = k;
        if (cond) cudaGraphSetConditional(cond, k < (uint32_t)n_iter ? 1u : 0u);
    }
}

// Trisection points of every targeted block's bracket (untargeted: 0, the
// median fills them in).
__global__ void k_kcal_mid(int nblk, const int32_t* __restrict__ Nsp, const float* __restrict__ lo,
                           const float* __restrict__ hi, float* __restrict__ T0,
                           float* __restrict__ T1, Control* ctl) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        const bool t = Nsp[b] > 0;
        const float w = (hi[b] - lo[b]) / 3.0f;
        T0[b] = t ? lo[b] + w : 0.0f;
        T1[b] = t ? lo[b] + 2.0f * w : 0.0f;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->tag = 1u + ctl->k;
        ctl->t = 0;
    }
}

// Trisection step: keep the part of the bracket between the higher point
// whose mean e_b is below e_s,b and the lower point whose mean is not (the
// points' span when noise makes those cross).
__global__ void k_kcal_update(int nblk, double inv_count, const double* __restrict__ es,
                              const int32_t* __restrict__ Nsp, const float* __restrict__ T0,
                              const float* __restrict__ T1, float* __restrict__ lo,
                              float* __restrict__ hi, double* __restrict__ ebar0,
                              double* __restrict__ ebar1, Control* ctl, int n_iter,
                              cudaGraphConditionalHandle cond) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        const double e0 = ebar0[b] * inv_count, e1 = ebar1[b] * inv_count;
        ebar0[b] = 0.0;
        ebar1[b] = 0.0;
        if (Nsp[b] <= 0) continue;
        float nlo = lo[b], nhi = hi[b];
        const float t[2] = {T0[b], T1[b]};
        const double e[2] = {e0, e1};
        for (int p = 0; p < 2; ++p) {
            if (e[p] < es[b]) { if (t[p] > nlo) nlo = t[p]; }
            else if (t[p] < nhi) nhi = t[p];
        }
        if (nlo > nhi) {
            nlo = t[0];
            nhi = t[1];
        }
        lo[b] = nlo;
        hi[b] = nhi;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t k = ctl->k + 1;
        ctl->k = k;
        if (cond) cudaGraphSetConditional(cond, k < (uint32_t)n_iter ? 1u : 0u);
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
template <typename S>
__global__ void k_accumulate(Geom g, const uint2* __restrict__ list, int64_t n_list, int colour,
                             const S* __restrict__ ang, int G, int groups, int r_off, int R,
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
            s += (double)Store<S>::load1(ang + ((size_t)(grp * 2 + colour) * plane + hs) * G + lane);
        }
        sum[(size_t)colour * plane + hs] += s;
    }
}

// Half-lattice accumulator <-> row-major grid (gap sites only; 0 at samples).
__global__ void k_sum_to_grid(Geom g, const uint8_t* __restrict__ mask,
                              const double* __restrict__ sum, double* __restrict__ out) {
    const int64_t n = (int64_t)g.H * g.W;
    const size_t plane = (size_t)g.H * g.Wh;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / g.W), x = (int)(i % g.W);
        const int c = (x + y) & 1;
        out[i] = mask[i] == MASK_GAP ? sum[(size_t)c * plane + (size_t)y * g.Wh + (x >> 1)] : 0.0;
    }
}

__global__ void k_grid_to_sum(Geom g, const uint8_t* __restrict__ mask,
                              const double* __restrict__ in, double* __restrict__ sum) {
    const int64_t n = (int64_t)g.H * g.W;
    const size_t plane = (size_t)g.H * g.Wh;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / g.W), x = (int)(i % g.W);
        const int c = (x + y) & 1;
        sum[(size_t)c * plane + (size_t)y * g.Wh + (x >> 1)] = mask[i] == MASK_GAP ? in[i] : 0.0;
    }
}

// Sec. 2.1 back-transform of the conditional mean; samples copied bit for bit.
__global__ void k_predict(Geom g, Slices sl, const float* __restrict__ values,
                          const uint8_t* __restrict__ mask, const double* __restrict__ sum,
                          double inv_r, float* __restrict__ out, const float* __restrict__ truth,
                          double* __restrict__ err) {
    const int64_t n = (int64_t)g.H * g.W;
    const int64_t n_warps = (n + 31) / 32 * 32;   // every lane of a warp runs every iteration
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_warps;
         i += (int64_t)gridDim.x * blockDim.x) {
        double ea = 0.0, e2 = 0.0;
        int s = -1;
        bool gap = false;
        if (i < n) {
            const uint8_t mk = mask[i];
            const int y = (int)(i / g.W), x = (int)(i % g.W);
            s = sl.of_block[(y / g.lb) * g.nbx + x / g.lb];
            if (mk == MASK_ABSENT) {
                out[i] = 0.0f;
            } else if (mk == 0) {
                out[i] = values[i];
            } else {
                gap = true;
                const double zmin = sl.zmin[s], zmax = sl.zmax[s];
                const double mphi = sum[hidx(g, (x + y) & 1, y, x)] * inv_r;
                const float z = (float)(zmin + (zmax - zmin) * mphi / 6.283185307179586476925);
                out[i] = z;
                if (truth) {
                    const double e = (double)truth[i] - (double)z;
                    ea = fabs(e);
                    e2 = e * e;
                }
            }
        }
        if (!truth) continue;
        // Per-slice error sums (Eqs. 3-4): one warp sum when all its sites
        // share a slice, per-site atomics otherwise.
        const int s0 = __shfl_sync(0xffffffffu, s, 0);
        if (__all_sync(0xffffffffu, s == s0)) {
            for (int d = 16; d > 0; d >>= 1) {
                ea += __shfl_xor_sync(0xffffffffu, ea, d);
                e2 += __shfl_xor_sync(0xffffffffu, e2, d);
            }
            if ((threadIdx.x & 31) == 0 && s0 >= 0 && (ea != 0.0 || e2 != 0.0)) {
                atomicAdd(&err[2 * s0], ea);
                atomicAdd(&err[2 * s0 + 1], e2);
            }
        } else if (s >= 0 && gap) {
            atomicAdd(&err[2 * s], ea);
            atomicAdd(&err[2 * s + 1], e2);
        }
    }
}

// ------------------------------------------------------- state access --
template <typename S>
__global__ void k_get_state(Geom g, const uint8_t* __restrict__ mask, const float* __restrict__ dang,
                            const S* __restrict__ ang, int G, int r, float* __restrict__ out) {
    const int64_t n = (int64_t)g.H * g.W;
    const size_t plane = (size_t)g.H * g.Wh;
    const int grp = r / G, lane = r % G;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / g.W), x = (int)(i % g.W);
        const int c = (x + y) & 1;
        const size_t hs = (size_t)y * g.Wh + (x >> 1);
        out[i] = mask[i] == MASK_GAP
                     ? Store<S>::load1(ang + ((size_t)(grp * 2 + c) * plane + hs) * G + lane)
                     : dang[(size_t)c * plane + hs];
    }
}

template <typename S>
__global__ void k_set_state(Geom g, const uint8_t* __restrict__ mask, S* __restrict__ ang,
                            int G, int r, const float* __restrict__ in) {
    const int64_t n = (int64_t)g.H * g.W;
    const size_t plane = (size_t)g.H * g.Wh;
    const int grp = r / G, lane = r % G;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (mask[i] != MASK_GAP) continue;
        const int y = (int)(i / g.W), x = (int)(i % g.W);
        const int c = (x + y) & 1;
        const size_t hs = (size_t)y * g.Wh + (x >> 1);
        Store<S>::store1(ang + ((size_t)(grp * 2 + c) * plane + hs) * G + lane, in[i]);
    }
}

// E_b from scratch in FP64 (one warp per block): Eq. 1 over the owned bonds.
template <typename S>
__global__ void k_block_energy(Geom g, const int32_t* __restrict__ of_block,
                               const uint8_t* __restrict__ mask,
                               const float* __restrict__ dang, const S* __restrict__ ang, int G,
                               int r, double q, double J, double* __restrict__ E) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= g.nblk) return;
    const size_t plane = (size_t)g.H * g.Wh;
    const int grp = r / G, ln = r % G;
    auto angle = [&](int y, int x) -> double {
        const int c = (x + y) & 1;
        const size_t hs = (size_t)y * g.Wh + (x >> 1);
        return mask[(int64_t)y * g.W + x] == MASK_GAP
                   ? (double)Store<S>::load1(ang + ((size_t)(grp * 2 + c) * plane + hs) * G + ln)
                   : (double)dang[(size_t)c * plane + hs];
    };
    // A bond exists between present sites of the same slice.
    auto bond = [&](int y2, int x2, int sb) {
        return y2 < g.H && x2 < g.W && mask[(int64_t)y2 * g.W + x2] != MASK_ABSENT &&
               of_block[(y2 / g.lb) * g.nbx + x2 / g.lb] == sb;
    };
    const int by = warp / g.nbx, bx = warp % g.nbx;
    const int y0 = by * g.lb, x0 = bx * g.lb;
    const int y1 = min(g.H, y0 + g.lb), x1 = min(g.W, x0 + g.lb);
    const int bw = x1 - x0, nsite = (y1 - y0) * bw;
    const int sb = of_block[warp];
    double s = 0.0;
    for (int j = lane; j < nsite; j += 32) {
        const int y = y0 + j / bw, x = x0 + j % bw;
        if (mask[(int64_t)y * g.W + x] == MASK_ABSENT) continue;
        const double pi = angle(y, x);
        if (bond(y, x + 1, sb)) s += -J * cos(q * (pi - angle(y, x + 1)));
        if (bond(y + 1, x, sb)) s += -J * cos(q * (pi - angle(y + 1, x)));
    }
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) E[warp] = s;
}

// --------------------------------------------------------------- moments --
// The energy matching's derivative (fluctuation identity): after every
// measured calibration sweep (block energies folded), per block the sums of
// E_b, E_b^2 and E_b times the right / lower neighbour block's energy in the
// same chain. S is [4][nblk].
__global__ void k_cal_moments(int nblk, int nbx, int Rp, int chains,
                              const double* __restrict__ ecur, double* __restrict__ S) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        double s1 = 0.0, s2 = 0.0, sr = 0.0, sd = 0.0;
        const bool right = b % nbx != nbx - 1, down = b + nbx < nblk;
        for (int r = 0; r < chains; ++r) {
            const double E = ecur[(size_t)b * Rp + r];
            s1 += E;
            s2 += E * E;
            if (right) sr += E * ecur[(size_t)(b + 1) * Rp + r];
            if (down) sd += E * ecur[(size_t)(b + nbx) * Rp + r];
        }
        S[b] += s1;
        S[nblk + b] += s2;
        S[2 * nblk + b] += sr;
        S[3 * nblk + b] += sd;
    }
}

// Moments from the sums over n = measured sweeps x chains: M[0] = <E_b>/N_b,
// M[1] = Var(E_b), M[2] = Cov(E_b, E_right), M[3] = Cov(E_b, E_down).
__global__ void k_moments_final(int nblk, int nbx, double inv_n, const int32_t* __restrict__ Nb,
                                const double* __restrict__ S, double* __restrict__ M) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        const double m1 = S[b] * inv_n;
        M[b] = Nb[b] > 0 ? m1 / (double)Nb[b] : 0.0;
        M[nblk + b] = S[nblk + b] * inv_n - m1 * m1;
        M[2 * nblk + b] =
            (b % nbx != nbx - 1) ? S[2 * nblk + b] * inv_n - m1 * (S[b + 1] * inv_n) : 0.0;
        M[3 * nblk + b] = (b + nbx < nblk) ? S[3 * nblk + b] * inv_n - m1 * (S[b + nbx] * inv_n)
                                           : 0.0;
    }
}

// Damped Newton step of every targeted block on beta:
// beta_b + (y_b - e_s,b) N_b / Var(E_b) (T doubled when that beta is <= 0;
// without variance T doubled or halved towards e_s,b, as <e_b> grows with T),
// kept within a factor 2 of the old T and within [t_lo, t_hi].
__global__ void k_newton_update(int nblk, const double* __restrict__ es,
                                const int32_t* __restrict__ Nsp, const int32_t* __restrict__ Nb,
                                const double* __restrict__ M, float* __restrict__ T, double t_lo,
                                double t_hi) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        if (Nsp[b] <= 0) continue;
        const double y = M[b], v = M[nblk + b], tb = (double)T[b];
        double tn;
        if (v > 0.0) {
            const double bn = 1.0 / tb + (y - es[b]) * (double)Nb[b] / v;
            tn = bn > 0.0 ? 1.0 / bn : 2.0 * tb;
        } else {
            tn = y < es[b] ? 2.0 * tb : 0.5 * tb;
        }
        tn = fmin(fmax(tn, 0.5 * tb), 2.0 * tb);
        T[b] = (float)fmin(fmax(tn, t_lo), t_hi);
    }
}

__global__ void k_newton_init(int nblk, float t_init, float t_lo, float t_hi,
                              float* __restrict__ T, float* __restrict__ lo,
                              float* __restrict__ hi) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        T[b] = t_init;
        lo[b] = t_lo;
        hi[b] = t_hi;
    }
}

// Vector-Jacobian product of y = <E>/N with respect to beta from the stored
// moments: grad_beta_b = -sum_a g_a Cov(E_a, E_b) / N_a over a = b and its
// four neighbouring blocks.
__global__ void k_energy_vjp(int nblk, int nbx, const int32_t* __restrict__ Nb,
                             const double* __restrict__ M, const double* __restrict__ g,
                             double* __restrict__ out) {
    const double* var = M + nblk;
    const double* cr = M + 2 * nblk;
    const double* cd = M + 3 * nblk;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        auto w = [&](int a) { return Nb[a] > 0 ? g[a] / (double)Nb[a] : 0.0; };
        double acc = w(b) * var[b];
        if (b % nbx != nbx - 1) acc += w(b + 1) * cr[b];
        if (b % nbx != 0) acc += w(b - 1) * cr[b - 1];
        if (b + nbx < nblk) acc += w(b + nbx) * cd[b];
        if (b >= nbx) acc += w(b - nbx) * cd[b - nbx];
        out[b] = -acc;
    }
}

__global__ void k_set_tag(Control* ctl, uint32_t tag) { ctl->tag = tag; }

// ------------------------------------------------------------------- sst --
// Sec. 2.2.3: site temperatures start from the block temperatures and are
// replaced n_s times by the mean over the square of radius r around every
// site (coordinates clamped to the grid). The square mean is the row mean
// of the column means, so a pass is a row pass then a column pass; both sum
// their window directly in FP64.
__global__ void k_sst_expand(Geom g, const float* __restrict__ T_blk, double* __restrict__ Ts) {
    const int64_t n = (int64_t)g.H * g.W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / g.W), x = (int)(i % g.W);
        Ts[i] = (double)T_blk[(y / g.lb) * g.nbx + x / g.lb];
    }
}

__global__ void k_sst_box(Geom g, Slices sl, const double* __restrict__ in,
                          double* __restrict__ out, int r, int along_x) {
    const int64_t n = (int64_t)g.H * g.W;
    const double inv = 1.0 / (double)(2 * r + 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / g.W), x = (int)(i % g.W);
        const int sb = sl.of_block[(y / g.lb) * g.nbx + x / g.lb];
        if (sb < 0) continue;
        const int4 rc = sl.rect[sb];   // coordinates clamp to the site's own field
        if (y >= rc.x + rc.z || x >= rc.y + rc.w) continue;
        double s = 0.0;
        if (along_x) {
            const double* row = in + (int64_t)y * g.W;
            for (int d = -r; d <= r; ++d) s += row[min(max(x + d, rc.y), rc.y + rc.w - 1)];
        } else {
            for (int d = -r; d <= r; ++d)
                s += in[(int64_t)min(max(y + d, rc.x), rc.x + rc.z - 1) * g.W + x];
        }
        out[i] = s * inv;
    }
}

__global__ void k_site_beta(int64_t n, const float* __restrict__ Tf, float* __restrict__ beta) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        beta[i] = 1.0f / Tf[i];
}

__global__ void k_sst_beta(int64_t n, const double* __restrict__ Ts, float* __restrict__ Tf,
                           float* __restrict__ beta) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float t = (float)Ts[i];
        Tf[i] = t;
        beta[i] = 1.0f / t;
    }
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

void launch_minmax_field(const float* values, const uint8_t* mask, int64_t n, uint32_t* mm,
                         cudaStream_t s) {
    k_minmax_field<<<grid_for(n, 256), 256, 0, s>>>(values, mask, n, mm);
}

void launch_minmax(const Geom& g, const int32_t* of_block, const float* values,
                   const uint8_t* mask, uint32_t* mm, cudaStream_t s) {
    k_minmax<<<grid_for((int64_t)g.H * g.W, 256), 256, 0, s>>>(g, of_block, values, mask, mm);
}

void launch_layout(const Geom& g, const Slices& sl, const float* values, const uint8_t* mask,
                   float* dang, cudaStream_t s) {
    k_layout<<<grid_for((int64_t)g.H * g.W, 256), 256, 0, s>>>(g, sl, values, mask, dang);
}

void launch_block_stats(const Geom& g, const Slices& sl, const float* values, const uint8_t* mask,
                        double q, double J, double* Es, int32_t* Nsp, int32_t* Nb, double* ssum,
                        int32_t* nsamp, int32_t* ngap0, int32_t* ngap1, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (int)(((int64_t)g.nblk * 32 + threads - 1) / threads);
    k_block_stats<<<blocks, threads, 0, s>>>(g, sl, values, mask, q, J, Es, Nsp, Nb, ssum, nsamp,
                                             ngap0, ngap1);
}

void launch_scan(const int32_t* cnt, int n, int32_t* out, cudaStream_t s) {
    k_scan_counts<<<1, 1024, 0, s>>>(cnt, n, out);
}

void launch_build_lists(const Geom& g, const int32_t* of_block, const uint8_t* mask,
                        const int32_t* start0, const int32_t* start1, uint2* list0, uint2* list1,
                        int32_t* split0, int32_t* split1, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (int)(((int64_t)g.nblk * 32 + threads - 1) / threads);
    k_build_lists<<<blocks, threads, 0, s>>>(g, of_block, mask, start0, start1, list0, list1,
                                             split0, split1);
}

namespace {
// Launch with programmatic dependent launch allowed: the kernel may start
// while the previous kernel on the stream finishes (every kernel launched
// this way executes griddepcontrol.wait before reading what its predecessor
// writes). A refused attribute falls back to a plain launch.
template <typename... KArgs, typename... Args>
void launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k, args...) != cudaSuccess) {
        cudaGetLastError();
        k<<<grid, block, 0, s>>>(args...);
    }
}

template <typename S> struct Tag { using type = S; };
// Calls f(Tag<S>) with the state element type of `storage` (an mpr_storage).
template <typename F> void with_storage(int storage, F&& f) {
    if (storage == 1) f(Tag<__nv_bfloat16>{});
    else if (storage == 2) f(Tag<__half>{});
    else f(Tag<float>{});
}
}  // namespace

void launch_init(const Geom& g, const Slices& sl, const uint2* list, int64_t n_list, int colour,
                 const float* init_angle, void* ang, int storage, int G, int Rp, int random,
                 Rng rng, uint32_t r_even, cudaStream_t s) {
    if (n_list == 0) return;
    with_storage(storage, [&](auto tag) {
        using S = typename decltype(tag)::type;
        k_init<S><<<grid_for(n_list * Rp, 256), 256, 0, s>>>(g, sl, list, n_list, colour,
                                                            init_angle, static_cast<S*>(ang), G,
                                                            Rp, random, rng, r_even);
    });
}

void launch_fill_samples(const Geom& g, const uint8_t* mask, const float* dang, void* ang,
                         int storage, int G, int groups, cudaStream_t s) {
    if (storage != 0) return;        // the 16-bit forms read samples from dang
    k_fill_samples<<<grid_for((int64_t)g.H * g.W * groups, 256), 256, 0, s>>>(
        g, mask, dang, static_cast<float*>(ang), G, groups);
}

namespace {
// The three forms of the realizations' half-step by warps per unit (one
// realization pair of one block): form 0 one warp, form 1 two, form 2 four
// (splitting the block's entries between them), in 128-thread CTAs.
template <int G, typename S>
void sweep_dispatch(const SweepArgs& a, int form, int grid, cudaStream_t s) {
    if (form == 3) launch_pdl(k_sweep_half<G, S>, grid, 128, s, a);
    else if (form == 2) launch_pdl(k_sweep<G, S, 4>, grid, 128, s, a);
    else if (form == 1) launch_pdl(k_sweep<G, S, 2>, grid, 128, s, a);
    else launch_pdl(k_sweep<G, S, 1>, grid, 128, s, a);
}

template <int G, typename S>
int sweep_occupancy(int form) {
    int n = 0;
    if (form == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep_half<G, S>, 128, 0);
    else if (form == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<G, S, 4>, 128, 0);
    else if (form == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<G, S, 2>, 128, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<G, S, 1>, 128, 0);
    return n > 0 ? n : 1;
}
}  // namespace

void launch_sweep(const SweepArgs& a, int G, int storage, int form, int grid, cudaStream_t s) {
    with_storage(storage, [&](auto tag) {
        using S = typename decltype(tag)::type;
        if (G == 2) sweep_dispatch<2, S>(a, form, grid, s);
        else sweep_dispatch<8, S>(a, form, grid, s);
    });
}

int sweep_blocks_per_sm(int G, int storage, int form) {
    int n = 1;
    with_storage(storage, [&](auto tag) {
        using S = typename decltype(tag)::type;
        n = G == 2 ? sweep_occupancy<2, S>(form) : sweep_occupancy<8, S>(form);
    });
    return n;
}

int sweep_items_per_cta(int G, int form) {
    (void)G;
    return form == 3 ? 8 : 4 >> form;
}

void launch_energy(const SweepArgs& a, int G, int storage, int n_sm, cudaStream_t s) {
    with_storage(storage, [&](auto tag) {
        using S = typename decltype(tag)::type;
        // As many CTAs as fit on the GPU at once (the kernel loops over items).
        int per_sm = 0;
        if (G == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_energy<2, S>, 128, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_energy<8, S>, 128, 0);
        const int grid = n_sm * (per_sm > 0 ? per_sm : 8);
        if (G == 2) k_energy<2, S><<<grid, 128, 0, s>>>(a);
        else k_energy<8, S><<<grid, 128, 0, s>>>(a);
    });
}

void launch_sweep_flat(const SweepArgs& a, int G, int64_t n_list, cudaStream_t s,
                       const FoldArgs* fold) {
    FoldArgs f{};
    if (fold) f = *fold;
    if (n_list == 0 && f.ctas == 0) return;
    const int64_t threads = n_list * (G / 2);
    const dim3 grid((unsigned)((threads + kFlatThreads - 1) / kFlatThreads + f.ctas),
                    (unsigned)a.groups);
    // Programmatic dependent launch: this half-step's prologue overlaps the
    // previous launch's tail (the kernel waits before touching its output).
    if (G == 2) launch_pdl(k_sweep_flat<2>, grid, kFlatThreads, s, a, n_list, f);
    else launch_pdl(k_sweep_flat<8>, grid, kFlatThreads, s, a, n_list, f);
}

void launch_sweep_cal(const SweepArgs& a, int G, cudaStream_t s, const FoldArgs* fold) {
    FoldArgs f{};
    if (fold) f = *fold;
    const int64_t units = (int64_t)a.g.nblk * a.groups * (G / 2);
    const dim3 grid((unsigned)((units + 3) / 4 + f.ctas));
    if (G == 2) launch_pdl(k_sweep_cal<2>, grid, 128, s, a, f);
    else launch_pdl(k_sweep_cal<8>, grid, 128, s, a, f);
}

// Lanes G.. Rp-1 of every block take the E_b of lane r mod G (all lanes hold
// the same state).
__global__ void k_ecur_broadcast(int nblk, int Rp, int G, double* __restrict__ ecur) {
    const int64_t n = (int64_t)nblk * Rp;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t % Rp);
        if (r >= G) ecur[t] = ecur[t - r + r % G];
    }
}

void launch_ecur_broadcast(int nblk, int Rp, int G, double* ecur, cudaStream_t s) {
    k_ecur_broadcast<<<grid_for((int64_t)nblk * Rp, 256), 256, 0, s>>>(nblk, Rp, G, ecur);
}

void launch_ecur_reset(int nblk, int Rp, const double* Es, double* ecur, double* eacc,
                       cudaStream_t s) {
    k_ecur_reset<<<grid_for((int64_t)nblk * Rp, 256), 256, 0, s>>>(nblk, Rp, Es, ecur, eacc);
}

void launch_stop_init(int nblk, int Rp, const int32_t* of_block, const double* es,
                      const double* inb, const int32_t* Nsp, const int32_t* ngap, const double* ecur,
                      int8_t* sigma, uint8_t* running, int32_t* stop, int32_t* tcount,
                      double* e_last, cudaStream_t s) {
    k_stop_init<<<grid_for((int64_t)nblk * Rp, 256), 256, 0, s>>>(
        nblk, Rp, of_block, es, inb, Nsp, ngap, ecur, sigma, running, stop, tcount, e_last);
}

void launch_stop_targeted(int G, int groups, int Rp, const int32_t* of_block, int grid,
                          Control* ctl, const uint32_t* work, uint32_t work_stride,
                          const double* es, const double* inb, const int32_t* Nsp, double* eacc,
                          double* ecur, const int8_t* sigma, uint8_t* running, int32_t* stop,
                          int32_t* tcount, double* e_last, int t_known, cudaStream_t s,
                          const StopWindow* win) {
    StopArgs sa{};
    if (win) sa.win = *win;
    sa.G = G;
    sa.groups = groups;
    sa.Rp = Rp;
    sa.of_block = of_block;
    sa.es = es;
    sa.inb = inb;
    sa.Nsp = Nsp;
    sa.eacc = eacc;
    sa.ecur = ecur;
    sa.sigma = sigma;
    sa.running = running;
    sa.stop = stop;
    sa.tcount = tcount;
    sa.e_last = e_last;
    launch_pdl(k_stop_targeted, grid, 256, s, sa, ctl, work, work_stride, t_known);
}

void launch_stop_rest(int nblk, int groups, int G, int Rp, int n_max, const int32_t* of_block,
                      int grid, Control* ctl, const uint32_t* work, uint32_t* work_all,
                      uint32_t work_stride, const int32_t* Nsp, uint8_t* running, int32_t* stop,
                      const int32_t* tcount, cudaGraphConditionalHandle cond, int t_known,
                      cudaStream_t s) {
    StopArgs sa{};
    sa.G = G;
    sa.groups = groups;
    sa.Rp = Rp;
    sa.nblk = nblk;
    sa.n_max = n_max;
    sa.of_block = of_block;
    sa.Nsp = Nsp;
    sa.running = running;
    sa.stop = stop;
    sa.tcount = const_cast<int32_t*>(tcount);
    launch_pdl(k_stop_rest, grid, 256, s, sa, cond, ctl, work, work_all, work_stride, t_known);
}

void launch_count_updates(int nblk, int Rp, const int32_t* stop, const int32_t* ngap,
                          unsigned long long* total, cudaStream_t s, const Control* ctl) {
    k_count_updates<<<grid_for((int64_t)nblk * Rp, 256), 256, 0, s>>>(nblk, Rp, stop, ngap, ctl,
                                                                      total);
}

void launch_cal_init(int nblk, float t_lo, float t_hi, float* lo, float* hi, double* ebar,
                     Control* ctl, cudaStream_t s) {
    k_cal_init<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, t_lo, t_hi, lo, hi, ebar, ctl);
}

void launch_cal_mid(int nblk, const int32_t* Nsp, const float* lo, const float* hi, float* T,
                    Control* ctl, cudaStream_t s) {
    k_cal_mid<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, Nsp, lo, hi, T, ctl);
}

void launch_cal_fill(const Slices& sl, int nbx, const int32_t* Nsp, float* T, float* beta,
                     cudaStream_t s) {
    k_cal_fill<<<sl.n, 1024, 0, s>>>(sl, nbx, Nsp, T, beta);
}

void launch_cal_step(int nblk, int Rp, int chains, int n_eq, int t_fixed, const Control* ctl,
                     const double* inb, double* eacc, double* ecur, double* ebar, cudaStream_t s,
                     int points, double* ebar_odd, double* ebar_pts) {
    k_cal_step<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, Rp, chains, n_eq, t_fixed, ctl, inb, eacc,
                                                  ecur, ebar, points, ebar_odd, ebar_pts);
}

void launch_kpts_mid(int nblk, int points, const int32_t* Nsp, const float* lo, const float* hi,
                     float* Tk, Control* ctl, cudaStream_t s) {
    k_kpts_mid<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, points, Nsp, lo, hi, Tk, ctl);
}

void launch_kpts_update(int nblk, int points, double inv_count, const double* es,
                        const int32_t* Nsp, const float* Tk, float* lo, float* hi,
                        double* ebar_pts, Control* ctl, int n_iter,
                        cudaGraphConditionalHandle cond, cudaStream_t s) {
    k_kpts_update<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, points, inv_count, es, Nsp, Tk, lo,
                                                     hi, ebar_pts, ctl, n_iter, cond);
}

void launch_kcal_mid(int nblk, const int32_t* Nsp, const float* lo, const float* hi, float* T0,
                     float* T1, Control* ctl, cudaStream_t s) {
    k_kcal_mid<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, Nsp, lo, hi, T0, T1, ctl);
}

void launch_kcal_update(int nblk, double inv_count, const double* es, const int32_t* Nsp,
                        const float* T0, const float* T1, float* lo, float* hi, double* ebar0,
                        double* ebar1, Control* ctl, int n_iter, cudaGraphConditionalHandle cond,
                        cudaStream_t s) {
    k_kcal_update<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, inv_count, es, Nsp, T0, T1, lo, hi,
                                                     ebar0, ebar1, ctl, n_iter, cond);
}

void launch_cal_update(int nblk, double inv_count, const double* es, const int32_t* Nsp,
                       const float* T, float* lo, float* hi, double* ebar, Control* ctl,
                       int n_bisect, cudaGraphConditionalHandle cond, cudaStream_t s) {
    k_cal_update<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, inv_count, es, Nsp, T, lo, hi, ebar,
                                                    ctl, n_bisect, cond);
}

void launch_accumulate(const Geom& g, const uint2* list, int64_t n_list, int colour,
                       const void* ang, int storage, int G, int groups, int r_off, int R,
                       double* sum, cudaStream_t s) {
    if (n_list == 0) return;
    with_storage(storage, [&](auto tag) {
        using S = typename decltype(tag)::type;
        k_accumulate<S><<<grid_for(n_list, 256), 256, 0, s>>>(
            g, list, n_list, colour, static_cast<const S*>(ang), G, groups, r_off, R, sum);
    });
}

void launch_sum_to_grid(const Geom& g, const uint8_t* mask, const double* sum, double* out,
                        cudaStream_t s) {
    k_sum_to_grid<<<grid_for((int64_t)g.H * g.W, 256), 256, 0, s>>>(g, mask, sum, out);
}

void launch_grid_to_sum(const Geom& g, const uint8_t* mask, const double* in, double* sum,
                        cudaStream_t s) {
    k_grid_to_sum<<<grid_for((int64_t)g.H * g.W, 256), 256, 0, s>>>(g, mask, in, sum);
}

void launch_predict(const Geom& g, const Slices& sl, const float* values, const uint8_t* mask,
                    const double* sum, double inv_r, float* out, const float* truth, double* err,
                    cudaStream_t s) {
    k_predict<<<grid_for((int64_t)g.H * g.W, 256), 256, 0, s>>>(g, sl, values, mask, sum, inv_r,
                                                               out, truth, err);
}

void launch_get_state(const Geom& g, const uint8_t* mask, const float* dang, const void* ang,
                      int storage, int G, int r, float* out, cudaStream_t s) {
    with_storage(storage, [&](auto tag) {
        using S = typename decltype(tag)::type;
        k_get_state<S><<<grid_for((int64_t)g.H * g.W, 256), 256, 0, s>>>(
            g, mask, dang, static_cast<const S*>(ang), G, r, out);
    });
}

void launch_set_state(const Geom& g, const uint8_t* mask, void* ang, int storage, int G, int r,
                      const float* in, cudaStream_t s) {
    with_storage(storage, [&](auto tag) {
        using S = typename decltype(tag)::type;
        k_set_state<S><<<grid_for((int64_t)g.H * g.W, 256), 256, 0, s>>>(
            g, mask, static_cast<S*>(ang), G, r, in);
    });
}

void launch_block_energy(const Geom& g, const int32_t* of_block, const uint8_t* mask,
                         const float* dang, const void* ang, int storage, int G, int r, double q,
                         double J, double* E, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (int)(((int64_t)g.nblk * 32 + threads - 1) / threads);
    with_storage(storage, [&](auto tag) {
        using S = typename decltype(tag)::type;
        k_block_energy<S><<<blocks, threads, 0, s>>>(g, of_block, mask, dang,
                                                     static_cast<const S*>(ang), G, r, q, J, E);
    });
}

void launch_sst(const Geom& g, const Slices& sl, const float* T_blk, int r, int n_s, double* Ts,
                double* tmp, float* Tf, float* beta, cudaStream_t s) {
    const int64_t n = (int64_t)g.H * g.W;
    const int grid = grid_for(n, 256);
    k_sst_expand<<<grid, 256, 0, s>>>(g, T_blk, Ts);
    for (int k = 0; k < n_s; ++k) {
        k_sst_box<<<grid, 256, 0, s>>>(g, sl, Ts, tmp, r, 1);
        k_sst_box<<<grid, 256, 0, s>>>(g, sl, tmp, Ts, r, 0);
    }
    k_sst_beta<<<grid, 256, 0, s>>>(n, Ts, Tf, beta);
}

void launch_site_beta(int64_t n, const float* Tf, float* beta, cudaStream_t s) {
    k_site_beta<<<grid_for(n, 256), 256, 0, s>>>(n, Tf, beta);
}

void launch_cal_moments(int nblk, int nbx, int Rp, int chains, const double* ecur, double* S,
                        cudaStream_t s) {
    k_cal_moments<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, nbx, Rp, chains, ecur, S);
}

void launch_moments_final(int nblk, int nbx, double inv_n, const int32_t* Nb, const double* S,
                          double* M, cudaStream_t s) {
    k_moments_final<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, nbx, inv_n, Nb, S, M);
}

void launch_newton_update(int nblk, const double* es, const int32_t* Nsp, const int32_t* Nb,
                          const double* M, float* T, double t_lo, double t_hi, cudaStream_t s) {
    k_newton_update<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, es, Nsp, Nb, M, T, t_lo, t_hi);
}

void launch_newton_init(int nblk, float t_init, float t_lo, float t_hi, float* T, float* lo,
                        float* hi, cudaStream_t s) {
    k_newton_init<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, t_init, t_lo, t_hi, T, lo, hi);
}

void launch_energy_vjp(int nblk, int nbx, const int32_t* Nb, const double* M, const double* g,
                       double* out, cudaStream_t s) {
    k_energy_vjp<<<grid_for(nblk, 256), 256, 0, s>>>(nblk, nbx, Nb, M, g, out);
}

void launch_set_tag(Control* ctl, uint32_t tag, cudaStream_t s) { k_set_tag<<<1, 1, 0, s>>>(ctl, tag); }

}  // namespace mpr
