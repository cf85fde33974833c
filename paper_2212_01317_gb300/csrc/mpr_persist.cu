// Persistent calibration: all bisection iterations of the per-block energy
// matching (Sec. 2.1, applied per block in Sec. 2.2.2) in one cooperative
// launch. The calibration runs one or a few chains over the whole field, so
// each half-step is small; launching it as a kernel per half-step pays a
// launch and a wave of latency 2 x (n_eq + n_meas) x n_bisect times. Here the
// phases are separated by a grid-wide barrier instead.
//
// The phases are separated by grid_sync (mpr_sweep.cuh), which never waits
// forever: the host then reports MPR_ETIMEOUT.
#include <cuda_runtime.h>

#include <cstdint>

#include "mpr_launch.h"
#include "mpr_sweep.cuh"

namespace mpr {

namespace {

__device__ __forceinline__ SweepArgs colour_args(const CalPersistArgs& a, int c) {
    SweepArgs s = a.sw;
    s.colour = c;
    s.list = a.list[c];
    s.start = a.start[c];
    s.split = a.split[c];
    return s;
}

// Adds the change of sweep `sweep` to E_b of every chain; past n_eq sweeps,
// adds e_b of every chain to the running sum of the iteration.
__device__ __forceinline__ void fold_sweep(const CalPersistArgs& a, int sweep, int tid, int nthr) {
    const int Rp = a.sw.Rp;
    double* ea = a.eacc2[sweep & 1];
    for (int b = tid; b < a.sw.g.nblk; b += nthr) {
        double s = 0.0;
        for (int r = 0; r < a.chains; ++r) {
            const size_t k = (size_t)b * Rp + r;
            const double E = a.sw.ecur[k] + ea[k];
            a.sw.ecur[k] = E;
            ea[k] = 0.0;
            s += E * a.inb[b];
        }
        if (sweep > a.n_eq) a.ebar[b] += s;
    }
}

}  // namespace

// One CTA of 512 threads (16 warps) per SM. Items are taken by groups of four
// warps (energy pass; sweeps with G = 8) or by single warps (sweeps with G = 2).
template <int G>
__global__ void __launch_bounds__(512, 1) k_cal_persistent(CalPersistArgs a) {
    unsigned int gen = 0;
    const unsigned long long lim = a.spin_limit;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthr = gridDim.x * blockDim.x;
    const int nblk = a.sw.g.nblk;
    const int Rp = a.sw.Rp;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;                       // warps per CTA
    const int gwarp = blockIdx.x * wpb + warp, nwarps = gridDim.x * wpb;
    const int quad = warp >> 2, nquad = wpb >> 2;          // four-warp groups
    const int gquad = blockIdx.x * nquad + quad, nquads = gridDim.x * nquad;
    const int n_items = nblk * a.sw.groups;
    const int n_sweeps = a.n_eq + a.n_meas;
    const size_t plane = (size_t)a.sw.g.H * a.sw.g.Wh;
    for (int k = 0; k <= a.n_bisect; ++k) {
        // Midpoints of the brackets; blocks without sample bonds take the
        // median of the targeted blocks' midpoints. k == n_bisect: final T.
        for (int b = tid; b < nblk; b += nthr)
            a.T[b] = a.Nsp[b] > 0 ? 0.5f * (a.lo[b] + a.hi[b]) : 0.0f;
        if (!grid_sync(a.bar, gen, lim)) return;
        if (blockIdx.x == 0) {
            const float med =
                median_targeted(a.T, a.Nsp, make_int4(0, 0, a.sw.g.nby, a.sw.g.nbx), a.sw.g.nbx);
            if (threadIdx.x == 0) *a.med = med;
        }
        if (!grid_sync(a.bar, gen, lim)) return;
        const float med = *(volatile float*)a.med;
        for (int b = tid; b < nblk; b += nthr) {
            float tb = a.T[b];
            if (a.Nsp[b] <= 0) {
                tb = med;
                a.T[b] = med;
            }
            a.beta[b] = tb > 0.0f ? 1.0f / tb : 0.0f;
        }
        if (k == a.n_bisect) break;
        // Fresh start of every chain (Sec. 3.3.3), E_b <- E_s,b, no pending change.
        for (int c = 0; c < 2; ++c) {
            const int64_t total = a.n_list[c] * Rp;
            for (int64_t t = tid; t < total; t += nthr) {
                const int64_t e = t / Rp;
                const int r = (int)(t % Rp);
                const uint2 en = a.list[c][e];
                const int y = en.x >> 16, x = en.x & 0xffff;
                float v = a.init_angle[en.y >> META_SHIFT];
                if (a.random_init) {
                    const int sl = a.sw.sl.of_block[en.y >> META_SHIFT];
                    uint32_t w[4];
                    philox4x32_10(local_index(a.sw.sl.rect[sl], y, x), 0xFFFFu << 16,
                                  (uint32_t)r >> 1, 0u, a.sw.rng.key0, a.sw.sl.key1[sl], w);
                    v = kTwoPi * u01(w[(r & 1) * 2]);
                }
                const int grp = r / G, lane = r % G;
                static_cast<float*>(a.sw.ang)[((size_t)(grp * 2 + c) * plane +
                                               (size_t)y * a.sw.g.Wh + (x >> 1)) * G + lane] = v;
            }
        }
        for (int64_t t = tid; t < (int64_t)nblk * Rp; t += nthr) {
            a.sw.ecur[t] = a.Es[t / Rp];
            a.eacc2[0][t] = 0.0;
            a.eacc2[1][t] = 0.0;
        }
        if (!grid_sync(a.bar, gen, lim)) return;
        // E_b of the start state from scratch.
        for (int c = 0; c < 2; ++c) {
            const SweepArgs s = colour_args(a, c);
            for (int it = gquad; it < n_items; it += nquads) energy_item<G, float>(s, it, warp & 3, 4);
        }
        if (!grid_sync(a.bar, gen, lim)) return;
        // n_eq + n_meas sweeps; the change of sweep t is folded into E_b while
        // sweep t + 1 runs (the two sweeps use different buffers).
        for (int sweep = 1; sweep <= n_sweeps; ++sweep) {
            const uint32_t ctr1 = (uint32_t)sweep | ((uint32_t)(1 + k) << 16);
            for (int c = 0; c < 2; ++c) {
                SweepArgs s = colour_args(a, c);
                s.eacc = a.eacc2[sweep & 1];
                if constexpr (G == 2) {
                    for (int it = gwarp; it < n_items; it += nwarps)
                        sweep_item<G, float>(s, it, 0, 1, ctr1);
                } else {
                    for (int it = gquad; it < n_items; it += nquads)
                        sweep_item<G, float>(s, it, warp & 3, 4, ctr1);
                }
                if (c == 0 && sweep > 1) fold_sweep(a, sweep - 1, tid, nthr);
                if (!grid_sync(a.bar, gen, lim)) return;
            }
        }
        // Last sweep's change, then the bisection step: <e_b> increases with
        // T, so keep the half of the bracket that contains e_s,b.
        fold_sweep(a, n_sweeps, tid, nthr);
        for (int b = tid; b < nblk; b += nthr) {
            const double e = a.ebar[b] * a.inv_count;
            a.ebar[b] = 0.0;
            if (a.Nsp[b] <= 0) continue;
            if (e < a.es[b]) a.lo[b] = a.T[b]; else a.hi[b] = a.T[b];
        }
        if (!grid_sync(a.bar, gen, lim)) return;
    }
}

template __global__ void k_cal_persistent<2>(CalPersistArgs);
template __global__ void k_cal_persistent<8>(CalPersistArgs);

int cal_persistent_blocks_per_sm(int G) {
    int n = 0;
    if (G == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cal_persistent<2>, 512, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cal_persistent<8>, 512, 0);
    return n > 1 ? 1 : n;   // one CTA per SM: fewer arrivals per barrier
}

cudaError_t launch_cal_persistent(const CalPersistArgs& a, int G, int grid, cudaStream_t s) {
    void* args[] = {const_cast<CalPersistArgs*>(&a)};
    if (G == 2)
        return cudaLaunchCooperativeKernel((const void*)k_cal_persistent<2>, dim3(grid), dim3(512),
                                           args, 0, s);
    return cudaLaunchCooperativeKernel((const void*)k_cal_persistent<8>, dim3(grid), dim3(512), args,
                                       0, s);
}

}  // namespace mpr
