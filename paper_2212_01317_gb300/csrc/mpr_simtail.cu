// The stop tail of a realization batch as one cooperative launch.
//
// Late in a batch few (block, realization) pairs still run (Sec. 3.4 reading:
// each pair sweeps until its first crossing of e_s,b, or n_max), so a sweep
// is four launches of nearly empty grids whose cost is launch and drain
// latency. Here one launch runs the remaining sweeps: colour 0, colour 1, the
// targeted stops, the closing stop part, each over the whole grid with a
// grid barrier between them; the barrier closing a sweep advances the
// device Control (sweep index, running count, next worklist), exactly as the
// closing stop kernel does. Every step runs the same device code as the
// per-launch path (sweep_item, stop_targeted_range, stop_rest_range), so the
// results are those of the per-launch loop.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mpr_launch.h"
#include "mpr_sweep.cuh"

namespace mpr {

constexpr int kTailThreads = 512;

template <int G, typename S>
__global__ void __launch_bounds__(kTailThreads, 2) k_sim_tail(SimTailArgs a) {
    constexpr int NP = G / 2;
    constexpr int WPC = kTailThreads / 32;
    const int warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * WPC + warp, nw = gridDim.x * WPC;
    const int64_t tid = (int64_t)blockIdx.x * kTailThreads + threadIdx.x;
    const int64_t nthr = (int64_t)gridDim.x * kTailThreads;
    __shared__ uint32_t s_t, s_n, s_tag;
    __shared__ int s_go;
    unsigned int gen = 0;
    const unsigned long long lim = a.spin_limit;
    Control* ctl = a.ctl;
    for (;;) {
        // Every CTA reads the Control after the same barrier, so all take the
        // same decision.
        if (threadIdx.x == 0) {
            const uint32_t t = ld_acquire(&ctl->t);
            const unsigned long long run = ld_acquire(&ctl->n_running);
            s_t = t;
            s_n = ld_acquire(&ctl->n_work[t & 1u]);
            s_tag = ld_acquire(&ctl->tag);
            s_go = run > 0 && (int)t <= a.st.n_max;
        }
        __syncthreads();
        if (!s_go) return;
        const uint32_t t = s_t, n_items = s_n;
        const uint32_t ctr1 = t | (s_tag << 16);
        const uint32_t par = t & 1u, nxt = par ^ 1u;
        const uint32_t* work = a.work_all + (size_t)par * a.sw.work_stride;
        // The worklist holds units (one realization pair of one block): one
        // warp per unit while they fill the grid; two or four (splitting a
        // block's entries) when they are few.
        int k = 1;
        while (k < 4 && (int64_t)n_items * 2 * k <= nw) k *= 2;
        const int npairs = a.sw.groups * NP;
        const int ngrp = nw / k, gi = gw / k, cw = gw % k;
        for (int c = 0; c < 2; ++c) {
            SweepArgs s = a.sw;
            s.colour = c;
            s.list = a.list[c];
            s.start = a.start[c];
            s.split = a.split[c];
            if (gi < ngrp)
                for (uint32_t it = (uint32_t)gi; it < n_items; it += (uint32_t)ngrp) {
                    const int u = (int)work[it];
                    const int b = u / npairs, p = u - b * npairs;
                    const int grp = p / NP, q = p - grp * NP;
                    sweep_item<G, S>(s, b * s.groups + grp, q + NP * cw, NP * k, ctr1);
                }
            if (!grid_sync(a.bar, gen, lim)) return;
        }
        stop_targeted_range(a.st, t, work, (int64_t)n_items * a.st.G, (int64_t)n_items * a.st.G,
                            tid, nthr);
        if (!grid_sync(a.bar, gen, lim)) return;
        unsigned cnt = stop_rest_range(a.st, t, work, (int64_t)n_items, (int64_t)n_items,
                                       a.work_all + (size_t)nxt * a.sw.work_stride,
                                       &ctl->n_work[nxt], tid, nthr);
        for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
        if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&ctl->n_running_acc, (unsigned long long)cnt);
        const bool ok = grid_sync_then(a.bar, gen, lim, [&] {
            const unsigned long long left = atomicExch(&ctl->n_running_acc, 0ull);
            ctl->n_running = left;
            ctl->n_work[par] = 0;
            ctl->t = t + 1;
        });
        if (!ok) return;
    }
}

namespace {
template <typename S> struct TailTag { using type = S; };
template <typename F> void with_storage_tail(int storage, F&& f) {
    if (storage == 1) f(TailTag<__nv_bfloat16>{});
    else if (storage == 2) f(TailTag<__half>{});
    else f(TailTag<float>{});
}
}  // namespace

int sim_tail_blocks_per_sm(int G, int storage) {
    int n = 0;
    with_storage_tail(storage, [&](auto tag) {
        using S = typename decltype(tag)::type;
        if (G == 2)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sim_tail<2, S>, kTailThreads, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sim_tail<8, S>, kTailThreads, 0);
    });
    return n < 2 ? n : 2;
}

cudaError_t launch_sim_tail(const SimTailArgs& a, int G, int storage, int grid, cudaStream_t s) {
    void* args[] = {const_cast<SimTailArgs*>(&a)};
    cudaError_t e = cudaSuccess;
    with_storage_tail(storage, [&](auto tag) {
        using S = typename decltype(tag)::type;
        const void* k = G == 2 ? (const void*)k_sim_tail<2, S> : (const void*)k_sim_tail<8, S>;
        e = cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kTailThreads), args, 0, s);
    });
    return e;
}

}  // namespace mpr
