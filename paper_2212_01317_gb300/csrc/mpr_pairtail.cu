// The stop tail of a realization batch with one CTA per realization pair.
//
// Realizations are independent chains (Sec. 3.4 reading: each (block,
// realization) pair sweeps until its first crossing of e_s,b, or n_max; the
// blocks without sample bonds of a realization stop once none of its
// targeted blocks runs), so the sweeps of one realization pair need no
// other pair's results. Late in a batch only a few of each pair's blocks
// still run; there, one CTA per pair runs the pair's remaining sweeps with
// CTA barriers between the phases (colour 0, colour 1, the targeted stops,
// the closing stop part) instead of a launch per phase. Its running units
// stay in shared memory. Every phase runs the same device code as the
// per-launch loop (sweep_item, stop_targeted_range, stop_rest_range) on the
// same data, so the results are those of the per-launch loop up to the
// order of the FP32 energy atomics.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mpr_launch.h"
#include "mpr_sweep.cuh"

namespace mpr {

namespace {

constexpr int kPairThreads = 1024;
constexpr int kPairWarps = kPairThreads / 32;

template <int G, typename S>
__global__ void __launch_bounds__(kPairThreads, 1) k_pair_tail(SimTailArgs a) {
    constexpr int NP = G / 2;
    __shared__ uint32_t s_units[2][kPairTailCap];
    __shared__ uint32_t s_n[2];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int npairs = a.sw.groups * NP;
    const int p = blockIdx.x;                         // this CTA's realization pair
    const int grp = p / NP, q = p - grp * NP;
    Control* ctl = a.ctl;
    const uint32_t t0 = ctl->t, tag = ctl->tag;
    const uint32_t n0 = ctl->n_work[t0 & 1u];
    const uint32_t* work = a.work_all + (size_t)(t0 & 1u) * a.sw.work_stride;
    if (tid == 0) {
        s_n[0] = 0;
        s_n[1] = 0;
    }
    __syncthreads();
    // This pair's units of the global worklist (the launch is only made when
    // the whole list fits one CTA's buffer).
    for (uint32_t i = tid; i < n0; i += kPairThreads) {
        const uint32_t u = work[i];
        if ((int)(u % (uint32_t)npairs) == p) {
            const uint32_t j = atomicAdd(&s_n[0], 1u);
            if (j < (uint32_t)kPairTailCap) s_units[0][j] = u;
        }
    }
    __syncthreads();
    if (tid == 0 && s_n[0] > (uint32_t)kPairTailCap) s_n[0] = kPairTailCap;   // never (host check)
    __syncthreads();
    int cur = 0;
    uint32_t t = t0;
    for (;;) {
        const uint32_t n = s_n[cur];
        if (n == 0 || (int)t > a.st.n_max) break;
        const uint32_t ctr1 = t | (tag << 16);
        // One warp per unit while they outnumber the warps; two or four
        // (splitting a block's entries) when they are few.
        int k = 1;
        while (k < 4 && (int)n * 2 * k <= kPairWarps) k *= 2;
        const int slot = warp / k, cw = warp - slot * k, nslot = kPairWarps / k;
        for (int c = 0; c < 2; ++c) {
            SweepArgs s = a.sw;
            s.colour = c;
            s.list = a.list[c];
            s.start = a.start[c];
            s.split = a.split[c];
            for (uint32_t it = slot; it < n; it += nslot) {
                const int b = (int)(s_units[cur][it] / (uint32_t)npairs);
                sweep_item<G, S>(s, b * s.groups + grp, q + NP * cw, NP * k, ctr1);
            }
            __syncthreads();
        }
        stop_targeted_range(a.st, t, s_units[cur], (int64_t)n * 2, (int64_t)n * 2, tid,
                            kPairThreads);
        if (tid == 0) s_n[cur ^ 1] = 0;
        __syncthreads();
        stop_rest_range(a.st, t, s_units[cur], n, n, s_units[cur ^ 1], &s_n[cur ^ 1], tid,
                        kPairThreads);
        __syncthreads();
        cur ^= 1;
        ++t;
    }
    // The last CTA to finish leaves the Control as the per-launch loop's
    // last closing stop kernel would: the sweep index after the last sweep
    // any pair ran, nothing running, empty worklists.
    if (tid == 0) {
        atomicMax(&ctl->t_tail, t);
        __threadfence();
        if (atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1) {
            __threadfence();
            const uint32_t tm = atomicExch(&ctl->t_tail, 0u);
            ctl->t = tm > t0 ? tm : t0;
            ctl->n_running = 0;
            ctl->n_running_acc = 0;
            ctl->n_work[0] = 0;
            ctl->n_work[1] = 0;
            ctl->ticket = 0;
            __threadfence();
        }
    }
}

template <typename S> struct PairTag { using type = S; };
template <typename F> void with_storage_pair(int storage, F&& f) {
    if (storage == 1) f(PairTag<__nv_bfloat16>{});
    else if (storage == 2) f(PairTag<__half>{});
    else f(PairTag<float>{});
}

}  // namespace

cudaError_t launch_pair_tail(const SimTailArgs& a, int G, int storage, int n_pairs,
                             cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    with_storage_pair(storage, [&](auto tag) {
        using S = typename decltype(tag)::type;
        if (G == 2) k_pair_tail<2, S><<<n_pairs, kPairThreads, 0, s>>>(a);
        else k_pair_tail<8, S><<<n_pairs, kPairThreads, 0, s>>>(a);
        e = cudaGetLastError();
    });
    return e;
}

}  // namespace mpr
