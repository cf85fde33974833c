// Block statistics (Sec. 2.1 transform range, Eq. 2 per block) of a field in
// device memory, computed without allocating any memory.
//
// Some callers cannot allocate device memory when they call us: a service
// that reserves all device memory at start-up and hands it to its own pool,
// code on a latency-critical path that must not pay for cudaFree's implicit
// device-wide synchronisation, or code that runs while the process is short
// of memory and must not fail for that reason. mpr_create allocates its
// context; this entry point instead works in a fixed scratch array that the
// library holds on every device that loads it, and writes only into buffers
// the caller passes.
#include <cuda_runtime.h>

#include <cstdint>

#include "mpr.h"
#include "mpr_internal.h"
#include "mpr_launch.h"
#include "mpr_ptrcheck.h"
#include "mpr_stats.cuh"

using namespace mpr;

namespace {

constexpr int kMaxBlocks = MPR_NOALLOC_MAX_BLOCKS;
constexpr size_t kHeader = 256;
constexpr size_t kScratchBytes = kHeader + (size_t)kMaxBlocks * (sizeof(double) + 3 * sizeof(int32_t));

// The scratch array: [0, 8) z-range in order-preserving uint32 form,
// [256, ...) per-block sample sums (double), sample counts and gap counts per
// colour (int32). Every call overwrites what it reads; nothing survives a call
// in a form the next one depends on.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Scratch {
    uint32_t* mm;
    double* ssum;
    int32_t* nsamp;
    int32_t* ng0;
    int32_t* ng1;
};

Scratch carve(unsigned char* base) {
    Scratch s;
    s.mm = reinterpret_cast<uint32_t*>(base);
    s.ssum = reinterpret_cast<double*>(base + kHeader);
    s.nsamp = reinterpret_cast<int32_t*>(base + kHeader + (size_t)kMaxBlocks * sizeof(double));
    s.ng0 = s.nsamp + kMaxBlocks;
    s.ng1 = s.ng0 + kMaxBlocks;
    return s;
}

// Device address of the scratch array on the current device (the host-side
// symbol is only a stand-in, not a device address). It is looked up on every
// call: the lookup allocates nothing, and an address kept from an earlier call
// would dangle after the device was reset (cudaDeviceReset) and its context
// re-created.
cudaError_t scratch_address(unsigned char** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned char*>(p);
    return cudaSuccess;
}

__device__ __forceinline__ float ord_to_float(uint32_t u) {
    const uint32_t v = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    return __uint_as_float(v);
}

// The min/max reduction accumulates into the scratch; start it from the
// identity of min and max.
__global__ void k_na_reset(uint32_t* mm) {
    mm[0] = 0xffffffffu;
    mm[1] = 0u;
}

// z_min / z_max as doubles (both 0 when there is no sample).
__global__ void k_na_range(const uint32_t* __restrict__ mm, double* __restrict__ zrange) {
    if (mm[0] == 0xffffffffu) {
        zrange[0] = 0.0;
        zrange[1] = 0.0;
    } else {
        zrange[0] = (double)ord_to_float(mm[0]);
        zrange[1] = (double)ord_to_float(mm[1]);
    }
}

// Eq. 2 per block with the range read from device memory: one warp per block,
// owned bonds (right and down), FP64 sums.
__global__ void k_na_block_stats(Geom g, const float* __restrict__ values,
                                 const uint8_t* __restrict__ mask, const double* __restrict__ zrange,
                                 double q, double J, double* __restrict__ Es,
                                 int32_t* __restrict__ Nsp, int32_t* __restrict__ Nb, Scratch sc) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= g.nblk) return;
    const double zmin = zrange[0], zmax = zrange[1];
    const bool degenerate = !(zmax > zmin);
    const int by = warp / g.nbx, bx = warp % g.nbx;
    const int y0 = by * g.lb, x0 = bx * g.lb;
    const int y1 = min(g.H, y0 + g.lb), x1 = min(g.W, x0 + g.lb);
    const double scale = degenerate ? 0.0 : 6.283185307179586476925 / (zmax - zmin);
    // (no absent sites: a bond crosses the block's right / lower edge unless
    // that edge is the grid's)
    const BlockSums r = block_sums<false>(values, mask, g.W, y0, x0, y1, x1, x1 < g.W, y1 < g.H,
                                          zmin, scale, q, J, true);
    if (lane == 0) {
        Es[warp] = r.es;
        Nsp[warp] = r.nsp;
        Nb[warp] = r.nb;
        sc.ssum[warp] = r.sm;
        sc.nsamp[warp] = r.ns;
        sc.ng0[warp] = r.g0;
        sc.ng1[warp] = r.g1;
    }
}

// One CTA: global sample mean (fallback of blocks without samples, Sec. 3.3.3),
// then each block's mean sample angle and gap count.
__global__ void k_na_finalize(int nblk, Scratch sc, float* __restrict__ mean_angle,
                              int32_t* __restrict__ n_gap) {
    __shared__ double s_sum[256];
    __shared__ long long s_cnt[256];
    double sum = 0.0;
    long long cnt = 0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        sum += sc.ssum[b];
        cnt += sc.nsamp[b];
    }
    s_sum[threadIdx.x] = sum;
    s_cnt[threadIdx.x] = cnt;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s_sum[threadIdx.x] += s_sum[threadIdx.x + w];
            s_cnt[threadIdx.x] += s_cnt[threadIdx.x + w];
        }
        __syncthreads();
    }
    const double gmean = s_cnt[0] > 0 ? s_sum[0] / (double)s_cnt[0] : 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        const int ns = sc.nsamp[b];
        mean_angle[b] = (float)(ns > 0 ? sc.ssum[b] / (double)ns : gmean);
        n_gap[b] = sc.ng0[b] + sc.ng1[b];
    }
}

// The pointer is device memory of `device` (the current one) or managed memory.
bool on_device(const void* p, int device) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return noalloc_pointer_ok(at.type, at.device, device);
}

}  // namespace

extern "C" mpr_status mpr_block_stats_noalloc(const mpr_grid* grid, const uint8_t* mask,
                                              const float* values, double q, double J,
                                              double* Es, int32_t* Nsp, int32_t* Nb,
                                              float* mean_angle, int32_t* n_gap, double* zrange,
                                              void* cuda_stream) {
    if (!grid || !mask || !values || !Es || !Nsp || !Nb || !mean_angle || !n_gap || !zrange)
        return MPR_EINVAL;
    const int H = grid->height, W = grid->width, lb = grid->block;
    if (H < 1 || W < 1 || H > MAX_SIDE || W > MAX_SIDE || lb < 1) return MPR_EINVAL;
    if (!(q > 0.0 && q <= 0.5) || !(J > 0.0)) return MPR_EINVAL;
    Geom g;
    g.H = H;
    g.W = W;
    g.Wh = (W + 1) / 2;
    g.lb = lb;
    g.nbx = (W + lb - 1) / lb;
    g.nby = (H + lb - 1) / lb;
    if ((int64_t)g.nbx * g.nby > kMaxBlocks) return MPR_EINVAL;  // beyond the scratch array
    g.nblk = g.nbx * g.nby;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return MPR_ECUDA;
    }
    const void* ptrs[] = {mask, values, Es, Nsp, Nb, mean_angle, n_gap, zrange};
    for (const void* p : ptrs)
        if (!on_device(p, device)) return MPR_EINVAL;
    unsigned char* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return MPR_ECUDA;
    const Scratch sc = carve(base);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int64_t n = (int64_t)H * W;
    k_na_reset<<<1, 1, 0, s>>>(sc.mm);
    launch_minmax_field(values, mask, n, sc.mm, s);
    k_na_range<<<1, 1, 0, s>>>(sc.mm, zrange);
    const int threads = 256;
    const int blocks = (int)(((int64_t)g.nblk * 32 + threads - 1) / threads);
    k_na_block_stats<<<blocks, threads, 0, s>>>(g, values, mask, zrange, q, J, Es, Nsp, Nb, sc);
    k_na_finalize<<<1, 256, 0, s>>>(g.nblk, sc, mean_angle, n_gap);
    return cudaPeekAtLastError() == cudaSuccess ? MPR_OK : MPR_ECUDA;
}
