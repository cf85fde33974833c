// The unconditional specific-energy curve e(T) and the calibration steps that
// read it (Sec. 2.1: plain MPR takes T from matching e_s against the energy of
// the simulated grid; on a lattice with no data that energy depends on T
// alone).
//
// The curve is measured the way the calibration measures a block: a data-free
// kCurveSide x kCurveSide lattice (open boundaries) with every angle started
// at pi, n_eq sweeps, then E / N_bonds averaged over n_meas sweeps. One CTA
// per temperature keeps its whole lattice in shared memory and runs every
// sweep in one launch (the lattice is 16 KB; a half-step is one pass of the
// CTA's threads over its colour, then a CTA barrier). Temperature k is
// realization k of the random-stream tag 0xFFFE under the key the caller
// gives (the library uses (0, 0): the curve is a function of the model's
// parameters alone).
//
// Its uses: the first calibration iteration's points around T0_b, where the
// curve reaches e_s,b (warm start), or T_b = T0_b itself (calibration method
// "curve", no conditional simulation).
#include <cuda_runtime.h>

#include <cstdint>

#include "mpr_curve.h"
#include "mpr_device.cuh"
#include "mpr_sweep.cuh"

namespace mpr {

namespace {

constexpr int kCurveThreads = 1024;
constexpr int kCurveSites = kCurveSide * kCurveSide;
constexpr uint32_t kCurveTag = 0xFFFEu;

__device__ __forceinline__ void cs(float q, float phi, float& c, float& s) { __sincosf(q * phi, &s, &c); }

__global__ void __launch_bounds__(kCurveThreads, 1)
k_energy_curve(const float* __restrict__ T, int n_eq, int n_meas, Model m, uint32_t key0,
               uint32_t key1, double* __restrict__ e_out) {
    __shared__ float phi[kCurveSites];
    __shared__ double red[kCurveThreads / 32];
    const int k = blockIdx.x;
    const float beta = 1.0f / T[k];
    uint32_t rk0[10];
#pragma unroll
    for (int r = 0; r < 10; ++r) rk0[r] = key0 + (uint32_t)r * 0x9E3779B9u;
    for (int i = threadIdx.x; i < kCurveSites; i += blockDim.x) phi[i] = 0.5f * kTwoPi;
    __syncthreads();
    constexpr int half = kCurveSide / 2;   // sites of one colour in a row
    const double n_bonds = 2.0 * kCurveSide * (kCurveSide - 1);
    double acc = 0.0;
    for (int s = 1; s <= n_eq + n_meas; ++s) {
        const uint32_t ctr1 = (uint32_t)s | (kCurveTag << 16);
        for (int c = 0; c < 2; ++c) {
            for (int j = threadIdx.x; j < kCurveSites / 2; j += blockDim.x) {
                const int y = j / half;
                const int x = 2 * (j % half) + ((y + c) & 1);
                const int i = y * kCurveSide + x;
                float C = 0.0f, S = 0.0f, cj, sj;
                if (x > 0) { cs(m.q, phi[i - 1], cj, sj); C += cj; S += sj; }
                if (x + 1 < kCurveSide) { cs(m.q, phi[i + 1], cj, sj); C += cj; S += sj; }
                if (y > 0) { cs(m.q, phi[i - kCurveSide], cj, sj); C += cj; S += sj; }
                if (y + 1 < kCurveSide) { cs(m.q, phi[i + kCurveSide], cj, sj); C += cj; S += sj; }
                uint32_t w[4];
                philox4x32_10_rk((uint32_t)i, ctr1, (uint32_t)k >> 1, 0u, rk0, key1, w);
                const int o = 2 * (k & 1);
                const SiteNew n = site_update<float>(phi[i], C, S, u01(w[o]), u01(w[o + 1]), beta, m);
                phi[i] = n.phi;
            }
            __syncthreads();
        }
        if (s <= n_eq) continue;
        // E / N_bonds of this sweep: each site's right and down bonds.
        float part = 0.0f;
        for (int i = threadIdx.x; i < kCurveSites; i += blockDim.x) {
            const int y = i / kCurveSide, x = i % kCurveSide;
            if (x + 1 < kCurveSide) part -= m.J * __cosf(m.q * (phi[i] - phi[i + 1]));
            if (y + 1 < kCurveSide) part -= m.J * __cosf(m.q * (phi[i] - phi[i + kCurveSide]));
        }
        double d = (double)part;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            acc += t / n_bonds;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) e_out[k] = n_meas > 0 ? acc / (double)n_meas : 0.0;
}

// T where the non-decreasing envelope of the curve reaches e_s (linear
// interpolation between the points around it, clamped to the end points).
// Explicitly rounded FP64 operations: no contraction into FMAs, so every
// host and device that evaluates it gets the same number.
__device__ double curve_T0(int n, const float* __restrict__ T, const double* __restrict__ e,
                           double es) {
    double prev = e[0];
    if (!(es > prev)) return (double)T[0];
    for (int k = 1; k < n; ++k) {
        const double ek = e[k] > prev ? e[k] : prev;
        if (es <= ek) {
            const double f = __ddiv_rn(__dsub_rn(es, prev), __dsub_rn(ek, prev));
            const double t0 = (double)T[k - 1], t1 = (double)T[k];
            return __dadd_rn(t0, __dmul_rn(__dsub_rn(t1, t0), f));
        }
        prev = ek;
    }
    return (double)T[n - 1];
}

// First calibration iteration of the warm start: the points of every targeted
// block evenly spaced on [T0 / w, T0 w] (two points: T0a, T0b; more: Tk[p]);
// untargeted blocks 0 (the median fills them in). Starts iteration ctl->k as
// the midpoint kernels do.
__global__ void k_warm_points(int nblk, int points, const int32_t* __restrict__ Nsp,
                              const double* __restrict__ es, const float* __restrict__ cT,
                              const double* __restrict__ ce, int cn, double w,
                              float* __restrict__ T0a, float* __restrict__ T0b,
                              float* __restrict__ Tk, Control* ctl) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        const bool t = Nsp[b] > 0;
        const double t0 = t ? curve_T0(cn, cT, ce, es[b]) : 0.0;
        const double a = __ddiv_rn(t0, w), c = __dmul_rn(t0, w);
        const double step = __ddiv_rn(__dsub_rn(c, a), (double)(points - 1));
        if (points == 2) {
            T0a[b] = t ? (float)a : 0.0f;
            T0b[b] = t ? (float)c : 0.0f;
        } else {
            for (int p = 0; p < points; ++p)
                Tk[(size_t)p * nblk + b] = t ? (float)__dadd_rn(a, __dmul_rn((double)p, step)) : 0.0f;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->tag = 1u + ctl->k;
        ctl->t = 0;
    }
}

// Calibration method "curve": T_b = T0_b for targeted blocks, 0 for the rest.
__global__ void k_curve_T(int nblk, const int32_t* __restrict__ Nsp, const double* __restrict__ es,
                          const float* __restrict__ cT, const double* __restrict__ ce, int cn,
                          float* __restrict__ T) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x)
        T[b] = Nsp[b] > 0 ? (float)curve_T0(cn, cT, ce, es[b]) : 0.0f;
}

int grid_of(int n) { return (n + 255) / 256 > 0 ? (n + 255) / 256 : 1; }

}  // namespace

void launch_energy_curve(const float* T, int n_T, int n_eq, int n_meas, const Model& m,
                         uint64_t seed, double* e_out, cudaStream_t s) {
    k_energy_curve<<<n_T, kCurveThreads, 0, s>>>(T, n_eq, n_meas, m, (uint32_t)(seed & 0xffffffffu),
                                                 (uint32_t)(seed >> 32), e_out);
}

void launch_warm_points(int nblk, int points, const int32_t* Nsp, const double* es,
                        const float* cT, const double* ce, int cn, double w, float* T0a,
                        float* T0b, float* Tk, Control* ctl, cudaStream_t s) {
    k_warm_points<<<grid_of(nblk), 256, 0, s>>>(nblk, points, Nsp, es, cT, ce, cn, w, T0a, T0b, Tk,
                                                ctl);
}

void launch_curve_T(int nblk, const int32_t* Nsp, const double* es, const float* cT,
                    const double* ce, int cn, float* T, cudaStream_t s) {
    k_curve_T<<<grid_of(nblk), 256, 0, s>>>(nblk, Nsp, es, cT, ce, cn, T);
}

}  // namespace mpr
