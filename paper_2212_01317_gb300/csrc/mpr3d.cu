// 3-D grids (D x H x W, 6-neighbour MPR Hamiltonian, cubic blocks): the
// space / space-time extension the paper names in its conclusions (Sec. 4).
// Everything but the geometry is the 2-D method: Sec. 2.1 transform, Eq. 2
// per block, per-block temperatures by bisection, checkerboard Metropolis +
// over-relaxation half-steps, incremental block energies, the per-block
// local-equilibrium stop (Sec. 3.4), realizations averaged and
// back-transformed.
//
// Layout: site (z, y, x), index i = (z H + y) W + x, colour (x + y + z) mod 2,
// half-lattice state [colour][D][H][ceil(W/2)][pairs] of float2 (a
// realization pair per element; sample angles in every lane); gap lists per
// colour, block-major, of (site index, block). A thread updates one gap
// site for one realization pair. Every site owns its +x, +y, +z bonds; a
// site on the low x / y / z face of its block hands that bond's change to
// the neighbouring block. The stop and calibration bookkeeping (per block
// and realization) are the 2-D kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "mpr.h"
#include "mpr_internal.h"
#include "mpr_launch.h"
#include "mpr_memory.h"
#include "mpr_sweep.cuh"

using namespace mpr;

namespace {

struct Geom3 {
    int D, H, W, Wh, lb, nbx, nby, nbz, nblk;
};

__device__ __forceinline__ int block3(const Geom3& g, int z, int y, int x) {
    return ((z / g.lb) * g.nby + y / g.lb) * g.nbx + x / g.lb;
}

// Element (pair p) of site (z, y, x) in the half-lattice of its colour.
__device__ __forceinline__ size_t hidx3(const Geom3& g, int c, int z, int y, int x, int np) {
    return ((((size_t)c * g.D + z) * g.H + y) * g.Wh + (x >> 1)) * np;
}

__device__ __forceinline__ uint32_t f2ord3(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void k3_minmax(const float* __restrict__ values, const uint8_t* __restrict__ mask,
                          int64_t n, uint32_t* __restrict__ mm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (mask[i]) continue;
        const uint32_t o = f2ord3(values[i]);
        atomicMin(&mm[0], o);
        atomicMax(&mm[1], o);
    }
}

// Sample angles (Sec. 2.1) in FP32, 0 at gaps.
__global__ void k3_layout(int64_t n, const float* __restrict__ values,
                          const uint8_t* __restrict__ mask, double zmin, double zmax,
                          int degenerate, float* __restrict__ phi_s) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        phi_s[i] = (mask[i] || degenerate)
                       ? 0.0f
                       : (float)(6.283185307179586476925 * ((double)values[i] - zmin) / (zmax - zmin));
}

// Eq. 2 per block (one warp per block, FP64): owned sample-sample bonds, all
// owned bonds, sample mean angle, gap counts per colour.
__global__ void k3_block_stats(Geom3 g, const float* __restrict__ values,
                               const uint8_t* __restrict__ mask, double zmin, double zmax,
                               int degenerate, double q, double J, double* __restrict__ Es,
                               int32_t* __restrict__ Nsp, int32_t* __restrict__ Nb,
                               double* __restrict__ ssum, int32_t* __restrict__ nsamp,
                               int32_t* __restrict__ ngap0, int32_t* __restrict__ ngap1) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= g.nblk) return;
    const int bx = warp % g.nbx, by = (warp / g.nbx) % g.nby, bz = warp / (g.nbx * g.nby);
    const int x0 = bx * g.lb, y0 = by * g.lb, z0 = bz * g.lb;
    const int x1 = min(g.W, x0 + g.lb), y1 = min(g.H, y0 + g.lb), z1 = min(g.D, z0 + g.lb);
    const int bw = x1 - x0, bh = y1 - y0, nsite = bw * bh * (z1 - z0);
    const double scale = degenerate ? 0.0 : 6.283185307179586476925 / (zmax - zmin);
    const int64_t HW = (int64_t)g.H * g.W;
    double es = 0.0, sm = 0.0;
    int nsp = 0, nb = 0, ns = 0, c0 = 0, c1 = 0;
    for (int j = lane; j < nsite; j += 32) {
        const int x = x0 + j % bw, y = y0 + (j / bw) % bh, z = z0 + j / (bw * bh);
        const int64_t i = z * HW + (int64_t)y * g.W + x;
        const bool gap = mask[i] != 0;
        const double pi = gap ? 0.0 : ((double)values[i] - zmin) * scale;
        if (gap) {
            if (((x + y + z) & 1) == 0) ++c0; else ++c1;
        } else {
            sm += pi;
            ++ns;
        }
        const int64_t nbr[3] = {x + 1 < g.W ? i + 1 : -1, y + 1 < g.H ? i + g.W : -1,
                                z + 1 < g.D ? i + HW : -1};
        for (int k = 0; k < 3; ++k) {
            if (nbr[k] < 0) continue;
            ++nb;
            if (!gap && !mask[nbr[k]]) {
                const double pj = ((double)values[nbr[k]] - zmin) * scale;
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
        c0 += __shfl_xor_sync(0xffffffffu, c0, d);
        c1 += __shfl_xor_sync(0xffffffffu, c1, d);
    }
    if (lane == 0) {
        Es[warp] = es;
        Nsp[warp] = nsp;
        Nb[warp] = nb;
        ssum[warp] = sm;
        nsamp[warp] = ns;
        ngap0[warp] = c0;
        ngap1[warp] = c1;
    }
}

// Gap lists, block-major (one warp per block): (site index, block id).
__global__ void k3_build_lists(Geom3 g, const uint8_t* __restrict__ mask,
                               const int32_t* __restrict__ start0,
                               const int32_t* __restrict__ start1, uint2* __restrict__ list0,
                               uint2* __restrict__ list1) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= g.nblk) return;
    const int bx = warp % g.nbx, by = (warp / g.nbx) % g.nby, bz = warp / (g.nbx * g.nby);
    const int x0 = bx * g.lb, y0 = by * g.lb, z0 = bz * g.lb;
    const int x1 = min(g.W, x0 + g.lb), y1 = min(g.H, y0 + g.lb), z1 = min(g.D, z0 + g.lb);
    const int bw = x1 - x0, bh = y1 - y0, nsite = bw * bh * (z1 - z0);
    const int64_t HW = (int64_t)g.H * g.W;
    int o0 = start0[warp], o1 = start1[warp];
    for (int j0 = 0; j0 < nsite; j0 += 32) {
        const int j = j0 + lane;
        bool take = false;
        int c = 0;
        int64_t i = 0;
        if (j < nsite) {
            const int x = x0 + j % bw, y = y0 + (j / bw) % bh, z = z0 + j / (bw * bh);
            i = z * HW + (int64_t)y * g.W + x;
            take = mask[i] != 0;
            c = (x + y + z) & 1;
        }
        const unsigned m0 = __ballot_sync(0xffffffffu, take && c == 0);
        const unsigned m1 = __ballot_sync(0xffffffffu, take && c == 1);
        if (take) {
            const unsigned below = (1u << lane) - 1u;
            const uint2 e = make_uint2((uint32_t)i, (uint32_t)warp);
            if (c == 0) list0[o0 + __popc(m0 & below)] = e;
            else list1[o1 + __popc(m1 & below)] = e;
        }
        o0 += __popc(m0);
        o1 += __popc(m1);
    }
}

struct Args3 {
    Geom3 g;
    Model m;
    uint32_t key0, key1;
    int colour;
    const uint2* list;
    int64_t n_list;
    float2* ang;             // [2][D][H][Wh][np]
    const float* beta;       // [nblk]
    const uint8_t* running;  // [nblk][Rp] or nullptr (every lane r < R)
    double* eacc;            // [nblk][Rp] FP64 per-sweep changes
    double* ecur;            // [nblk][Rp] (energy pass)
    int np, R, Rp;
    uint32_t pair_base;      // Philox counter word 2 of lane pair 0 (realization base / 2)
    uint32_t ctr1;           // t | tag << 16
    int energy;
};

// The six neighbours' angles of site (z, y, x) for one realization pair, and
// which of them exist. Order: -x, +x, -y, +y, -z, +z.
__device__ __forceinline__ void neighbours3(const Args3& a, int z, int y, int x, int p, float2 v[6],
                                            bool ex[6]) {
    const Geom3& g = a.g;
    const int co = a.colour ^ 1;
    ex[0] = x > 0;
    ex[1] = x + 1 < g.W;
    ex[2] = y > 0;
    ex[3] = y + 1 < g.H;
    ex[4] = z > 0;
    ex[5] = z + 1 < g.D;
    const int nz[6] = {z, z, z, z, z - 1, z + 1};
    const int ny[6] = {y, y, y - 1, y + 1, y, y};
    const int nx[6] = {x - 1, x + 1, x, x, x, x};
#pragma unroll
    for (int d = 0; d < 6; ++d)
        v[d] = ex[d] ? a.ang[hidx3(g, co, nz[d], ny[d], nx[d], a.np) + p] : make_float2(0.f, 0.f);
}

// One half-step: thread per (gap entry of the colour, realization pair).
__global__ void __launch_bounds__(256) k3_sweep(Args3 a) {
    const Geom3& g = a.g;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t e = t / a.np;
    const int p = (int)(t % a.np);
    const int lane = threadIdx.x & 31;
    float ao0 = 0.f, ao1 = 0.f, ae[3][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    int b = -1;
    if (e < a.n_list) {
        const uint2 en = a.list[e];
        b = (int)en.y;
        const int64_t HW = (int64_t)g.H * g.W;
        const int z = (int)(en.x / HW), y = (int)((en.x % HW) / g.W), x = (int)(en.x % g.W);
        const int rl = 2 * p;
        bool run0, run1;
        if (a.running) {
            run0 = a.running[(size_t)b * a.Rp + rl] != 0;
            run1 = a.running[(size_t)b * a.Rp + rl + 1] != 0;
        } else {
            run0 = rl < a.R;
            run1 = rl + 1 < a.R;
        }
        if (run0 || run1) {
            uint32_t w[4];
            philox4x32_10(en.x, a.ctr1, a.pair_base + (uint32_t)p, 0u, a.key0, a.key1, w);
            float2 v[6];
            bool ex[6];
            neighbours3(a, z, y, x, p, v, ex);
            float nc0[6], ns0[6], nc1[6], ns1[6];
            float C0 = 0.f, S0 = 0.f, C1 = 0.f, S1 = 0.f;
#pragma unroll
            for (int d = 0; d < 6; ++d) {
                const float mk = ex[d] ? 1.0f : 0.0f;
                float s0, c0, s1, c1;
                __sincosf(a.m.q * v[d].x, &s0, &c0);
                __sincosf(a.m.q * v[d].y, &s1, &c1);
                nc0[d] = mk * c0; ns0[d] = mk * s0; nc1[d] = mk * c1; ns1[d] = mk * s1;
            }
            C0 = ((nc0[0] + nc0[1]) + (nc0[2] + nc0[3])) + (nc0[4] + nc0[5]);
            S0 = ((ns0[0] + ns0[1]) + (ns0[2] + ns0[3])) + (ns0[4] + ns0[5]);
            C1 = ((nc1[0] + nc1[1]) + (nc1[2] + nc1[3])) + (nc1[4] + nc1[5]);
            S1 = ((ns1[0] + ns1[1]) + (ns1[2] + ns1[3])) + (ns1[4] + ns1[5]);
            const size_t h = hidx3(g, a.colour, z, y, x, a.np) + p;
            const float2 ph = a.ang[h];
            float2 out = ph;
            const float beta = a.beta[b];
            // faces of the block whose bond belongs to the neighbouring block
            const bool edge[3] = {x > 0 && x % g.lb == 0, y > 0 && y % g.lb == 0,
                                  z > 0 && z % g.lb == 0};
            const float J = a.m.J;
            if (run0) {
                const SiteNew n = site_update<float>(ph.x, C0, S0, u01(w[0]), u01(w[1]), beta, a.m);
                out.x = n.phi;
                ao0 += n.dE;
                if (edge[0] || edge[1] || edge[2]) {
                    float cn, sn;
                    final_cs(n, C0, S0, cn, sn);
                    const float dc = cn - n.co, ds = sn - n.so;
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        if (edge[k]) {
                            const float d = -J * (dc * nc0[2 * k] + ds * ns0[2 * k]);
                            ao0 -= d;
                            ae[k][0] += d;
                        }
                }
            }
            if (run1) {
                const SiteNew n = site_update<float>(ph.y, C1, S1, u01(w[2]), u01(w[3]), beta, a.m);
                out.y = n.phi;
                ao1 += n.dE;
                if (edge[0] || edge[1] || edge[2]) {
                    float cn, sn;
                    final_cs(n, C1, S1, cn, sn);
                    const float dc = cn - n.co, ds = sn - n.so;
#pragma unroll
                    for (int k = 0; k < 3; ++k)
                        if (edge[k]) {
                            const float d = -J * (dc * nc1[2 * k] + ds * ns1[2 * k]);
                            ao1 -= d;
                            ae[k][1] += d;
                        }
                }
            }
            a.ang[h] = out;
        }
    }
    if (!a.energy) return;
    // Block changes: one warp sum when every lane works on the same block
    // and pair (block-major lists make that the common case), else atomics.
    const int key = b < 0 ? -1 : b * a.np + p;
    const int k0 = __shfl_sync(0xffffffffu, key, 0);
    const bool uni = __all_sync(0xffffffffu, key == k0) && k0 >= 0;
    const size_t off[4] = {0, 1, (size_t)g.nbx, (size_t)g.nbx * g.nby};
    float vals[4][2] = {{ao0, ao1}, {ae[0][0], ae[0][1]}, {ae[1][0], ae[1][1]}, {ae[2][0], ae[2][1]}};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float v0 = vals[k][0], v1 = vals[k][1];
        if (uni) {
            for (int d = 16; d > 0; d >>= 1) {
                v0 += __shfl_xor_sync(0xffffffffu, v0, d);
                v1 += __shfl_xor_sync(0xffffffffu, v1, d);
            }
            if (lane != 0) continue;
        }
        if (b < 0 || (v0 == 0.0f && v1 == 0.0f)) continue;
        double* ea = a.eacc + ((size_t)b - off[k]) * a.Rp + 2 * p;
        if (v0 != 0.0f) atomicAdd(ea, (double)v0);
        if (v1 != 0.0f) atomicAdd(ea + 1, (double)v1);
    }
}

// Block energies from scratch (FP64 atomics into ecur, which holds E_s,b):
// colour 1 adds every bond of its gap sites, colour 0 only the bonds to
// sample neighbours, each to the block that owns it.
__global__ void k3_energy(Args3 a, const uint8_t* __restrict__ mask) {
    const Geom3& g = a.g;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t e = t / a.np;
    const int p = (int)(t % a.np);
    if (e >= a.n_list) return;
    const uint2 en = a.list[e];
    const int b = (int)en.y;
    const int64_t HW = (int64_t)g.H * g.W;
    const int z = (int)(en.x / HW), y = (int)((en.x % HW) / g.W), x = (int)(en.x % g.W);
    float2 v[6];
    bool ex[6];
    neighbours3(a, z, y, x, p, v, ex);
    const float2 ph = a.ang[hidx3(g, a.colour, z, y, x, a.np) + p];
    const int64_t ni[6] = {-1, 1, -(int64_t)g.W, (int64_t)g.W, -HW, HW};
    const size_t owner_off[6] = {1, 0, (size_t)g.nbx, 0, (size_t)g.nbx * g.nby, 0};
    const bool face[6] = {x % g.lb == 0, false, y % g.lb == 0, false, z % g.lb == 0, false};
    for (int d = 0; d < 6; ++d) {
        if (!ex[d]) continue;
        if (a.colour == 0 && mask[(int64_t)en.x + ni[d]]) continue;   // gap-gap bonds: colour 1
        const double b0 = -a.m.J * cos((double)a.m.q * ((double)ph.x - (double)v[d].x));
        const double b1 = -a.m.J * cos((double)a.m.q * ((double)ph.y - (double)v[d].y));
        const size_t ob = (size_t)b - (face[d] ? owner_off[d] : 0);
        atomicAdd(&a.ecur[ob * a.Rp + 2 * p], b0);
        atomicAdd(&a.ecur[ob * a.Rp + 2 * p + 1], b1);
    }
}

// State: samples in every lane, gaps at their block's mean sample angle.
__global__ void k3_init(Geom3 g, const float* __restrict__ phi_s, const uint8_t* __restrict__ mask,
                        const float* __restrict__ init_angle, float2* __restrict__ ang, int np) {
    const int64_t n = (int64_t)g.D * g.H * g.W;
    const int64_t HW = (int64_t)g.H * g.W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * np;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / np;
        const int p = (int)(t % np);
        const int z = (int)(i / HW), y = (int)((i % HW) / g.W), x = (int)(i % g.W);
        const float v = mask[i] ? init_angle[block3(g, z, y, x)] : phi_s[i];
        ang[hidx3(g, (x + y + z) & 1, z, y, x, np) + p] = make_float2(v, v);
    }
}

__global__ void k3_accumulate(Geom3 g, const uint2* __restrict__ list, int64_t n_list, int colour,
                              const float2* __restrict__ ang, int np, int R,
                              double* __restrict__ sum) {
    const int64_t HW = (int64_t)g.H * g.W;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_list;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t i = list[e].x;
        const int z = (int)(i / HW), y = (int)((i % HW) / g.W), x = (int)(i % g.W);
        const size_t h = hidx3(g, colour, z, y, x, np);
        double s = 0.0;
        for (int r = 0; r < R; ++r) {
            const float2 v = ang[h + r / 2];
            s += (double)((r & 1) ? v.y : v.x);
        }
        sum[i] += s;
    }
}

__global__ void k3_predict(int64_t n, const float* __restrict__ values,
                           const uint8_t* __restrict__ mask, const double* __restrict__ sum,
                           double inv_r, double zmin, double zmax, float* __restrict__ out,
                           const float* __restrict__ truth, double* __restrict__ err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!mask[i]) {
            out[i] = values[i];
            continue;
        }
        const float z = (float)(zmin + (zmax - zmin) * sum[i] * inv_r / 6.283185307179586476925);
        out[i] = z;
        if (truth) {
            const double d = (double)truth[i] - (double)z;
            atomicAdd(&err[0], fabs(d));
            atomicAdd(&err[1], d * d);
        }
    }
}

__global__ void k3_get_state(Geom3 g, const float2* __restrict__ ang, int np, int r,
                             float* __restrict__ out) {
    const int64_t n = (int64_t)g.D * g.H * g.W;
    const int64_t HW = (int64_t)g.H * g.W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int z = (int)(i / HW), y = (int)((i % HW) / g.W), x = (int)(i % g.W);
        const float2 v = ang[hidx3(g, (x + y + z) & 1, z, y, x, np) + r / 2];
        out[i] = (r & 1) ? v.y : v.x;
    }
}

__global__ void k3_set_state(Geom3 g, const uint8_t* __restrict__ mask, float2* __restrict__ ang,
                             int np, int r, const float* __restrict__ in) {
    const int64_t n = (int64_t)g.D * g.H * g.W;
    const int64_t HW = (int64_t)g.H * g.W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!mask[i]) continue;
        const int z = (int)(i / HW), y = (int)((i % HW) / g.W), x = (int)(i % g.W);
        float2& v = ang[hidx3(g, (x + y + z) & 1, z, y, x, np) + r / 2];
        if (r & 1) v.y = in[i]; else v.x = in[i];
    }
}

__global__ void k3_fill_valid(uint8_t* running, int64_t n, int Rp, int R) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x)
        running[t] = (int)(t % Rp) < R ? 1 : 0;
}

inline int grid_of(int64_t n, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 32));
}

}  // namespace

struct mpr3_ctx {
    mpr_options opt{};
    Geom3 g{};
    Model m{};
    uint32_t key0 = 0, key1 = 0;
    cudaStream_t s = nullptr;
    int device = 0;
    std::string err;
    std::vector<void*> owned;
    double zmin = 0, zmax = 0;
    int degenerate = 0, calibrated = 0;
    int64_t n = 0, n_gap[2] = {0, 0};
    float *values = nullptr, *phi_s = nullptr, *init_angle = nullptr;
    uint8_t* mask = nullptr;
    uint2* list[2] = {nullptr, nullptr};
    int32_t* start[2] = {nullptr, nullptr};
    double *Es = nullptr, *es = nullptr, *inb = nullptr, *ssum = nullptr;
    int32_t *Nsp = nullptr, *Nb = nullptr, *nsamp = nullptr, *ngap = nullptr,
            *ngap_c[2] = {nullptr, nullptr}, *zero_slices = nullptr;
    int32_t* Nsp_cal = nullptr;  // calibrating blocks: sample bonds and gap sites
    float *T = nullptr, *beta = nullptr, *lo = nullptr, *hi = nullptr;
    double* ebar = nullptr;
    double* sum = nullptr;
    double* err_buf = nullptr;
    uint32_t* mm = nullptr;
    // batch
    int np = 0, R = 0, Rp = 0, batch_open = 0, t = 0;
    size_t ang_cap = 0, blk_cap = 0;
    int64_t n_allocs = 0;      // allocations seen by the alloc_test hook
    float2* ang = nullptr;
    double* eacc = nullptr;
    double *ecur = nullptr, *e_last = nullptr;
    uint8_t* running = nullptr;
    int32_t *stop = nullptr, *tcount = nullptr;
    int8_t* sigma = nullptr;
    uint32_t* work = nullptr;
    Control* ctl = nullptr;
    unsigned long long* counter = nullptr;
    int4* blk_rect = nullptr;
    int64_t realizations = 0, gap_updates = 0, cal_updates = 0;
    int64_t r_next = 0;          // index of the next realization (batches start even)
    uint32_t pair_base = 0;
    // profiling (opt.profile): event pairs around the realizations' sweeps
    // (their two half-steps) and around the calibration's iterations
    int64_t launches = 0, sim_hs = 0, cal_hs = 0;
    double sim_ms = 0.0, cal_ms = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_sim, ev_cal;
    unsigned long long* h_run = nullptr;   // pinned: running counts of two sweep chunks
};

namespace {

mpr_status fail3(mpr3_ctx* c, mpr_status st, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return st;
}

#define CK3(call)                                                                             \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail3(ctx, e_ == cudaErrorMemoryAllocation ? MPR_ENOMEM : MPR_ECUDA,       \
                         "%s failed: %s", #call, cudaGetErrorString(e_));                     \
    } while (0)
#define CKL3()                                                                                \
    do {                                                                                      \
        ++ctx->launches;                                                                      \
        cudaError_t e_ = cudaPeekAtLastError();                                               \
        if (e_ != cudaSuccess)                                                                \
            return fail3(ctx, MPR_ECUDA, "kernel launch failed: %s", cudaGetErrorString(e_)); \
    } while (0)
#define TRY3(x)                                  \
    do {                                         \
        mpr_status st_ = (x);                    \
        if (st_ != MPR_OK) return st_;           \
    } while (0)

template <class T>
mpr_status alloc3(mpr3_ctx* ctx, T** p, size_t count) {
    *p = nullptr;
    // Test hook: the alloc_test-th allocation of the context is refused.
    if (ctx->opt.alloc_test > 0 && ++ctx->n_allocs == ctx->opt.alloc_test)
        return fail3(ctx, MPR_ENOMEM, "allocation %d refused by the alloc_test hook",
                     ctx->opt.alloc_test);
    void* q = nullptr;
    if (pool_alloc(&q, std::max<size_t>(count, 1) * sizeof(T), ctx->device, ctx->s) !=
        cudaSuccess) {
        cudaGetLastError();
        return fail3(ctx, MPR_ENOMEM, "allocation of %zu bytes failed", count * sizeof(T));
    }
    ctx->owned.push_back(q);
    *p = static_cast<T*>(q);
    return MPR_OK;
}

void free3(mpr3_ctx* ctx, void* p) {
    if (!p) return;
    auto it = std::find(ctx->owned.begin(), ctx->owned.end(), p);
    if (it != ctx->owned.end()) ctx->owned.erase(it);
    pool_free(p, ctx->s);
}

Slices slices3(mpr3_ctx* ctx) {
    Slices sl{};
    sl.n = 1;
    sl.rect0 = make_int4(0, 0, ctx->g.D * ctx->g.H, ctx->g.W);
    sl.blk = ctx->blk_rect;
    sl.of_block = ctx->zero_slices;
    return sl;
}

// Batch buffers for `lanes` realization lanes (pairs of realizations).
mpr_status ensure3(mpr3_ctx* ctx, int lanes) {
    const int np = (lanes + 1) / 2, Rp = 2 * np;
    const size_t ang_need = 2 * (size_t)ctx->g.D * ctx->g.H * ctx->g.Wh * np;
    // (a failed allocation leaves the capacity at 0 and every pointer of its
    // group null, so the next call allocates the group again)
    if (ang_need > ctx->ang_cap) {
        free3(ctx, ctx->ang);
        ctx->ang = nullptr;
        ctx->ang_cap = 0;
        TRY3(alloc3(ctx, &ctx->ang, ang_need));
        ctx->ang_cap = ang_need;
    }
    const size_t blk = (size_t)ctx->g.nblk * Rp;
    if (blk > ctx->blk_cap) {
        for (void* p : {(void*)ctx->eacc, (void*)ctx->ecur, (void*)ctx->e_last, (void*)ctx->running,
                        (void*)ctx->stop, (void*)ctx->sigma, (void*)ctx->work, (void*)ctx->tcount})
            free3(ctx, p);
        ctx->eacc = nullptr; ctx->ecur = nullptr; ctx->e_last = nullptr; ctx->running = nullptr;
        ctx->stop = nullptr; ctx->sigma = nullptr; ctx->work = nullptr; ctx->tcount = nullptr;
        ctx->blk_cap = 0;
        TRY3(alloc3(ctx, &ctx->eacc, blk));
        TRY3(alloc3(ctx, &ctx->ecur, blk));
        TRY3(alloc3(ctx, &ctx->e_last, blk));
        TRY3(alloc3(ctx, &ctx->running, blk));
        TRY3(alloc3(ctx, &ctx->stop, blk));
        TRY3(alloc3(ctx, &ctx->sigma, blk));
        TRY3(alloc3(ctx, &ctx->work, 2 * (size_t)ctx->g.nblk * np));
        TRY3(alloc3(ctx, &ctx->tcount, (size_t)Rp));
        ctx->blk_cap = blk;
    }
    ctx->np = np;
    ctx->Rp = Rp;
    CK3(cudaMemsetAsync(ctx->eacc, 0, blk * sizeof(double), ctx->s));
    CK3(cudaMemsetAsync(ctx->ctl, 0, sizeof(Control), ctx->s));
    return MPR_OK;
}

Args3 args3(mpr3_ctx* ctx, int colour, bool simulate) {
    Args3 a{};
    a.g = ctx->g;
    a.m = ctx->m;
    a.key0 = ctx->key0;
    a.key1 = ctx->key1;
    a.colour = colour;
    a.list = ctx->list[colour];
    a.n_list = ctx->n_gap[colour];
    a.ang = ctx->ang;
    a.beta = ctx->beta;
    a.running = simulate ? ctx->running : nullptr;
    a.eacc = ctx->eacc;
    a.ecur = ctx->ecur;
    a.np = ctx->np;
    a.pair_base = simulate ? ctx->pair_base : 0u;
    a.R = ctx->R;
    a.Rp = ctx->Rp;
    a.energy = 1;
    return a;
}

mpr_status init3(mpr3_ctx* ctx) {
    const int64_t n = ctx->n;
    k3_init<<<grid_of(n * ctx->np), 256, 0, ctx->s>>>(ctx->g, ctx->phi_s, ctx->mask,
                                                      ctx->init_angle, ctx->ang, ctx->np);
    CKL3();
    return MPR_OK;
}

mpr_status energy3(mpr3_ctx* ctx) {
    launch_ecur_reset(ctx->g.nblk, ctx->Rp, ctx->Es, ctx->ecur, ctx->eacc, ctx->s);
    CKL3();
    for (int c = 0; c < 2; ++c) {
        Args3 a = args3(ctx, c, false);
        a.R = ctx->Rp;
        if (a.n_list == 0) continue;
        k3_energy<<<grid_of(a.n_list * a.np), 256, 0, ctx->s>>>(a, ctx->mask);
        CKL3();
    }
    return MPR_OK;
}

mpr_status halfstep3(mpr3_ctx* ctx, int colour, uint32_t ctr1, bool simulate) {
    Args3 a = args3(ctx, colour, simulate);
    a.ctr1 = ctr1;
    if (a.n_list == 0) return MPR_OK;
    const int64_t threads = a.n_list * a.np;
    k3_sweep<<<(unsigned)((threads + 255) / 256), 256, 0, ctx->s>>>(a);
    CKL3();
    return MPR_OK;
}

// After a stream synchronisation: the recorded event pairs into the totals.
void collect3(mpr3_ctx* ctx) {
    for (int which = 0; which < 2; ++which) {
        auto& v = which ? ctx->ev_cal : ctx->ev_sim;
        double& acc = which ? ctx->cal_ms : ctx->sim_ms;
        for (auto& pr : v) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) acc += ms;
            else cudaGetLastError();
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        v.clear();
    }
}

// An event pair on the context's stream when profiling (nullptr otherwise).
std::pair<cudaEvent_t, cudaEvent_t> begin_timing3(mpr3_ctx* ctx) {
    std::pair<cudaEvent_t, cudaEvent_t> e{nullptr, nullptr};
    if (!ctx->opt.profile) return e;
    if (cudaEventCreate(&e.first) != cudaSuccess || cudaEventCreate(&e.second) != cudaSuccess) {
        cudaGetLastError();
        if (e.first) cudaEventDestroy(e.first);
        return {nullptr, nullptr};
    }
    cudaEventRecord(e.first, ctx->s);
    return e;
}

mpr_status sweep3(mpr3_ctx* ctx) {
    ctx->t += 1;
    const auto ev = begin_timing3(ctx);
    for (int c = 0; c < 2; ++c) TRY3(halfstep3(ctx, c, (uint32_t)ctx->t, true));
    ctx->sim_hs += 2;
    if (ev.first) {
        cudaEventRecord(ev.second, ctx->s);
        ctx->ev_sim.push_back(ev);
    }
    const int64_t items = (int64_t)ctx->g.nblk * ctx->np;
    const int grid = (int)std::min<int64_t>((items * 2 + 255) / 256, 152 * 16);
    launch_stop_targeted(2, ctx->np, ctx->Rp, ctx->zero_slices, grid, ctx->ctl, ctx->work,
                         (uint32_t)items, ctx->es, ctx->inb, ctx->Nsp, ctx->eacc, ctx->ecur,
                         ctx->sigma, ctx->running, ctx->stop, ctx->tcount, ctx->e_last, -1, ctx->s);
    CKL3();
    launch_stop_rest(ctx->g.nblk, ctx->np, 2, ctx->Rp, ctx->opt.n_max, ctx->zero_slices, grid,
                     ctx->ctl, ctx->work, ctx->work, (uint32_t)items, ctx->Nsp, ctx->running,
                     ctx->stop, ctx->tcount, 0, -1, ctx->s);
    CKL3();
    return MPR_OK;
}

}  // namespace

extern "C" {

void mpr3_destroy(mpr3_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->s);
    collect3(ctx);
    for (void* p : ctx->owned) pool_free(p, ctx->s);
    cudaStreamSynchronize(ctx->s);
    pinned_release(ctx->h_run);
    delete ctx;
}

mpr_status mpr3_get_profile(mpr3_ctx* ctx, mpr_profile* p) {
    if (!ctx || !p) return MPR_EINVAL;
    if (cudaStreamSynchronize(ctx->s) != cudaSuccess) return fail3(ctx, MPR_ECUDA, "sync failed");
    collect3(ctx);
    std::memset(p, 0, sizeof(*p));
    p->kernel_launches = ctx->launches;
    p->sim_halfstep_launches = ctx->sim_hs;
    p->cal_halfstep_launches = ctx->cal_hs;
    p->sim_halfstep_ms = ctx->sim_ms;
    p->cal_halfstep_ms = ctx->cal_ms;
    return MPR_OK;
}

const char* mpr3_last_error(const mpr3_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

mpr_status mpr3_create(const mpr_grid3* grid, const uint8_t* mask_in, const float* values_in,
                       const mpr_options* opt_in, mpr3_ctx** out) {
    if (!out) return MPR_EINVAL;
    *out = nullptr;
    if (!grid || !mask_in || !values_in) return MPR_EINVAL;
    const int D = grid->depth, H = grid->height, W = grid->width, lb = grid->block;
    if (D < 1 || H < 1 || W < 1 || lb < 1 || (int64_t)D * H * W > 0x7fffffffLL) return MPR_EINVAL;
    mpr3_ctx* ctx = new (std::nothrow) mpr3_ctx();
    if (!ctx) return MPR_ENOMEM;
    auto bail = [&](mpr_status st) {
        mpr3_destroy(ctx);
        return st;
    };
    if (opt_in) ctx->opt = *opt_in; else mpr_default_options(&ctx->opt);
    const mpr_options& o = ctx->opt;
    if (!(o.q > 0.0 && o.q <= 0.5) || !(o.J > 0.0) || o.n_max < 1 || o.n_max > 65535 ||
        o.n_eq < 0 || o.n_meas < 1 || o.n_eq + o.n_meas > 65535 || o.n_bisect < 0 ||
        o.cal_chains < 1 || o.cal_chains > 4096 || !(o.t_lo > 0.0f && o.t_hi > o.t_lo) ||
        o.stop_rule != MPR_STOP_CROSS ||   // (3-D: the first-crossing stop only)
        o.alloc_test < 0)
        return bail(MPR_EINVAL);
    Geom3& g = ctx->g;
    g.D = D; g.H = H; g.W = W; g.Wh = (W + 1) / 2; g.lb = lb;
    g.nbx = (W + lb - 1) / lb; g.nby = (H + lb - 1) / lb; g.nbz = (D + lb - 1) / lb;
    if ((int64_t)g.nbx * g.nby * g.nbz > MAX_BLOCKS) return bail(MPR_EINVAL);
    g.nblk = g.nbx * g.nby * g.nbz;
    ctx->m.q = (float)o.q;
    ctx->m.J = (float)o.J;
    ctx->m.inv_q = (float)(1.0 / o.q);
    ctx->m.overrelax = o.overrelax ? 1 : 0;
    ctx->key0 = (uint32_t)(o.seed & 0xffffffffu);
    ctx->key1 = (uint32_t)(o.seed >> 32) ^ o.slice_id;
    ctx->s = (cudaStream_t)o.cuda_stream;
    if (cudaGetDevice(&ctx->device) != cudaSuccess) return bail(MPR_ECUDA);
    const int64_t n = (int64_t)D * H * W;
    ctx->n = n;
    mpr_status st;
#define ST3(x) do { st = (x); if (st != MPR_OK) return bail(st); } while (0)
    ST3(alloc3(ctx, &ctx->values, n));
    ST3(alloc3(ctx, &ctx->mask, n));
    ST3(alloc3(ctx, &ctx->phi_s, n));
    ST3(alloc3(ctx, &ctx->sum, n));
    for (auto* p : {&ctx->Es, &ctx->es, &ctx->inb, &ctx->ssum, &ctx->ebar})
        ST3(alloc3(ctx, p, g.nblk));
    for (auto* p : {&ctx->Nsp, &ctx->Nb, &ctx->nsamp, &ctx->ngap, &ctx->ngap_c[0], &ctx->ngap_c[1],
                    &ctx->zero_slices, &ctx->Nsp_cal})
        ST3(alloc3(ctx, p, g.nblk));
    for (auto* p : {&ctx->init_angle, &ctx->T, &ctx->beta, &ctx->lo, &ctx->hi})
        ST3(alloc3(ctx, p, g.nblk));
    ST3(alloc3(ctx, &ctx->start[0], g.nblk + 1));
    ST3(alloc3(ctx, &ctx->start[1], g.nblk + 1));
    ST3(alloc3(ctx, &ctx->err_buf, 2));
    ST3(alloc3(ctx, &ctx->mm, 2));
    ST3(alloc3(ctx, &ctx->ctl, 1));
    ST3(alloc3(ctx, &ctx->counter, 1));
    ST3(alloc3(ctx, &ctx->blk_rect, 1));
    const int4 bk = make_int4(0, 0, g.nbz * g.nby, g.nbx);
    if (cudaMemcpyAsync(ctx->values, values_in, n * 4, cudaMemcpyDefault, ctx->s) ||
        cudaMemcpyAsync(ctx->mask, mask_in, n, cudaMemcpyDefault, ctx->s) ||
        cudaMemsetAsync(ctx->zero_slices, 0, g.nblk * 4, ctx->s) ||
        cudaMemcpyAsync(ctx->blk_rect, &bk, sizeof(bk), cudaMemcpyHostToDevice, ctx->s) ||
        cudaMemsetAsync(ctx->sum, 0, n * 8, ctx->s))
        return bail(MPR_ECUDA);
    uint32_t mm[2] = {0xffffffffu, 0u};
    if (cudaMemcpyAsync(ctx->mm, mm, 8, cudaMemcpyHostToDevice, ctx->s)) return bail(MPR_ECUDA);
    k3_minmax<<<grid_of(n), 256, 0, ctx->s>>>(ctx->values, ctx->mask, n, ctx->mm);
    if (cudaMemcpyAsync(mm, ctx->mm, 8, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaStreamSynchronize(ctx->s))
        return bail(MPR_ECUDA);
    if (mm[0] == 0xffffffffu) {
        ctx->degenerate = 1;
    } else {
        ctx->zmin = (double)ord2f(mm[0]);
        ctx->zmax = (double)ord2f(mm[1]);
        ctx->degenerate = !(ctx->zmax > ctx->zmin);
    }
    k3_layout<<<grid_of(n), 256, 0, ctx->s>>>(n, ctx->values, ctx->mask, ctx->zmin, ctx->zmax,
                                              ctx->degenerate, ctx->phi_s);
    const int bblocks = (int)(((int64_t)g.nblk * 32 + 255) / 256);
    k3_block_stats<<<bblocks, 256, 0, ctx->s>>>(g, ctx->values, ctx->mask, ctx->zmin, ctx->zmax,
                                                ctx->degenerate, o.q, o.J, ctx->Es, ctx->Nsp,
                                                ctx->Nb, ctx->ssum, ctx->nsamp, ctx->ngap_c[0],
                                                ctx->ngap_c[1]);
    launch_scan(ctx->ngap_c[0], g.nblk, ctx->start[0], ctx->s);
    launch_scan(ctx->ngap_c[1], g.nblk, ctx->start[1], ctx->s);
    std::vector<int32_t> s0(g.nblk + 1), s1(g.nblk + 1), nsp(g.nblk), nsm(g.nblk), ng0(g.nblk),
        ng1(g.nblk), nbv(g.nblk);
    std::vector<double> ssum(g.nblk), esv(g.nblk);
    if (cudaPeekAtLastError() ||
        cudaMemcpyAsync(s0.data(), ctx->start[0], s0.size() * 4, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(s1.data(), ctx->start[1], s1.size() * 4, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(nsp.data(), ctx->Nsp, g.nblk * 4, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(nsm.data(), ctx->nsamp, g.nblk * 4, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(ng0.data(), ctx->ngap_c[0], g.nblk * 4, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(ng1.data(), ctx->ngap_c[1], g.nblk * 4, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(ssum.data(), ctx->ssum, g.nblk * 8, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(esv.data(), ctx->Es, g.nblk * 8, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(nbv.data(), ctx->Nb, g.nblk * 4, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaStreamSynchronize(ctx->s))
        return bail(MPR_ECUDA);
    ctx->n_gap[0] = s0[g.nblk];
    ctx->n_gap[1] = s1[g.nblk];
    int64_t pairs = 0, samples = 0;
    double gsum = 0.0;
    std::vector<float> init(g.nblk);
    std::vector<int32_t> ng(g.nblk);
    std::vector<double> es_h(g.nblk), inb_h(g.nblk);
    std::vector<int32_t> nsp_cal(g.nblk);
    for (int b = 0; b < g.nblk; ++b) {
        nsp_cal[b] = (ng0[b] + ng1[b]) > 0 ? nsp[b] : 0;
        pairs += nsp[b];
        samples += nsm[b];
        gsum += ssum[b];
        ng[b] = ng0[b] + ng1[b];
        es_h[b] = nsp[b] > 0 ? esv[b] / (double)nsp[b] : 0.0;
        inb_h[b] = nbv[b] > 0 ? 1.0 / (double)nbv[b] : 0.0;
    }
    const double gmean = samples ? gsum / (double)samples : 0.0;
    for (int b = 0; b < g.nblk; ++b) init[b] = (float)(nsm[b] > 0 ? ssum[b] / nsm[b] : gmean);
    if (pairs == 0 && ctx->n_gap[0] + ctx->n_gap[1] > 0) {
        mpr3_destroy(ctx);
        return MPR_ENOSAMPLES;
    }
    ST3(alloc3(ctx, &ctx->list[0], ctx->n_gap[0]));
    ST3(alloc3(ctx, &ctx->list[1], ctx->n_gap[1]));
    if (cudaMemcpyAsync(ctx->init_angle, init.data(), g.nblk * 4, cudaMemcpyHostToDevice, ctx->s) ||
        cudaMemcpyAsync(ctx->es, es_h.data(), g.nblk * 8, cudaMemcpyHostToDevice, ctx->s) ||
        cudaMemcpyAsync(ctx->inb, inb_h.data(), g.nblk * 8, cudaMemcpyHostToDevice, ctx->s) ||
        cudaMemcpyAsync(ctx->ngap, ng.data(), g.nblk * 4, cudaMemcpyHostToDevice, ctx->s) ||
        cudaMemcpyAsync(ctx->Nsp_cal, nsp_cal.data(), g.nblk * 4, cudaMemcpyHostToDevice, ctx->s))
        return bail(MPR_ECUDA);
    k3_build_lists<<<bblocks, 256, 0, ctx->s>>>(g, ctx->mask, ctx->start[0], ctx->start[1],
                                                ctx->list[0], ctx->list[1]);
    if (cudaPeekAtLastError() || cudaStreamSynchronize(ctx->s)) return bail(MPR_ECUDA);
#undef ST3
    *out = ctx;
    return MPR_OK;
}

mpr_status mpr3_get_block_stats(mpr3_ctx* ctx, double* Es, int32_t* Nsp, int32_t* Nb,
                                float* mean_angle, int32_t* n_gap) {
    if (!ctx) return MPR_EINVAL;
    const size_t nb = (size_t)ctx->g.nblk;
    if (Es) CK3(cudaMemcpyAsync(Es, ctx->Es, nb * 8, cudaMemcpyDefault, ctx->s));
    if (Nsp) CK3(cudaMemcpyAsync(Nsp, ctx->Nsp, nb * 4, cudaMemcpyDefault, ctx->s));
    if (Nb) CK3(cudaMemcpyAsync(Nb, ctx->Nb, nb * 4, cudaMemcpyDefault, ctx->s));
    if (mean_angle) CK3(cudaMemcpyAsync(mean_angle, ctx->init_angle, nb * 4, cudaMemcpyDefault, ctx->s));
    if (n_gap) CK3(cudaMemcpyAsync(n_gap, ctx->ngap, nb * 4, cudaMemcpyDefault, ctx->s));
    CK3(cudaStreamSynchronize(ctx->s));
    return MPR_OK;
}

mpr_status mpr3_set_temperatures(mpr3_ctx* ctx, const float* T) {
    if (!ctx || !T) return MPR_EINVAL;
    ctx->err.clear();
    const int nb = ctx->g.nblk;
    std::vector<float> h(nb), bt(nb);
    CK3(cudaMemcpyAsync(h.data(), T, nb * 4, cudaMemcpyDefault, ctx->s));
    CK3(cudaStreamSynchronize(ctx->s));
    for (int b = 0; b < nb; ++b) {
        if (!(h[b] > 0.0f) || !std::isfinite(h[b])) return fail3(ctx, MPR_EINVAL, "T_%d not > 0", b);
        bt[b] = 1.0f / h[b];
    }
    CK3(cudaMemcpyAsync(ctx->T, h.data(), nb * 4, cudaMemcpyHostToDevice, ctx->s));
    CK3(cudaMemcpyAsync(ctx->beta, bt.data(), nb * 4, cudaMemcpyHostToDevice, ctx->s));
    CK3(cudaStreamSynchronize(ctx->s));
    ctx->calibrated = 1;
    return MPR_OK;
}

// Bisection on the per-block T (Sec. 2.1 energy matching per block): every
// iteration starts the chains afresh, runs n_eq + n_meas sweeps at the
// midpoints and keeps the half of each bracket on the side of e_s,b.
mpr_status mpr3_calibrate(mpr3_ctx* ctx, float* T_out) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    const Geom3& g = ctx->g;
    const mpr_options& o = ctx->opt;
    ctx->batch_open = 0;
    const Slices sl = slices3(ctx);
    if (ctx->degenerate) {
        std::vector<float> h(g.nblk, o.t_lo);
        TRY3(mpr3_set_temperatures(ctx, h.data()));
    } else {
        const int chains = o.cal_chains;
        TRY3(ensure3(ctx, chains));
        ctx->R = chains;
        launch_cal_init(g.nblk, o.t_lo, o.t_hi, ctx->lo, ctx->hi, ctx->ebar, ctx->ctl, ctx->s);
        CKL3();
        const double inv_count = 1.0 / ((double)o.n_meas * (double)chains);
        const auto ev = begin_timing3(ctx);
        for (int k = 0; k < o.n_bisect; ++k) {
            launch_cal_mid(g.nblk, ctx->Nsp_cal, ctx->lo, ctx->hi, ctx->T, ctx->ctl, ctx->s);
            ++ctx->launches;
            launch_cal_fill(sl, g.nbx, ctx->Nsp_cal, ctx->T, ctx->beta, ctx->s);
            CKL3();
            TRY3(init3(ctx));
            TRY3(energy3(ctx));
            for (int sw = 1; sw <= o.n_eq + o.n_meas; ++sw) {
                const uint32_t ctr1 = (uint32_t)sw | ((uint32_t)(1 + k) << 16);
                for (int c = 0; c < 2; ++c) TRY3(halfstep3(ctx, c, ctr1, false));
                launch_cal_step(g.nblk, ctx->Rp, chains, o.n_eq, sw, ctx->ctl, ctx->inb, ctx->eacc,
                                ctx->ecur, ctx->ebar, ctx->s);
                CKL3();
            }
            launch_cal_update(g.nblk, inv_count, ctx->es, ctx->Nsp_cal, ctx->T, ctx->lo, ctx->hi,
                              ctx->ebar, ctx->ctl, o.n_bisect, 0, ctx->s);
            CKL3();
        }
        if (ev.first) {
            cudaEventRecord(ev.second, ctx->s);
            ctx->ev_cal.push_back(ev);
        }
        ctx->cal_hs += (int64_t)o.n_bisect * (o.n_eq + o.n_meas) * 2;
        launch_cal_mid(g.nblk, ctx->Nsp_cal, ctx->lo, ctx->hi, ctx->T, ctx->ctl, ctx->s);
        ++ctx->launches;
        launch_cal_fill(sl, g.nbx, ctx->Nsp_cal, ctx->T, ctx->beta, ctx->s);
        CKL3();
        ctx->cal_updates += (int64_t)o.n_bisect * (o.n_eq + o.n_meas) * chains *
                            (ctx->n_gap[0] + ctx->n_gap[1]);
        ctx->calibrated = 1;
    }
    if (T_out) CK3(cudaMemcpyAsync(T_out, ctx->T, g.nblk * 4, cudaMemcpyDefault, ctx->s));
    CK3(cudaStreamSynchronize(ctx->s));
    return MPR_OK;
}

mpr_status mpr3_sim_begin(mpr3_ctx* ctx, int32_t n) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    if (n < 1 || n > 65534) return fail3(ctx, MPR_EINVAL, "n_realizations in [1, 65534]");
    if (ctx->batch_open) return fail3(ctx, MPR_ESTATE, "a batch is open");
    if (!ctx->calibrated) return fail3(ctx, MPR_ESTATE, "calibrate or set temperatures first");
    const int64_t base = (ctx->r_next + 1) / 2 * 2;   // lane pairs align with Philox blocks
    if (base + n > (int64_t)0x1FFFFFFFF) return fail3(ctx, MPR_EINVAL, "realization index overflow");
    ctx->pair_base = (uint32_t)(base / 2);
    TRY3(ensure3(ctx, n));
    ctx->R = n;
    ctx->t = 0;
    const int64_t nbr = (int64_t)ctx->g.nblk * ctx->Rp;
    k3_fill_valid<<<grid_of(nbr), 256, 0, ctx->s>>>(ctx->running, nbr, ctx->Rp, n);
    CKL3();
    TRY3(init3(ctx));
    CK3(cudaMemsetAsync(ctx->tcount, 0, ctx->Rp * sizeof(int32_t), ctx->s));
    TRY3(energy3(ctx));
    launch_stop_init(ctx->g.nblk, ctx->Rp, ctx->zero_slices, ctx->es, ctx->inb, ctx->Nsp,
                     ctx->ngap, ctx->ecur, ctx->sigma, ctx->running, ctx->stop, ctx->tcount,
                     ctx->e_last, ctx->s);
    CKL3();
    const int64_t items = (int64_t)ctx->g.nblk * ctx->np;
    launch_stop_rest(ctx->g.nblk, ctx->np, 2, ctx->Rp, ctx->opt.n_max, ctx->zero_slices,
                     (int)std::min<int64_t>((items + 255) / 256, 152 * 16), ctx->ctl, nullptr,
                     ctx->work, (uint32_t)items, ctx->Nsp, ctx->running, ctx->stop, ctx->tcount, 0,
                     -1, ctx->s);
    CKL3();
    ctx->batch_open = 1;
    return MPR_OK;
}

mpr_status mpr3_halfstep(mpr3_ctx* ctx, int32_t colour, int32_t t, int32_t tag) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    if (!ctx->batch_open) return fail3(ctx, MPR_ESTATE, "no open batch");
    if (colour < 0 || colour > 1 || t < 0 || t > 65535 || tag < 0 || tag > 65535)
        return fail3(ctx, MPR_EINVAL, "bad colour, t or tag");
    TRY3(halfstep3(ctx, colour, (uint32_t)t | ((uint32_t)tag << 16), true));
    CK3(cudaStreamSynchronize(ctx->s));
    return MPR_OK;
}

mpr_status mpr3_sim_end(mpr3_ctx* ctx) {
    if (!ctx) return MPR_EINVAL;
    if (!ctx->batch_open) return fail3(ctx, MPR_ESTATE, "no open batch");
    for (int c = 0; c < 2; ++c) {
        if (ctx->n_gap[c] == 0) continue;
        k3_accumulate<<<grid_of(ctx->n_gap[c]), 256, 0, ctx->s>>>(
            ctx->g, ctx->list[c], ctx->n_gap[c], c, ctx->ang, ctx->np, ctx->R, ctx->sum);
        CKL3();
    }
    CK3(cudaMemsetAsync(ctx->counter, 0, 8, ctx->s));
    launch_count_updates(ctx->g.nblk, ctx->Rp, ctx->stop, ctx->ngap, ctx->counter, ctx->s);
    CKL3();
    unsigned long long h = 0;
    CK3(cudaMemcpyAsync(&h, ctx->counter, 8, cudaMemcpyDeviceToHost, ctx->s));
    CK3(cudaStreamSynchronize(ctx->s));
    ctx->gap_updates += (int64_t)h;
    ctx->realizations += ctx->R;
    ctx->r_next = (int64_t)ctx->pair_base * 2 + ctx->R;
    ctx->batch_open = 0;
    return MPR_OK;
}

// Sweeps are queued in chunks of four; after each chunk the running count is
// copied to pinned memory, and the host checks the count of the chunk before
// the one it just queued, so the GPU never waits for the host. Sweeps queued
// after everything stopped find no running pair.
mpr_status mpr3_simulate(mpr3_ctx* ctx, int32_t n) {
    if (!ctx) return MPR_EINVAL;
    mpr_status st = mpr3_sim_begin(ctx, n);
    if (st != MPR_OK) return st;
    if (!ctx->h_run) {
        ctx->h_run = static_cast<unsigned long long*>(pinned_slot());
        if (!ctx->h_run) return fail3(ctx, MPR_ENOMEM, "pinned memory");
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail3(ctx, MPR_ECUDA, "cudaEventCreate failed");
    }
    int c = 0;
    while (st == MPR_OK && ctx->t < ctx->opt.n_max) {
        for (int i = 0; i < 4 && st == MPR_OK && ctx->t < ctx->opt.n_max; ++i) st = sweep3(ctx);
        if (st != MPR_OK) break;
        if (cudaMemcpyAsync(ctx->h_run + (c & 1), &ctx->ctl->n_running, sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, ctx->s) != cudaSuccess ||
            cudaEventRecord(ev[c & 1], ctx->s) != cudaSuccess) {
            st = fail3(ctx, MPR_ECUDA, "reading the running count failed");
            break;
        }
        if (c >= 1) {
            if (cudaEventSynchronize(ev[(c - 1) & 1]) != cudaSuccess) {
                st = fail3(ctx, MPR_ECUDA, "event synchronisation failed");
                break;
            }
            if (ctx->h_run[(c - 1) & 1] == 0) break;
        }
        ++c;
    }
    cudaStreamSynchronize(ctx->s);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (st == MPR_OK) st = mpr3_sim_end(ctx);
    return st;
}

mpr_status mpr3_get_state(mpr3_ctx* ctx, int32_t r, float* out) {
    if (!ctx || !out) return MPR_EINVAL;
    if (!ctx->batch_open || r < 0 || r >= ctx->R) return fail3(ctx, MPR_ESTATE, "no such realization");
    float* d = nullptr;
    TRY3(alloc3(ctx, &d, ctx->n));
    k3_get_state<<<grid_of(ctx->n), 256, 0, ctx->s>>>(ctx->g, ctx->ang, ctx->np, r, d);
    mpr_status st = cudaPeekAtLastError() == cudaSuccess ? MPR_OK : MPR_ECUDA;
    if (st == MPR_OK && (cudaMemcpyAsync(out, d, ctx->n * 4, cudaMemcpyDefault, ctx->s) ||
                         cudaStreamSynchronize(ctx->s)))
        st = MPR_ECUDA;
    free3(ctx, d);
    return st;
}

mpr_status mpr3_set_state(mpr3_ctx* ctx, int32_t r, const float* in) {
    if (!ctx || !in) return MPR_EINVAL;
    if (!ctx->batch_open || r < 0 || r >= ctx->R) return fail3(ctx, MPR_ESTATE, "no such realization");
    float* d = nullptr;
    TRY3(alloc3(ctx, &d, ctx->n));
    mpr_status st = MPR_OK;
    if (cudaMemcpyAsync(d, in, ctx->n * 4, cudaMemcpyDefault, ctx->s)) st = MPR_ECUDA;
    if (st == MPR_OK) {
        k3_set_state<<<grid_of(ctx->n), 256, 0, ctx->s>>>(ctx->g, ctx->mask, ctx->ang, ctx->np, r, d);
        if (cudaPeekAtLastError() || cudaStreamSynchronize(ctx->s)) st = MPR_ECUDA;
    }
    free3(ctx, d);
    return st;
}

mpr_status mpr3_predict(mpr3_ctx* ctx, float* out, const float* truth, double* aae_rase) {
    if (!ctx || !out) return MPR_EINVAL;
    ctx->err.clear();
    const int64_t gaps = ctx->n_gap[0] + ctx->n_gap[1];
    if (ctx->realizations == 0 && gaps > 0) return fail3(ctx, MPR_ESTATE, "no realization yet");
    float *o = nullptr, *tr = nullptr;
    TRY3(alloc3(ctx, &o, ctx->n));
    mpr_status st = MPR_OK;
    if (truth) {
        st = alloc3(ctx, &tr, ctx->n);
        if (st == MPR_OK && cudaMemcpyAsync(tr, truth, ctx->n * 4, cudaMemcpyDefault, ctx->s))
            st = MPR_ECUDA;
    }
    if (st == MPR_OK && cudaMemsetAsync(ctx->err_buf, 0, 16, ctx->s)) st = MPR_ECUDA;
    if (st == MPR_OK) {
        const double inv_r = ctx->realizations > 0 ? 1.0 / (double)ctx->realizations : 0.0;
        k3_predict<<<grid_of(ctx->n), 256, 0, ctx->s>>>(ctx->n, ctx->values, ctx->mask, ctx->sum,
                                                        inv_r, ctx->zmin, ctx->zmax, o, tr,
                                                        ctx->err_buf);
        double h[2] = {0, 0};
        if (cudaPeekAtLastError() ||
            cudaMemcpyAsync(out, o, ctx->n * 4, cudaMemcpyDefault, ctx->s) ||
            cudaMemcpyAsync(h, ctx->err_buf, 16, cudaMemcpyDeviceToHost, ctx->s) ||
            cudaStreamSynchronize(ctx->s))
            st = MPR_ECUDA;
        if (st == MPR_OK && truth && aae_rase) {
            aae_rase[0] = gaps ? h[0] / (double)gaps : 0.0;
            aae_rase[1] = gaps ? std::sqrt(h[1] / (double)gaps) : 0.0;
        }
    }
    free3(ctx, o);
    free3(ctx, tr);
    return st;
}

mpr_status mpr3_get_info(const mpr3_ctx* ctx, mpr3_info* info) {
    if (!ctx || !info) return MPR_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->depth = ctx->g.D;
    info->height = ctx->g.H;
    info->width = ctx->g.W;
    info->block = ctx->g.lb;
    info->nblk = ctx->g.nblk;
    info->n_gap = ctx->n_gap[0] + ctx->n_gap[1];
    info->zmin = ctx->zmin;
    info->zmax = ctx->zmax;
    info->realizations = ctx->realizations;
    info->gap_updates = ctx->gap_updates;
    info->cal_gap_updates = ctx->cal_updates;
    return MPR_OK;
}

}  // extern "C"
