// Device building blocks of the SV-MPR sweep: Philox4x32-10, the (0,1)
// uniform, and one Metropolis + over-relaxation update of a gap site.
#pragma once
#include <cstdint>

#include "mpr_internal.h"

namespace mpr {

constexpr float kTwoPi = 6.28318530717958647692f;

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies; the key advances by the Weyl constants between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t out[4]) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t pa = (uint64_t)0xD2511F53u * c0;
        const uint64_t pb = (uint64_t)0xCD9E8D57u * c2;
        c0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
        c1 = (uint32_t)pb;
        c2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
        c3 = (uint32_t)pa;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// The same generator with the round keys of key word 0 given (k0 + r W0 for
// r = 0 .. 9, taken from kernel parameters, where the XOR reads them
// directly); key word 1 advances in the loop.
__device__ __forceinline__ void philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 const uint32_t (&rk0)[10], uint32_t k1,
                                                 uint32_t out[4]) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t pa = (uint64_t)0xD2511F53u * c0;
        const uint64_t pb = (uint64_t)0xCD9E8D57u * c2;
        c0 = (uint32_t)(pb >> 32) ^ c1 ^ rk0[round];
        c1 = (uint32_t)pb;
        c2 = (uint32_t)(pa >> 32) ^ c3 ^ (k1 + (uint32_t)round * 0xBB67AE85u);
        c3 = (uint32_t)pa;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// (((x >> 8) | 1) * 2^-24): an odd multiple of 2^-24 in (0,1), exact in FP32
// and equal to the oracle's value. Built from the bits: f = 1 + (x >> 9) 2^-23
// is a float with mantissa x >> 9, and f - (1 - 2^-24) = (2 (x >> 9) + 1)
// 2^-24 has at most 24 significant bits, so the one subtraction is exact
// (1 - 2^-24 is itself a float, 0x3F7FFFFF).
__device__ __forceinline__ float u01(uint32_t x) {
    return __uint_as_float(0x3F800000u | (x >> 9)) - 0.999999940395355224609375f;
}

// psi = atan2(S, C) for S >= 0, psi in [0, pi]: atan(t) = t P(t^2) on
// t = min/max of (|C|, S) in [0, 1], then the octant is restored. P is a
// degree-7 near-minimax fit (gen_atan_poly.py; |error| < 7e-8 on [0, 1]).
__device__ __forceinline__ float atan2_upper(float S, float C) {
    const float ax = fabsf(C);
    const float mn = fminf(ax, S), mx = fmaxf(ax, S);
    const float t = __fdividef(mn, mx);
    const float z = t * t;
    float p = -4.054566845e-03f;
    p = fmaf(p, z, 2.186295763e-02f);
    p = fmaf(p, z, -5.591232702e-02f);
    p = fmaf(p, z, 9.642197192e-02f);
    p = fmaf(p, z, -1.390862912e-01f);
    p = fmaf(p, z, 1.994656622e-01f);
    p = fmaf(p, z, -3.332985938e-01f);
    p = fmaf(p, z, 9.999993443e-01f);
    float a = t * p;
    a = (S > ax) ? (1.57079632679489662f - a) : a;
    return (C < 0.0f) ? (3.14159265358979324f - a) : a;
}

// Outcome of one site update.
struct SiteNew {
    float phi;      // new angle
    float dE;       // energy change of the Metropolis move (0 when rejected)
    float co, so;   // cos, sin of q * old angle
    float ca, sa;   // cos, sin of q * angle after the Metropolis move
    bool refl;      // over-relaxation applied
};

// cos / sin of q times the final angle: after a reflection,
// q phi'' = 2 psi - q phi_a with cos 2psi = (C^2 - S^2)/R^2, sin 2psi = 2CS/R^2.
__device__ __forceinline__ void final_cs(const SiteNew& n, float C, float S, float& c, float& s) {
    if (n.refl) {
        const float ir2 = __fdividef(1.0f, C * C + S * S);
        const float c2 = (C * C - S * S) * ir2;
        const float s2 = 2.0f * C * S * ir2;
        c = c2 * n.ca + s2 * n.sa;
        s = s2 * n.ca - c2 * n.sa;
    } else {
        c = n.ca;
        s = n.sa;
    }
}

}  // namespace mpr
