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
        const uint32_t lo_a = 0xD2511F53u * c0;
        const uint32_t hi_a = __umulhi(0xD2511F53u, c0);
        const uint32_t lo_b = 0xCD9E8D57u * c2;
        const uint32_t hi_b = __umulhi(0xCD9E8D57u, c2);
        c0 = hi_b ^ c1 ^ k0;
        c1 = lo_b;
        c2 = hi_a ^ c3 ^ k1;
        c3 = lo_a;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// Odd multiple of 2^-24 in (0,1): exact in FP32, identical to the oracle's value.
__device__ __forceinline__ float u01(uint32_t x) {
    return __uint2float_rz((x >> 8) | 1u) * 5.9604644775390625e-08f;
}

// Result of one site update: new angle and (cos, sin) of q times it.
struct SiteNew {
    float phi, c, s;
};

// Metropolis with an independent uniform proposal on [0, 2pi] at inverse
// temperature beta, then (optionally) the restricted over-relaxation
// reflection of q*phi about psi = atan2(S, C), kept when it lands in
// [0, 2pi]. (C, S) is the neighbour field sum_j (cos q phi_j, sin q phi_j);
// the site energy is -J (C cos q phi + S sin q phi), so
// dE = J [(C co + S so) - (C cp + S sp)].
__device__ __forceinline__ SiteNew site_update(float phi, float C, float S, float u0, float u1,
                                               float beta, const Model& m) {
    float so, co, sp, cp;
    __sincosf(m.q * phi, &so, &co);
    const float php = kTwoPi * u0;
    __sincosf(m.q * php, &sp, &cp);
    const float dE = m.J * ((C * co + S * so) - (C * cp + S * sp));
    const bool acc = (dE <= 0.0f) || (u1 < __expf(-dE * beta));
    SiteNew n;
    n.phi = acc ? php : phi;
    n.c = acc ? cp : co;
    n.s = acc ? sp : so;
    if (m.overrelax && (C != 0.0f || S != 0.0f)) {
        const float psi = atan2f(S, C);
        const float por = (2.0f * psi - m.q * n.phi) * m.inv_q;
        if (por >= 0.0f && por <= kTwoPi) {
            // cos/sin of 2 psi from (C, S): no transcendental needed.
            const float r2 = C * C + S * S;
            const float ir2 = __fdividef(1.0f, r2);
            const float c2 = (C * C - S * S) * ir2;
            const float s2 = 2.0f * C * S * ir2;
            const float nc = c2 * n.c + s2 * n.s;
            const float ns = s2 * n.c - c2 * n.s;
            n.phi = por;
            n.c = nc;
            n.s = ns;
        }
    }
    return n;
}

}  // namespace mpr
