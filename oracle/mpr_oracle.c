/*
 * CPU oracle for SV-MPR gap filling (Lach & Zukovic, arXiv 2212.01317).
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow FP64 restatement of the method that
 * the CUDA library is checked against. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code with the CUDA
 * library; the two meet only in the seeded inputs they are given.
 *
 * Every function follows the paper's definitions in the paper's order, one
 * site or one bond at a time. Where the paper is silent the documented
 * readings are:
 *   - open (free) boundaries, 4-neighbour bonds, J = 1, q = 1/2 by default;
 *   - a site owns its right and down bonds and a bond belongs to the block
 *     of its owner (Sec. 2.2.2 "bond with two of its neighbors");
 *   - e_s,b = E_s,b / N_SP,b over owned sample-sample bonds (Eq. 2 read per
 *     bond, so both sides of the energy match are per-bond averages);
 *   - Metropolis with an independent uniform proposal on [0, 2pi], accept iff
 *     dE <= 0 or u1 < exp(-dE/T), followed by a restricted over-relaxation
 *     reflection about the local field direction, kept only when it lands in
 *     [0, 2pi];
 *   - random numbers from Philox4x32-10 with key (seed_lo, seed_hi ^ slice)
 *     and counter (site, sweep | tag << 16, realization >> 1, 0); realization
 *     r uses words 2(r&1) (proposal) and 2(r&1)+1 (acceptance);
 *   - local-equilibrium stop: a block stops at the first sweep t >= 1 at which
 *     its specific energy has reached its sample energy from the side it
 *     started on (Sec. 3.4 defers the exact test to the earlier MPR-GPU work);
 *   - calibration by per-block bisection on T, each iteration re-initialised.
 */
#include "mpr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI 6.283185307179586476925286766559

/* ---------------------------------------------------------------- model -- */

void orc_model_init(orc_model* m, int32_t H, int32_t W, int32_t lb, double q, double J,
                    uint64_t seed, uint32_t slice) {
    memset(m, 0, sizeof(*m));
    m->H = H;
    m->W = W;
    m->lb = lb;
    m->nbx = (W + lb - 1) / lb;
    m->nby = (H + lb - 1) / lb;
    m->nblk = m->nbx * m->nby;
    m->q = q;
    m->J = J;
    m->key0 = (uint32_t)(seed & 0xffffffffu);
    m->key1 = (uint32_t)(seed >> 32) ^ slice;
    m->overrelax = 1;
    m->K = 0;
    m->threads = 0;
    m->T_site = NULL;
    m->D = 1;
    m->nbz = 1;
    m->storage = 0;
    m->stop_rule = 0;
    m->n_fit = 20;
    m->n_f = 5;
}

/* ------------------------------------------------------- stored angles -- */
/* The precision form stores gap angles as BF16 (8 significant bits) or FP16
 * (11, with subnormals below 2^-14) and computes in FP32: a value is first
 * rounded to FP32, then to the stored type, each to the nearest
 * representable value with ties to the even one. */
static float bits_to_float(uint32_t u) {
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
}

static uint32_t float_to_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    return u;
}

/* Keep the top 32 - drop bits of the FP32 pattern, rounding the dropped part
 * to nearest, ties to even (exact while the exponent does not overflow). */
static float round_pattern(float f, int drop) {
    const uint32_t u = float_to_bits(f);
    const uint32_t half = (1u << (drop - 1)) - 1u;
    const uint32_t odd = (u >> drop) & 1u;
    return bits_to_float((u + half + odd) & ~((1u << drop) - 1u));
}

double orc_round_store(double v, int32_t storage) {
    if (storage == 0 || isnan(v)) return v;
    const float f = (float)v;
    if (storage == 1) return (double)round_pattern(f, 16);
    /* FP16: spacing 2^-24 below 2^-14 (subnormals), else 10 fraction bits. */
    if (fabsf(f) < 6.103515625e-05f) return (double)(nearbyintf(f * 16777216.0f) / 16777216.0f);
    return (double)round_pattern(f, 13);
}

static int block_of(const orc_model* m, int y, int x) { return (y / m->lb) * m->nbx + x / m->lb; }

/* ----------------------------------------------------------------- Philox -- */
/* Philox4x32-10 as defined by Salmon, Moraes, Dror & Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 products
 * with the round multipliers, the key advanced by the Weyl constants between
 * rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint64_t MA = 0xD2511F53u, MB = 0xCD9E8D57u;
    const uint32_t WA = 0x9E3779B9u, WB = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t pa = MA * (uint64_t)c0;
        uint64_t pb = MB * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)pb;
        uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)pa;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += WA;
        k1 += WB;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Top 24 bits with the lowest forced to 1, times 2^-24: an odd multiple of
 * 2^-24 in (0,1), exactly representable in FP32 and FP64. */
double orc_u01(uint32_t x) { return (double)((x >> 8) | 1u) * (1.0 / 16777216.0); }

void orc_site_uniforms(const orc_model* m, int64_t i, uint32_t t, uint32_t tag, uint32_t r,
                       double* u0, double* u1) {
    uint32_t ctr[4] = {(uint32_t)i, t | (tag << 16), r >> 1, 0u};
    uint32_t key[2] = {m->key0, m->key1};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    int o = (int)(r & 1u) * 2;
    *u0 = orc_u01(w[o]);
    *u1 = orc_u01(w[o + 1]);
}

/* -------------------------------------------------------------- transform -- */
/* Sec. 2.1: the data are mapped linearly onto spin angles in [0, 2pi]; the
 * extremes are taken over the samples (the only values known). */
int orc_transform(int64_t n, const float* values, const uint8_t* mask, double* zmin,
                  double* zmax, double* phi) {
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        if (mask[i]) continue;
        double v = (double)values[i];
        if (v < lo) lo = v;
        if (v > hi) hi = v;
    }
    *zmin = lo;
    *zmax = hi;
    int degenerate = !(hi > lo);
    for (int64_t i = 0; i < n; ++i) {
        if (mask[i]) { phi[i] = 0.0; continue; }
        phi[i] = degenerate ? 0.0 : TWO_PI * ((double)values[i] - lo) / (hi - lo);
    }
    return degenerate;
}

/* Sec. 2.1 / Sec. 3.2: prediction = back-transformed conditional mean; samples copied. */
void orc_backtransform(int64_t n, const double* mean_phi, const uint8_t* mask,
                       const float* values, double zmin, double zmax, float* out) {
    for (int64_t i = 0; i < n; ++i) {
        if (!mask[i]) { out[i] = values[i]; continue; }
        out[i] = (float)(zmin + (zmax - zmin) * mean_phi[i] / TWO_PI);
    }
}

/* ----------------------------------------------------------------- energy -- */
static double bond_energy(const orc_model* m, double a, double b) {
    return -m->J * cos(m->q * (a - b));
}

/* Eq. 2 applied per block: sample-sample bonds owned by the block, their count,
 * and every owned bond (N_b). Also the block's sample mean angle (Sec. 3.3.3). */
void orc_block_stats(const orc_model* m, const double* phi, const uint8_t* mask,
                     double* Es, int64_t* Nsp, int64_t* Nb, double* mean_angle,
                     int64_t* n_gap, int64_t* n_sample, double* global_mean) {
    const int H = m->H, W = m->W;
    double gsum = 0.0;
    int64_t gcnt = 0;
    for (int b = 0; b < m->nblk; ++b) {
        Es[b] = 0.0; Nsp[b] = 0; Nb[b] = 0; mean_angle[b] = 0.0; n_gap[b] = 0; n_sample[b] = 0;
    }
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            int64_t i = (int64_t)y * W + x;
            int b = block_of(m, y, x);
            if (mask[i]) {
                n_gap[b] += 1;
            } else {
                n_sample[b] += 1;
                mean_angle[b] += phi[i];
                gsum += phi[i];
                gcnt += 1;
            }
            /* right bond */
            if (x + 1 < W) {
                Nb[b] += 1;
                if (!mask[i] && !mask[i + 1]) {
                    Es[b] += bond_energy(m, phi[i], phi[i + 1]);
                    Nsp[b] += 1;
                }
            }
            /* down bond */
            if (y + 1 < H) {
                Nb[b] += 1;
                if (!mask[i] && !mask[i + W]) {
                    Es[b] += bond_energy(m, phi[i], phi[i + W]);
                    Nsp[b] += 1;
                }
            }
        }
    }
    for (int b = 0; b < m->nblk; ++b)
        if (n_sample[b] > 0) mean_angle[b] /= (double)n_sample[b];
    *global_mean = gcnt > 0 ? gsum / (double)gcnt : 0.0;
}

void orc_block_energy(const orc_model* m, const double* phi, double* E) {
    const int H = m->H, W = m->W, lb = m->lb;
    int nthreads = m->threads;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    for (int b = 0; b < m->nblk; ++b) {
        int by = b / m->nbx, bx = b % m->nbx;
        double s = 0.0;
        for (int y = by * lb; y < (by + 1) * lb && y < H; ++y) {
            for (int x = bx * lb; x < (bx + 1) * lb && x < W; ++x) {
                int64_t i = (int64_t)y * W + x;
                if (x + 1 < W) s += bond_energy(m, phi[i], phi[i + 1]);
                if (y + 1 < H) s += bond_energy(m, phi[i], phi[i + W]);
            }
        }
        E[b] = s;
    }
}

double orc_total_energy(const orc_model* m, const double* phi) {
    double s = 0.0;
    for (int y = 0; y < m->H; ++y)
        for (int x = 0; x < m->W; ++x) {
            int64_t i = (int64_t)y * m->W + x;
            if (x + 1 < m->W) s += bond_energy(m, phi[i], phi[i + 1]);
            if (y + 1 < m->H) s += bond_energy(m, phi[i], phi[i + m->W]);
        }
    return s;
}

/* ----------------------------------------------------------------- update -- */
/* One conditional MC update of gap site i (Sec. 2.1: only prediction sites move;
 * samples are fixed), at the temperature of its block (Sec. 2.2.2). */
/* Metropolis (+ over-relaxation) update of site i given its neighbours nb[nn]. */
static void update_core(const orc_model* m, double* phi, int64_t i, const int64_t* nb, int nn,
                        double T, uint32_t t, uint32_t tag, uint32_t r, orc_diag* d) {
    double u0, u1;
    orc_site_uniforms(m, i, t, tag, r, &u0, &u1);

    const double phi_old = phi[i];
    double phi_prop;
    if (m->K > 0) {
        int k = (int)floor((double)m->K * u0);
        if (k >= m->K) k = m->K - 1;
        phi_prop = TWO_PI * (double)k / (double)m->K;
    } else if (m->storage != 0) {
        /* Precision form: the FP32 product, rounded to the stored type. */
        const float prop32 = 6.28318530717958647692f * (float)u0;
        phi_prop = orc_round_store((double)prop32, m->storage);
    } else {
        phi_prop = TWO_PI * u0;
    }

    /* dE = H(after) - H(before), Eq. 1 restricted to the bonds of site i. */
    double dE = 0.0;
    for (int k = 0; k < nn; ++k) {
        double pj = phi[nb[k]];
        dE += -m->J * cos(m->q * (phi_prop - pj)) + m->J * cos(m->q * (phi_old - pj));
    }
    const double theta = -T * log(u1);
    int accepted = (dE <= 0.0) || (u1 < exp(-dE / T));
    double phi_new = accepted ? phi_prop : phi_old;

    /* Over-relaxation: reflect q*phi about the direction psi of the local
     * field sum_j (cos q phi_j, sin q phi_j); the site energy
     * -J (C cos q phi + S sin q phi) is unchanged. Kept only inside [0, 2pi]. */
    double phi_or = NAN, R = 0.0;
    int or_applied = 0;
    if (m->overrelax && m->K == 0) {
        double C = 0.0, S = 0.0;
        for (int k = 0; k < nn; ++k) {
            C += cos(m->q * phi[nb[k]]);
            S += sin(m->q * phi[nb[k]]);
        }
        R = sqrt(C * C + S * S);
        if (C != 0.0 || S != 0.0) {
            double psi = atan2(S, C);
            phi_or = (2.0 * psi - m->q * phi_new) / m->q;
            if (phi_or >= 0.0 && phi_or <= TWO_PI) {
                phi_new = orc_round_store(phi_or, m->storage);
                or_applied = 1;
            }
        }
    }
    phi[i] = phi_new;
    if (d) {
        d->dE = dE;
        d->theta = theta;
        d->phi_or = phi_or;
        d->R = R;
        d->phi_old = phi_old;
        d->phi_prop = phi_prop;
        d->accepted = accepted;
        d->or_applied = or_applied;
    }
}

void orc_update_site(const orc_model* m, double* phi, const uint8_t* mask, int64_t i,
                     double T, uint32_t t, uint32_t tag, uint32_t r, orc_diag* d) {
    (void)mask;
    const int W = m->W, H = m->H;
    const int y = (int)(i / W), x = (int)(i % W);
    int64_t nb[4];
    int nn = 0;
    if (x > 0) nb[nn++] = i - 1;
    if (x + 1 < W) nb[nn++] = i + 1;
    if (y > 0) nb[nn++] = i - W;
    if (y + 1 < H) nb[nn++] = i + W;
    update_core(m, phi, i, nb, nn, T, t, tag, r, d);
}

/* Sec. 2.2.2 single checkerboard: the sites of one sub-grid have all their
 * neighbours on the other, so one colour is updated at a time (here in raster
 * order; any order gives the same result). */
/* Sec. 2.2.3: smoothing of the block temperatures into site temperatures,
 * written out as the plain window mean (no separable or running-sum form). */
void orc_sst_temperatures(const orc_model* m, const double* T_blk, int32_t r_s, int32_t n_s,
                          double* T_site) {
    const int H = m->H, W = m->W;
    const int64_t n = (int64_t)H * W;
    double* tmp = (double*)malloc(sizeof(double) * (size_t)n);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) T_site[(int64_t)y * W + x] = T_blk[block_of(m, y, x)];
    const double inv = 1.0 / ((double)(2 * r_s + 1) * (double)(2 * r_s + 1));
    for (int pass = 0; pass < n_s; ++pass) {
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                double s = 0.0;
                for (int dy = -r_s; dy <= r_s; ++dy) {
                    int yy = y + dy;
                    yy = yy < 0 ? 0 : (yy >= H ? H - 1 : yy);
                    for (int dx = -r_s; dx <= r_s; ++dx) {
                        int xx = x + dx;
                        xx = xx < 0 ? 0 : (xx >= W ? W - 1 : xx);
                        s += T_site[(int64_t)yy * W + xx];
                    }
                }
                tmp[(int64_t)y * W + x] = s * inv;
            }
        for (int64_t i = 0; i < n; ++i) T_site[i] = tmp[i];
    }
    free(tmp);
}

void orc_halfstep(const orc_model* m, double* phi, const uint8_t* mask, int colour,
                  const double* T_blk, const uint8_t* active, uint32_t t, uint32_t tag,
                  uint32_t r, orc_diag* diag) {
    const int H = m->H, W = m->W;
    int nthreads = m->threads;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    for (int y = 0; y < H; ++y) {
        for (int x = (y + colour) & 1; x < W; x += 2) {
            int64_t i = (int64_t)y * W + x;
            if (!mask[i]) continue;
            int b = block_of(m, y, x);
            if (active && !active[b]) continue;
            const double T = m->T_site ? m->T_site[i] : T_blk[b];
            orc_update_site(m, phi, mask, i, T, t, tag, r, diag ? &diag[i] : NULL);
        }
    }
}

/* ------------------------------------------------------------------- init -- */
void orc_init_block_mean(const orc_model* m, double* phi, const uint8_t* mask,
                         const double* mean_angle, const int64_t* n_sample, double global_mean) {
    for (int y = 0; y < m->H; ++y)
        for (int x = 0; x < m->W; ++x) {
            int64_t i = (int64_t)y * m->W + x;
            if (!mask[i]) continue;
            int b = block_of(m, y, x);
            phi[i] = n_sample[b] > 0 ? mean_angle[b] : global_mean;
        }
}

void orc_init_random(const orc_model* m, double* phi, const uint8_t* mask, uint32_t r) {
    for (int64_t i = 0; i < (int64_t)m->H * m->W; ++i) {
        if (!mask[i]) continue;
        double u0, u1;
        orc_site_uniforms(m, i, 0u, 0xFFFFu, r, &u0, &u1);
        phi[i] = TWO_PI * u0;
    }
}

/* ------------------------------------------------------------------- stop -- */
/* t = 0 bookkeeping: a block without gap sites has nothing to simulate and is
 * stopped; sigma_b records from which side e_b starts relative to e_s,b. */
void orc_stop_init(const orc_model* m, const double* E0, const double* Es, const int64_t* Nsp,
                   const int64_t* Nb, const int64_t* n_gap, int8_t* sigma, uint8_t* active,
                   int32_t* stop_sweep) {
    int targeted_active = 0;
    for (int b = 0; b < m->nblk; ++b) {
        sigma[b] = 0;
        active[b] = n_gap[b] > 0;
        stop_sweep[b] = active[b] ? -1 : 0;
        if (Nsp[b] > 0) {
            double es = Es[b] / (double)Nsp[b];
            double e0 = E0[b] / (double)Nb[b];
            sigma[b] = (int8_t)((es > e0) - (es < e0));
            if (active[b]) targeted_active = 1;
        }
    }
    if (!targeted_active)
        for (int b = 0; b < m->nblk; ++b)
            if (active[b]) { active[b] = 0; stop_sweep[b] = 0; }
}

/* After sweep t: a targeted block stops once sigma_b (e_b(t) - e_s,b) >= 0; a
 * block without sample bonds stops when no targeted block is left running;
 * every block stops at t = n_max. Returns the number of blocks still active. */
int orc_stop_update(const orc_model* m, int32_t t, int32_t n_max, const double* E,
                    const double* Es, const int64_t* Nsp, const int64_t* Nb, const int8_t* sigma,
                    uint8_t* active, int32_t* stop_sweep) {
    int targeted_active = 0;
    for (int b = 0; b < m->nblk; ++b) {
        if (!active[b] || Nsp[b] == 0) continue;
        double es = Es[b] / (double)Nsp[b];
        double e = E[b] / (double)Nb[b];
        if ((double)sigma[b] * (e - es) >= 0.0) {
            active[b] = 0;
            stop_sweep[b] = t;
        } else {
            targeted_active = 1;
        }
    }
    int left = 0;
    for (int b = 0; b < m->nblk; ++b) {
        if (!active[b]) continue;
        if ((Nsp[b] == 0 && !targeted_active) || t >= n_max) {
            active[b] = 0;
            stop_sweep[b] = t;
        } else {
            left += 1;
        }
    }
    return left;
}

double orc_window_slope(const orc_model* m, int32_t t, const double* hist, int b) {
    double num = 0.0;
    for (int j = 0; j < m->n_fit; ++j) {
        const int32_t s = t - m->n_fit + 1 + j;
        num += (double)(2 * j - (m->n_fit - 1)) * hist[(int64_t)(s % m->n_fit) * m->nblk + b];
    }
    return num;
}

int orc_stop_update_window(const orc_model* m, int32_t t, int32_t n_max, const double* Es,
                           const int64_t* Nsp, const int8_t* sigma, const double* hist,
                           uint8_t* active, int32_t* stop_sweep) {
    const int32_t first = m->n_fit + m->n_f;
    const int test = t >= first && (t - first) % m->n_f == 0;
    int targeted_active = 0;
    for (int b = 0; b < m->nblk; ++b) {
        if (!active[b] || Nsp[b] == 0) continue;
        int stop = 0;
        if (test) {
            const double num = orc_window_slope(m, t, hist, b);
            stop = (double)sigma[b] * num <= 0.0;
        }
        if (stop) {
            active[b] = 0;
            stop_sweep[b] = t;
        } else {
            targeted_active = 1;
        }
    }
    (void)Es;
    int left = 0;
    for (int b = 0; b < m->nblk; ++b) {
        if (!active[b]) continue;
        if ((Nsp[b] == 0 && !targeted_active) || t >= n_max) {
            active[b] = 0;
            stop_sweep[b] = t;
        } else {
            left += 1;
        }
    }
    return left;
}

int orc_simulate_one(const orc_model* m, double* phi, const uint8_t* mask, const double* T_blk,
                     const double* Es, const int64_t* Nsp, const int64_t* Nb,
                     const int64_t* n_gap, int32_t n_max, uint32_t r, int32_t* stop_sweep,
                     double* e_trace) {
    const int nblk = m->nblk;
    double* E = (double*)malloc(sizeof(double) * nblk);
    int8_t* sigma = (int8_t*)malloc(nblk);
    uint8_t* active = (uint8_t*)malloc(nblk);
    double* hist = m->stop_rule == 1 ? (double*)malloc(sizeof(double) * nblk * m->n_fit) : NULL;
    orc_block_energy(m, phi, E);
    if (e_trace)
        for (int b = 0; b < nblk; ++b) e_trace[b] = Nb[b] > 0 ? E[b] / (double)Nb[b] : 0.0;
    orc_stop_init(m, E, Es, Nsp, Nb, n_gap, sigma, active, stop_sweep);
    int left = 0;
    for (int b = 0; b < nblk; ++b) left += active[b];
    int t = 0;
    while (left > 0 && t < n_max) {
        t += 1;
        orc_halfstep(m, phi, mask, 0, T_blk, active, (uint32_t)t, 0u, r, NULL);
        orc_halfstep(m, phi, mask, 1, T_blk, active, (uint32_t)t, 0u, r, NULL);
        orc_block_energy(m, phi, E);
        if (e_trace)
            for (int b = 0; b < nblk; ++b)
                e_trace[(int64_t)t * nblk + b] = Nb[b] > 0 ? E[b] / (double)Nb[b] : 0.0;
        if (hist) {
            for (int b = 0; b < nblk; ++b)
                hist[(int64_t)(t % m->n_fit) * nblk + b] = Nb[b] > 0 ? E[b] / (double)Nb[b] : 0.0;
            left = orc_stop_update_window(m, t, n_max, Es, Nsp, sigma, hist, active, stop_sweep);
        } else {
            left = orc_stop_update(m, t, n_max, E, Es, Nsp, Nb, sigma, active, stop_sweep);
        }
    }
    free(E);
    free(sigma);
    free(active);
    free(hist);
    return t;
}

/* The sampling variant of the conditional mean (Sec. 2.1 predicts with the
 * mean of the conditional distribution): instead of independent realizations
 * each stopped at local equilibrium, one chain from phi (the block-mean
 * start) runs n_equil sweeps with every block active, then n_samples further
 * sweeps, and its state after each of those is one sample: sum[i] += phi_i
 * at every gap site. Realization index r, tag 0, sweeps t = 1, 2, ... */
void orc_sample_chain(const orc_model* m, double* phi, const uint8_t* mask, const double* T_blk,
                      int32_t n_equil, int32_t n_samples, uint32_t r, double* sum) {
    const int64_t n = (int64_t)m->H * m->W;
    for (int t = 1; t <= n_equil + n_samples; ++t) {
        orc_halfstep(m, phi, mask, 0, T_blk, NULL, (uint32_t)t, 0u, r, NULL);
        orc_halfstep(m, phi, mask, 1, T_blk, NULL, (uint32_t)t, 0u, r, NULL);
        if (t <= n_equil) continue;
        for (int64_t i = 0; i < n; ++i)
            if (mask[i]) sum[i] += phi[i];
    }
}

/* ------------------------------------------------------------ calibration -- */
static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Median of the targeted blocks' temperatures: the middle element for an odd
 * count, the mean of the two middle elements for an even count. */
double orc_median_targeted(int32_t nblk, const double* T, const int64_t* Nsp) {
    double* v = (double*)malloc(sizeof(double) * (nblk > 0 ? nblk : 1));
    int n = 0;
    for (int b = 0; b < nblk; ++b)
        if (Nsp[b] > 0) v[n++] = T[b];
    double med = 0.0;
    if (n > 0) {
        qsort(v, (size_t)n, sizeof(double), cmp_double);
        med = (n & 1) ? v[n / 2] : 0.5 * (v[n / 2 - 1] + v[n / 2]);
    }
    free(v);
    return med;
}

/* Sec. 2.1 estimates T by matching the simulated specific energy with e_s;
 * Sec. 2.2.2 does this per block. Each bisection iteration k: every targeted
 * block takes the midpoint of its bracket, blocks without sample bonds take
 * the median of those midpoints; the initialised state is equilibrated for
 * n_eq sweeps and e_b is averaged over n_meas further sweeps (and over the
 * chains); then the bracket half on the wrong side of e_s,b is dropped
 * (<e_b> increases with T). Random numbers use tag 1 + k. */
/* Blocks that calibrate: those with sample bonds (a target e_s,b) and gap
 * sites (whose temperature the method uses). A block with sample bonds but
 * no gap site has e_b = e_s,b exactly and nothing to fill; like a block
 * without sample bonds it takes the median of the calibrating blocks' T and
 * does not count towards it. Returns Nsp with the others set to 0. */
static int64_t* calib_targets(const orc_model* m, const uint8_t* mask, const int64_t* Nsp,
                              int three_d) {
    int64_t* t = (int64_t*)calloc((size_t)m->nblk, sizeof(int64_t));
    const int D = three_d ? m->D : 1;
    for (int z = 0; z < D; ++z)
        for (int y = 0; y < m->H; ++y)
            for (int x = 0; x < m->W; ++x) {
                const int64_t i = ((int64_t)z * m->H + y) * m->W + x;
                if (!mask[i]) continue;
                const int b = ((z / m->lb) * m->nby + y / m->lb) * m->nbx + x / m->lb;
                t[b] = 1;
            }
    for (int b = 0; b < m->nblk; ++b) t[b] = t[b] ? Nsp[b] : 0;
    return t;
}

void orc_calibrate(const orc_model* m, const double* phi_init, const uint8_t* mask,
                   const double* Es, const int64_t* Nsp_all, const int64_t* Nb, int32_t n_eq,
                   int32_t n_meas, int32_t n_bisect, int32_t chains, double T_lo, double T_hi,
                   double* T_out, double* ebar_trace) {
    int64_t* Nsp = calib_targets(m, mask, Nsp_all, 0);
    const int nblk = m->nblk;
    const int64_t n = (int64_t)m->H * m->W;
    double* lo = (double*)malloc(sizeof(double) * nblk);
    double* hi = (double*)malloc(sizeof(double) * nblk);
    double* T = (double*)malloc(sizeof(double) * nblk);
    double* ebar = (double*)malloc(sizeof(double) * nblk);
    double* E = (double*)malloc(sizeof(double) * nblk);
    double* phi = (double*)malloc(sizeof(double) * n);
    for (int b = 0; b < nblk; ++b) { lo[b] = T_lo; hi[b] = T_hi; }
    for (int k = 0; k < n_bisect; ++k) {
        for (int b = 0; b < nblk; ++b) T[b] = 0.5 * (lo[b] + hi[b]);
        double med = orc_median_targeted(nblk, T, Nsp);
        for (int b = 0; b < nblk; ++b) {
            if (Nsp[b] == 0) T[b] = med;
            ebar[b] = 0.0;
        }
        for (int c = 0; c < chains; ++c) {
            memcpy(phi, phi_init, sizeof(double) * n);
            for (int s = 1; s <= n_eq + n_meas; ++s) {
                orc_halfstep(m, phi, mask, 0, T, NULL, (uint32_t)s, (uint32_t)(1 + k), (uint32_t)c, NULL);
                orc_halfstep(m, phi, mask, 1, T, NULL, (uint32_t)s, (uint32_t)(1 + k), (uint32_t)c, NULL);
                if (s > n_eq) {
                    orc_block_energy(m, phi, E);
                    for (int b = 0; b < nblk; ++b)
                        if (Nb[b] > 0) ebar[b] += E[b] / (double)Nb[b];
                }
            }
        }
        for (int b = 0; b < nblk; ++b) {
            ebar[b] /= (double)n_meas * (double)chains;
            if (ebar_trace) ebar_trace[(int64_t)k * nblk + b] = ebar[b];
            if (Nsp[b] == 0) continue;
            double es = Es[b] / (double)Nsp[b];
            if (ebar[b] < es) lo[b] = T[b]; else hi[b] = T[b];
        }
    }
    for (int b = 0; b < nblk; ++b) T_out[b] = 0.5 * (lo[b] + hi[b]);
    double med = orc_median_targeted(nblk, T_out, Nsp);
    for (int b = 0; b < nblk; ++b)
        if (Nsp[b] == 0) T_out[b] = med;
    free(lo); free(hi); free(T); free(ebar); free(E); free(phi);
    free(Nsp);
}

/* ----------------------------------------------------------------- scores -- */
void orc_calibrate_points(const orc_model* m, const double* phi_init, const uint8_t* mask,
                          const double* Es, const int64_t* Nsp_all, const int64_t* Nb, int32_t n_eq,
                          int32_t n_meas, int32_t n_iter, int32_t chains, int32_t points,
                          double T_lo, double T_hi, const double* T0_warm, double warm,
                          int32_t n_eq_next, double* T_out, double* ebar_trace,
                          double* pts_trace) {
    int64_t* Nsp = calib_targets(m, mask, Nsp_all, 0);
    const int nblk = m->nblk;
    const int64_t n = (int64_t)m->H * m->W;
    /* continued chains: one state per (chain, point), kept across iterations */
    const int keep = n_eq_next >= 0;
    double* states = keep ? (double*)malloc(sizeof(double) * n * (size_t)chains * points) : NULL;
    double* lo = (double*)malloc(sizeof(double) * nblk);
    double* hi = (double*)malloc(sizeof(double) * nblk);
    double* T = (double*)malloc(sizeof(double) * nblk * (size_t)points);
    double* ebar = (double*)malloc(sizeof(double) * nblk * (size_t)points);
    double* E = (double*)malloc(sizeof(double) * nblk);
    double* phi = (double*)malloc(sizeof(double) * n);
    for (int b = 0; b < nblk; ++b) { lo[b] = T_lo; hi[b] = T_hi; }
    for (int k = 0; k < n_iter; ++k) {
        for (int p = 0; p < points; ++p) {
            double* Tp = T + (int64_t)p * nblk;
            for (int b = 0; b < nblk; ++b) {
                if (k == 0 && T0_warm && points > 1) {
                    /* warm start: the points evenly spaced on [T0 / w, T0 w] */
                    const double a = T0_warm[b] / warm, c = T0_warm[b] * warm;
                    Tp[b] = a + (double)p * (c - a) / (double)(points - 1);
                } else {
                    Tp[b] = lo[b] + (double)(p + 1) * (hi[b] - lo[b]) / (double)(points + 1);
                }
            }
            const double med = orc_median_targeted(nblk, Tp, Nsp);
            for (int b = 0; b < nblk; ++b) {
                if (Nsp[b] == 0) Tp[b] = med;
                ebar[(int64_t)p * nblk + b] = 0.0;
            }
        }
        for (int c = 0; c < chains; ++c)
            for (int p = 0; p < points; ++p) {
                const double* Tp = T + (int64_t)p * nblk;
                const uint32_t r = (uint32_t)(c * points + p);
                double* ph = keep ? states + (int64_t)r * n : phi;
                if (!keep || k == 0) memcpy(ph, phi_init, sizeof(double) * n);
                const int neq = (keep && k > 0) ? n_eq_next : n_eq;
                for (int s = 1; s <= neq + n_meas; ++s) {
                    orc_halfstep(m, ph, mask, 0, Tp, NULL, (uint32_t)s, (uint32_t)(1 + k), r, NULL);
                    orc_halfstep(m, ph, mask, 1, Tp, NULL, (uint32_t)s, (uint32_t)(1 + k), r, NULL);
                    if (s <= neq) continue;
                    orc_block_energy(m, ph, E);
                    for (int b = 0; b < nblk; ++b)
                        if (Nb[b] > 0) ebar[(int64_t)p * nblk + b] += E[b] / (double)Nb[b];
                }
            }
        for (int b = 0; b < nblk; ++b) {
            if (Nsp[b] == 0) continue;
            const double es = Es[b] / (double)Nsp[b];
            double nlo = lo[b], nhi = hi[b];
            for (int p = 0; p < points; ++p) {
                const double e = ebar[(int64_t)p * nblk + b] / ((double)n_meas * (double)chains);
                const double tp = T[(int64_t)p * nblk + b];
                const int64_t at = ((int64_t)k * points + p) * nblk + b;
                if (ebar_trace) ebar_trace[at] = e;
                if (pts_trace) pts_trace[at] = tp;
                if (e < es) { if (tp > nlo) nlo = tp; }
                else if (tp < nhi) nhi = tp;
            }
            if (nlo > nhi) {   /* the means crossed on noise: keep the points' span */
                nlo = T[b];
                nhi = T[(int64_t)(points - 1) * nblk + b];
            }
            lo[b] = nlo;
            hi[b] = nhi;
        }
    }
    for (int b = 0; b < nblk; ++b) T_out[b] = 0.5 * (lo[b] + hi[b]);
    const double med = orc_median_targeted(nblk, T_out, Nsp);
    for (int b = 0; b < nblk; ++b)
        if (Nsp[b] == 0) T_out[b] = med;
    free(lo); free(hi); free(T); free(ebar); free(E); free(phi); free(states);
    free(Nsp);
}

/* ------------------------------------------ unconditional e(T) curve -- */

/* Specific energy of the data-free lattice: plain MPR matches e_s against the
 * equilibrium energy of the whole grid (Sec. 2.1); with no data at all that
 * energy is a function of T alone, the unconditional curve e(T). Here it is
 * measured the way the calibration measures a block: an L x L lattice of gap
 * sites (open boundaries), every angle started at pi (the middle of the
 * range: a data-free stand-in for the block-mean start), n_eq sweeps, then
 * E / N_bonds (N_bonds = 2 L (L - 1)) averaged over n_meas sweeps.
 * Temperature k runs as realization k with tag 0xFFFE (key: seed, slice 0);
 * overrelax as in the model (1: Metropolis then the reflection). */
void orc_energy_curve(double q, double J, uint64_t seed, int32_t overrelax, int32_t L, int32_t n_T,
                      const double* T, int32_t n_eq, int32_t n_meas, double* e_out) {
    orc_model lm;
    orc_model_init(&lm, L, L, L, q, J, seed, 0u);
    lm.overrelax = overrelax;
    const int64_t n = (int64_t)L * L;
    const double n_bonds = 2.0 * (double)L * (double)(L - 1);
    double* phi = (double*)malloc(sizeof(double) * n);
    uint8_t* mask = (uint8_t*)malloc((size_t)n);
    memset(mask, 1, (size_t)n);
    for (int k = 0; k < n_T; ++k) {
        const double Tk[1] = {T[k]};
        for (int64_t i = 0; i < n; ++i) phi[i] = 0.5 * TWO_PI;
        double acc = 0.0;
        for (int s = 1; s <= n_eq + n_meas; ++s) {
            orc_halfstep(&lm, phi, mask, 0, Tk, NULL, (uint32_t)s, 0xFFFEu, (uint32_t)k, NULL);
            orc_halfstep(&lm, phi, mask, 1, Tk, NULL, (uint32_t)s, 0xFFFEu, (uint32_t)k, NULL);
            if (s > n_eq) acc += orc_total_energy(&lm, phi) / n_bonds;
        }
        e_out[k] = n_meas > 0 ? acc / (double)n_meas : 0.0;
    }
    free(phi);
    free(mask);
}

/* The temperature at which the curve reaches e_s. The curve is first made
 * non-decreasing (each value raised to the largest one before it: Monte Carlo
 * noise can make neighbouring points cross, while <e> grows with T), then read
 * by linear interpolation between the two points around e_s; clamped to the
 * first and last temperature. */
double orc_curve_T0(int32_t n, const double* T, const double* e, double e_s) {
    double prev = e[0];
    if (!(e_s > prev)) return T[0];
    for (int k = 1; k < n; ++k) {
        const double ek = e[k] > prev ? e[k] : prev;
        if (e_s <= ek) {
            const double f = (e_s - prev) / (ek - prev);
            return T[k - 1] + (T[k] - T[k - 1]) * f;
        }
        prev = ek;
    }
    return T[n - 1];
}

/* --------------------------------------------- moments and Newton (f1) -- */

void orc_energy_moments(const orc_model* m, double* phi, const uint8_t* mask, const double* T,
                        int32_t n_eq, int32_t n_meas, int32_t chains, uint32_t tag,
                        const int64_t* Nb, double* mean_e, double* var_E, double* cov_r,
                        double* cov_d) {
    const int nblk = m->nblk, nbx = m->nbx;
    const int64_t n = (int64_t)m->H * m->W;
    double* E = (double*)malloc(sizeof(double) * nblk);
    double* s1 = (double*)calloc((size_t)nblk, sizeof(double));
    double* s2 = (double*)calloc((size_t)nblk, sizeof(double));
    double* sr = (double*)calloc((size_t)nblk, sizeof(double));
    double* sd = (double*)calloc((size_t)nblk, sizeof(double));
    for (int c = 0; c < chains; ++c) {
        double* ph = phi + (int64_t)c * n;
        for (int s = 1; s <= n_eq + n_meas; ++s) {
            orc_halfstep(m, ph, mask, 0, T, NULL, (uint32_t)s, tag, (uint32_t)c, NULL);
            orc_halfstep(m, ph, mask, 1, T, NULL, (uint32_t)s, tag, (uint32_t)c, NULL);
            if (s <= n_eq) continue;
            orc_block_energy(m, ph, E);
            for (int b = 0; b < nblk; ++b) {
                s1[b] += E[b];
                s2[b] += E[b] * E[b];
                if (b % nbx != nbx - 1) sr[b] += E[b] * E[b + 1];
                if (b + nbx < nblk) sd[b] += E[b] * E[b + nbx];
            }
        }
    }
    const double inv = 1.0 / ((double)n_meas * (double)chains);
    for (int b = 0; b < nblk; ++b) {
        const double m1 = s1[b] * inv;
        if (mean_e) mean_e[b] = Nb[b] > 0 ? m1 / (double)Nb[b] : 0.0;
        if (var_E) var_E[b] = s2[b] * inv - m1 * m1;
        if (cov_r) cov_r[b] = (b % nbx != nbx - 1) ? sr[b] * inv - m1 * s1[b + 1] * inv : 0.0;
        if (cov_d) cov_d[b] = (b + nbx < nblk) ? sd[b] * inv - m1 * s1[b + nbx] * inv : 0.0;
    }
    free(E); free(s1); free(s2); free(sr); free(sd);
}

#define NEWTON_STEP 2.0   /* largest factor by which one Newton step moves T */

void orc_calibrate_newton(const orc_model* m, const double* phi_init, const uint8_t* mask,
                          const double* Es, const int64_t* Nsp_all, const int64_t* Nb, int32_t n_eq,
                          int32_t n_meas, int32_t n_newton, int32_t chains, double T_lo,
                          double T_hi, double T0, double* T_out, double* trace) {
    int64_t* Nsp = calib_targets(m, mask, Nsp_all, 0);
    const int nblk = m->nblk;
    const int64_t n = (int64_t)m->H * m->W;
    double* T = (double*)malloc(sizeof(double) * nblk);
    double* y = (double*)malloc(sizeof(double) * nblk);
    double* v = (double*)malloc(sizeof(double) * nblk);
    double* phi = (double*)malloc(sizeof(double) * n * (size_t)chains);
    for (int c = 0; c < chains; ++c) memcpy(phi + (int64_t)c * n, phi_init, sizeof(double) * n);
    for (int b = 0; b < nblk; ++b) T[b] = T0;
    for (int k = 0; k < n_newton; ++k) {
        const double med = orc_median_targeted(nblk, T, Nsp);
        for (int b = 0; b < nblk; ++b)
            if (Nsp[b] == 0) T[b] = med;
        if (trace) memcpy(trace + (int64_t)k * nblk, T, sizeof(double) * nblk);
        orc_energy_moments(m, phi, mask, T, n_eq, n_meas, chains, (uint32_t)(1 + k), Nb, y, v,
                           NULL, NULL);
        for (int b = 0; b < nblk; ++b) {
            if (Nsp[b] == 0) continue;
            const double es = Es[b] / (double)Nsp[b];
            double tn;
            if (v[b] > 0.0) {
                const double bn = 1.0 / T[b] + (y[b] - es) * (double)Nb[b] / v[b];
                tn = bn > 0.0 ? 1.0 / bn : NEWTON_STEP * T[b];
            } else {
                tn = y[b] < es ? NEWTON_STEP * T[b] : T[b] / NEWTON_STEP;
            }
            tn = tn < T[b] / NEWTON_STEP ? T[b] / NEWTON_STEP
                                         : (tn > NEWTON_STEP * T[b] ? NEWTON_STEP * T[b] : tn);
            T[b] = tn < T_lo ? T_lo : (tn > T_hi ? T_hi : tn);
        }
    }
    const double med = orc_median_targeted(nblk, T, Nsp);
    for (int b = 0; b < nblk; ++b) T_out[b] = Nsp[b] == 0 ? med : T[b];
    free(T); free(y); free(v); free(phi);
    free(Nsp);
}

/* ------------------------------------------------------------- 3-D -- */

void orc3_model_init(orc_model* m, int32_t D, int32_t H, int32_t W, int32_t lb, double q,
                     double J, uint64_t seed, uint32_t slice) {
    orc_model_init(m, H, W, lb, q, J, seed, slice);
    m->D = D;
    m->nbz = (D + lb - 1) / lb;
    m->nblk = m->nbx * m->nby * m->nbz;
}

static int block3(const orc_model* m, int z, int y, int x) {
    return ((z / m->lb) * m->nby + y / m->lb) * m->nbx + x / m->lb;
}

void orc3_block_stats(const orc_model* m, const double* phi, const uint8_t* mask, double* Es,
                      int64_t* Nsp, int64_t* Nb, double* mean_angle, int64_t* n_gap,
                      int64_t* n_sample, double* global_mean) {
    const int D = m->D, H = m->H, W = m->W;
    const int64_t HW = (int64_t)H * W;
    double gsum = 0.0;
    int64_t gcnt = 0;
    for (int b = 0; b < m->nblk; ++b) {
        Es[b] = 0.0; Nsp[b] = 0; Nb[b] = 0; mean_angle[b] = 0.0; n_gap[b] = 0; n_sample[b] = 0;
    }
    for (int z = 0; z < D; ++z)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const int64_t i = (int64_t)z * HW + (int64_t)y * W + x;
                const int b = block3(m, z, y, x);
                if (mask[i]) {
                    n_gap[b] += 1;
                } else {
                    n_sample[b] += 1;
                    mean_angle[b] += phi[i];
                    gsum += phi[i];
                    gcnt += 1;
                }
                const int64_t nb[3] = {x + 1 < W ? i + 1 : -1, y + 1 < H ? i + W : -1,
                                       z + 1 < D ? i + HW : -1};
                for (int k = 0; k < 3; ++k) {
                    if (nb[k] < 0) continue;
                    Nb[b] += 1;
                    if (!mask[i] && !mask[nb[k]]) {
                        Es[b] += bond_energy(m, phi[i], phi[nb[k]]);
                        Nsp[b] += 1;
                    }
                }
            }
    for (int b = 0; b < m->nblk; ++b)
        if (n_sample[b] > 0) mean_angle[b] /= (double)n_sample[b];
    *global_mean = gcnt > 0 ? gsum / (double)gcnt : 0.0;
}

void orc3_block_energy(const orc_model* m, const double* phi, double* E) {
    const int D = m->D, H = m->H, W = m->W;
    const int64_t HW = (int64_t)H * W;
    for (int b = 0; b < m->nblk; ++b) E[b] = 0.0;
    for (int z = 0; z < D; ++z)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const int64_t i = (int64_t)z * HW + (int64_t)y * W + x;
                const int b = block3(m, z, y, x);
                if (x + 1 < W) E[b] += bond_energy(m, phi[i], phi[i + 1]);
                if (y + 1 < H) E[b] += bond_energy(m, phi[i], phi[i + W]);
                if (z + 1 < D) E[b] += bond_energy(m, phi[i], phi[i + HW]);
            }
}

void orc3_update_site(const orc_model* m, double* phi, const uint8_t* mask, int64_t i, double T,
                      uint32_t t, uint32_t tag, uint32_t r, orc_diag* d) {
    (void)mask;
    const int D = m->D, H = m->H, W = m->W;
    const int64_t HW = (int64_t)H * W;
    const int z = (int)(i / HW), y = (int)((i % HW) / W), x = (int)(i % W);
    int64_t nb[6];
    int nn = 0;
    if (x > 0) nb[nn++] = i - 1;
    if (x + 1 < W) nb[nn++] = i + 1;
    if (y > 0) nb[nn++] = i - W;
    if (y + 1 < H) nb[nn++] = i + W;
    if (z > 0) nb[nn++] = i - HW;
    if (z + 1 < D) nb[nn++] = i + HW;
    update_core(m, phi, i, nb, nn, T, t, tag, r, d);
}

void orc3_halfstep(const orc_model* m, double* phi, const uint8_t* mask, int colour,
                   const double* T_blk, const uint8_t* active, uint32_t t, uint32_t tag,
                   uint32_t r, orc_diag* diag) {
    const int D = m->D, H = m->H, W = m->W;
    const int64_t HW = (int64_t)H * W;
    for (int z = 0; z < D; ++z)
        for (int y = 0; y < H; ++y)
            for (int x = (y + z + colour) & 1; x < W; x += 2) {
                const int64_t i = (int64_t)z * HW + (int64_t)y * W + x;
                if (!mask[i]) continue;
                const int b = block3(m, z, y, x);
                if (active && !active[b]) continue;
                orc3_update_site(m, phi, mask, i, T_blk[b], t, tag, r, diag ? &diag[i] : NULL);
            }
}

void orc3_init_block_mean(const orc_model* m, double* phi, const uint8_t* mask,
                          const double* mean_angle, const int64_t* n_sample, double global_mean) {
    const int64_t HW = (int64_t)m->H * m->W;
    for (int z = 0; z < m->D; ++z)
        for (int y = 0; y < m->H; ++y)
            for (int x = 0; x < m->W; ++x) {
                const int64_t i = (int64_t)z * HW + (int64_t)y * m->W + x;
                if (!mask[i]) continue;
                const int b = block3(m, z, y, x);
                phi[i] = n_sample[b] > 0 ? mean_angle[b] : global_mean;
            }
}

int orc3_simulate_one(const orc_model* m, double* phi, const uint8_t* mask, const double* T_blk,
                      const double* Es, const int64_t* Nsp, const int64_t* Nb,
                      const int64_t* n_gap, int32_t n_max, uint32_t r, int32_t* stop_sweep,
                      double* e_trace) {
    const int nblk = m->nblk;
    double* E = (double*)malloc(sizeof(double) * nblk);
    int8_t* sigma = (int8_t*)malloc(nblk);
    uint8_t* active = (uint8_t*)malloc(nblk);
    orc3_block_energy(m, phi, E);
    if (e_trace)
        for (int b = 0; b < nblk; ++b) e_trace[b] = Nb[b] > 0 ? E[b] / (double)Nb[b] : 0.0;
    orc_stop_init(m, E, Es, Nsp, Nb, n_gap, sigma, active, stop_sweep);
    int left = 0;
    for (int b = 0; b < nblk; ++b) left += active[b];
    int t = 0;
    while (left > 0 && t < n_max) {
        t += 1;
        orc3_halfstep(m, phi, mask, 0, T_blk, active, (uint32_t)t, 0u, r, NULL);
        orc3_halfstep(m, phi, mask, 1, T_blk, active, (uint32_t)t, 0u, r, NULL);
        orc3_block_energy(m, phi, E);
        if (e_trace)
            for (int b = 0; b < nblk; ++b)
                e_trace[(int64_t)t * nblk + b] = Nb[b] > 0 ? E[b] / (double)Nb[b] : 0.0;
        left = orc_stop_update(m, t, n_max, E, Es, Nsp, Nb, sigma, active, stop_sweep);
    }
    free(E);
    free(sigma);
    free(active);
    return t;
}

void orc3_calibrate(const orc_model* m, const double* phi_init, const uint8_t* mask,
                    const double* Es, const int64_t* Nsp_all, const int64_t* Nb, int32_t n_eq,
                    int32_t n_meas, int32_t n_bisect, int32_t chains, double T_lo, double T_hi,
                    double* T_out) {
    int64_t* Nsp = calib_targets(m, mask, Nsp_all, 1);
    const int nblk = m->nblk;
    const int64_t n = (int64_t)m->D * m->H * m->W;
    double* lo = (double*)malloc(sizeof(double) * nblk);
    double* hi = (double*)malloc(sizeof(double) * nblk);
    double* T = (double*)malloc(sizeof(double) * nblk);
    double* ebar = (double*)malloc(sizeof(double) * nblk);
    double* E = (double*)malloc(sizeof(double) * nblk);
    double* phi = (double*)malloc(sizeof(double) * n);
    for (int b = 0; b < nblk; ++b) { lo[b] = T_lo; hi[b] = T_hi; }
    for (int k = 0; k < n_bisect; ++k) {
        for (int b = 0; b < nblk; ++b) T[b] = 0.5 * (lo[b] + hi[b]);
        const double med = orc_median_targeted(nblk, T, Nsp);
        for (int b = 0; b < nblk; ++b) {
            if (Nsp[b] == 0) T[b] = med;
            ebar[b] = 0.0;
        }
        for (int c = 0; c < chains; ++c) {
            memcpy(phi, phi_init, sizeof(double) * n);
            for (int s = 1; s <= n_eq + n_meas; ++s) {
                orc3_halfstep(m, phi, mask, 0, T, NULL, (uint32_t)s, (uint32_t)(1 + k), (uint32_t)c, NULL);
                orc3_halfstep(m, phi, mask, 1, T, NULL, (uint32_t)s, (uint32_t)(1 + k), (uint32_t)c, NULL);
                if (s <= n_eq) continue;
                orc3_block_energy(m, phi, E);
                for (int b = 0; b < nblk; ++b)
                    if (Nb[b] > 0) ebar[b] += E[b] / (double)Nb[b];
            }
        }
        for (int b = 0; b < nblk; ++b) {
            ebar[b] /= (double)n_meas * (double)chains;
            if (Nsp[b] == 0) continue;
            const double es = Es[b] / (double)Nsp[b];
            if (ebar[b] < es) lo[b] = T[b]; else hi[b] = T[b];
        }
    }
    for (int b = 0; b < nblk; ++b) T_out[b] = 0.5 * (lo[b] + hi[b]);
    const double med = orc_median_targeted(nblk, T_out, Nsp);
    for (int b = 0; b < nblk; ++b)
        if (Nsp[b] == 0) T_out[b] = med;
    free(lo); free(hi); free(T); free(ebar); free(E); free(phi);
    free(Nsp);
}

/* Eqs. 3-4: AAE and RASE over the P prediction sites. */
void orc_scores(int64_t n, const float* pred, const float* truth, const uint8_t* mask,
                double* aae, double* rase) {
    double sa = 0.0, s2 = 0.0;
    int64_t P = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!mask[i]) continue;
        double e = (double)truth[i] - (double)pred[i];
        sa += fabs(e);
        s2 += e * e;
        P += 1;
    }
    *aae = P ? sa / (double)P : 0.0;
    *rase = P ? sqrt(s2 / (double)P) : 0.0;
}
