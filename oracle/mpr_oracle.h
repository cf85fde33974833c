/*
 * CPU oracle for SV-MPR gap filling (Lach & Zukovic, arXiv 2212.01317).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, FP64 restatement of the
 * method used to check the CUDA library. Only the test-suite, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the product path never
 * does. It shares no code with the CUDA library.
 *
 * Layout: angles phi are full-grid, row-major double arrays [H*W] per
 * realization; mask is uint8 [H*W] with 1 = gap (prediction site, G_P) and
 * 0 = sample (G_S). Blocks are lb x lb squares, b = (y/lb)*nbx + x/lb.
 */
#ifndef MPR_ORACLE_H
#define MPR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t H, W, lb;        /* grid and block side l_b */
    int32_t nbx, nby, nblk;  /* filled by orc_model_init */
    double q, J;             /* Eq. 1 parameters */
    uint32_t key0, key1;     /* Philox key: (seed_lo, seed_hi ^ slice) */
    int32_t overrelax;       /* 1: Metropolis followed by over-relaxation */
    int32_t K;               /* 0: continuous angles; K>0: K discrete levels, OR off */
    int32_t threads;         /* OpenMP threads (<=0: library default) */
    const double* T_site;    /* NULL: block temperatures (BST); else H*W site
                                temperatures (SST, Sec. 2.2.3) used by the updates */
    int32_t D, nbz;          /* 3-D grids (orc3_*): depth and block layers; 1 in 2-D */
    int32_t storage;         /* stored gap angles (the precision form): 0 exact (FP64),
                                1 BF16, 2 FP16. A proposal is the FP32 product of 2pi and
                                u0, rounded to the stored type before its energy is taken;
                                a reflected angle is rounded too (via FP32, ties to even). */
    int32_t stop_rule;       /* 0 CROSS (first crossing of e_s,b), 1 WINDOW (end of the
                                energy drift, tested on the last n_fit sweeps every n_f) */
    int32_t n_fit, n_f;      /* WINDOW: window length and test period (Sec. 3.4: 20, 5) */
} orc_model;

/* v rounded to the stored type of `storage` (0: v itself), via FP32, ties to even. */
double orc_round_store(double v, int32_t storage);

void orc_model_init(orc_model* m, int32_t H, int32_t W, int32_t lb, double q, double J,
                    uint64_t seed, uint32_t slice);

/* Philox4x32-10 (Salmon et al., SC'11) and the (0,1) uniform used by the chain. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u01(uint32_t x);
/* The two uniforms (u0 proposal, u1 acceptance) of site i, sweep t, tag, realization r. */
void orc_site_uniforms(const orc_model* m, int64_t i, uint32_t t, uint32_t tag, uint32_t r,
                       double* u0, double* u1);

/* Sec. 2.1: linear map of sample values onto [0, 2pi]; returns 1 if z_max == z_min. */
int orc_transform(int64_t n, const float* values, const uint8_t* mask, double* zmin,
                  double* zmax, double* phi);
void orc_backtransform(int64_t n, const double* mean_phi, const uint8_t* mask,
                       const float* values, double zmin, double zmax, float* out);

/* Eq. 2 per block with owned-bond counting (Sec. 2.2.2). */
void orc_block_stats(const orc_model* m, const double* phi, const uint8_t* mask,
                     double* Es, int64_t* Nsp, int64_t* Nb, double* mean_angle,
                     int64_t* n_gap, int64_t* n_sample, double* global_mean);
/* Eq. 1 restricted to the bonds owned by each block. */
void orc_block_energy(const orc_model* m, const double* phi, double* E);
/* Eq. 1 over the whole grid. */
double orc_total_energy(const orc_model* m, const double* phi);

/* Per-site diagnostics of one update (margins of the floating-point decisions). */
typedef struct {
    double dE, theta;   /* Metropolis: accept iff dE < theta (theta = -T ln u1) */
    double phi_or;      /* over-relaxed candidate (NaN when skipped) */
    double R;           /* |C + iS| of the neighbour field (OR conditioning) */
    double phi_old, phi_prop;
    int32_t accepted, or_applied;
} orc_diag;

/* SST site temperatures (Sec. 2.2.3): every site starts from its block's T,
 * then n_s times every site's T is replaced by the mean over the square of
 * side 2 r_s + 1 centred on it, with coordinates clamped to the grid.
 * T_blk[nblk] -> T_site[H*W]. */
void orc_sst_temperatures(const orc_model* m, const double* T_blk, int32_t r_s, int32_t n_s,
                          double* T_site);

/* Metropolis (+ OR) update of gap site i at temperature T, in place. */
void orc_update_site(const orc_model* m, double* phi, const uint8_t* mask, int64_t i,
                     double T, uint32_t t, uint32_t tag, uint32_t r, orc_diag* d);
/* One checkerboard half-step (Sec. 2.2.2): all gap sites of `colour` whose block
 * is active. T_blk[nblk]; active[nblk] (NULL = all active); diag[H*W] or NULL. */
void orc_halfstep(const orc_model* m, double* phi, const uint8_t* mask, int colour,
                  const double* T_blk, const uint8_t* active, uint32_t t, uint32_t tag,
                  uint32_t r, orc_diag* diag);

/* Sec. 3.3.3 initialisation: gaps <- block sample mean (fallback: global mean). */
void orc_init_block_mean(const orc_model* m, double* phi, const uint8_t* mask,
                         const double* mean_angle, const int64_t* n_sample, double global_mean);
/* Plain-MPR random initialisation: gaps <- 2*pi*u from the reserved tag 0xFFFF. */
void orc_init_random(const orc_model* m, double* phi, const uint8_t* mask, uint32_t r);

/* Local-equilibrium simulation of one realization with per-block stop (Sec. 3.4).
 * phi holds the initial state on entry and the final state on exit.
 * stop_sweep[nblk] receives each block's stop sweep. e_trace (nullable) receives
 * e_b(t) for t = 0..n_max as [(n_max+1) * nblk] (unused entries untouched).
 * Returns the number of sweeps run. */
/* The WINDOW rule after sweep t (Sec. 3.4 names n_fit = 20, the length of the
 * energy series the equilibrium test uses, and n_f = 5, its period; the first
 * test comes after n_fit + n_f sweeps). hist[(s mod n_fit) * nblk + b] holds
 * e_b(s) for the sweeps s of the window (the caller writes e_b(t) before the
 * call). At t = n_fit + n_f + k n_f, a targeted active block stops once the
 * least-squares slope of e_b over sweeps t - n_fit + 1 .. t no longer has the
 * sign sigma_b of e_s,b - e_b(0) (sigma_b = 0: at the first test). Blocks
 * without sample bonds and n_max as in orc_stop_update. */
int orc_stop_update_window(const orc_model* m, int32_t t, int32_t n_max, const double* Es,
                           const int64_t* Nsp, const int8_t* sigma, const double* hist,
                           uint8_t* active, int32_t* stop_sweep);
/* The numerator of that slope: sum_j (2 j - (n_fit - 1)) e_b(t - n_fit + 1 + j). */
double orc_window_slope(const orc_model* m, int32_t t, const double* hist, int b);

int orc_simulate_one(const orc_model* m, double* phi, const uint8_t* mask, const double* T_blk,
                     const double* Es, const int64_t* Nsp, const int64_t* Nb,
                     const int64_t* n_gap, int32_t n_max, uint32_t r, int32_t* stop_sweep,
                     double* e_trace);

/* Sampling variant: one chain from phi (modified) runs n_equil sweeps with
 * every block active, then n_samples sweeps, adding its state after each to
 * sum[i] at the gap sites (realization r, tag 0, sweeps 1, 2, ...). */
void orc_sample_chain(const orc_model* m, double* phi, const uint8_t* mask, const double* T_blk,
                      int32_t n_equil, int32_t n_samples, uint32_t r, double* sum);

/* Stop bookkeeping shared by orc_simulate_one and step-wise callers:
 * decide stops after sweep t given block energies E[nblk]. */
void orc_stop_init(const orc_model* m, const double* E0, const double* Es, const int64_t* Nsp,
                   const int64_t* Nb, const int64_t* n_gap, int8_t* sigma, uint8_t* active,
                   int32_t* stop_sweep);
int orc_stop_update(const orc_model* m, int32_t t, int32_t n_max, const double* E,
                    const double* Es, const int64_t* Nsp, const int64_t* Nb, const int8_t* sigma,
                    uint8_t* active, int32_t* stop_sweep);

/* Block-temperature calibration by bisection (Sec. 2.1 energy matching applied
 * per block as in Sec. 2.2.2). phi_init holds the initialised state (copied for
 * every chain of every iteration). T_out[nblk]. ebar_trace (nullable) gets the
 * per-iteration measured energies [n_bisect * nblk]. */
void orc_calibrate(const orc_model* m, const double* phi_init, const uint8_t* mask,
                   const double* Es, const int64_t* Nsp, const int64_t* Nb, int32_t n_eq,
                   int32_t n_meas, int32_t n_bisect, int32_t chains, double T_lo, double T_hi,
                   double* T_out, double* ebar_trace);
/* Calibration by k-section (points = 1: the bisection above; points = 2:
 * trisection): iteration k evaluates every targeted block at the `points`
 * temperatures splitting its bracket into points + 1 equal parts (untargeted
 * blocks at the median of the targeted blocks' temperatures of the same
 * point), with `chains` fresh chains per point (realization index
 * c * points + p for chain c at point p, tag 1 + k), and keeps the part of
 * the bracket between the highest point whose mean e_b is below e_s,b and
 * the lowest point whose mean is not (between the first and last point if
 * noise makes those cross). T_out: bracket midpoints, untargeted blocks at
 * the median. Warm start (T0_warm != NULL, points >= 2): the first
 * iteration's points are evenly spaced on [T0_warm[b] / warm, T0_warm[b] warm]
 * instead (T0 from the unconditional curve, orc_curve_T0); the same rule then
 * keeps [T_lo, first point], a span between points, or [last point, T_hi].
 * n_eq_next < 0: every iteration restarts its chains from phi_init and runs
 * n_eq + n_meas sweeps; n_eq_next >= 0: each (chain, point) keeps its state
 * from one iteration to the next (the first starts from phi_init with n_eq
 * sweeps of equilibration, later ones run n_eq_next, then n_meas).
 * ebar_trace / pts_trace: NULL, or n_iter * points * nblk doubles receiving,
 * at ((k * points + p) * nblk + b), iteration k's mean e_b and temperature at
 * point p of every targeted block. */
void orc_calibrate_points(const orc_model* m, const double* phi_init, const uint8_t* mask,
                          const double* Es, const int64_t* Nsp, const int64_t* Nb, int32_t n_eq,
                          int32_t n_meas, int32_t n_iter, int32_t chains, int32_t points,
                          double T_lo, double T_hi, const double* T0_warm, double warm,
                          int32_t n_eq_next, double* T_out, double* ebar_trace,
                          double* pts_trace);

/* Unconditional specific energy e(T[k]) of a data-free L x L lattice (Sec. 2.1
 * energy matching without data): angles start at pi, n_eq sweeps, then the
 * mean of E / (2 L (L - 1)) over n_meas sweeps; temperature k is realization
 * k of tag 0xFFFE under key (seed, slice 0). */
void orc_energy_curve(double q, double J, uint64_t seed, int32_t overrelax, int32_t L, int32_t n_T,
                      const double* T, int32_t n_eq, int32_t n_meas, double* e_out);
/* T where the non-decreasing envelope of the curve (T[k], e[k]) reaches e_s,
 * by linear interpolation, clamped to [T[0], T[n-1]]. */
double orc_curve_T0(int32_t n, const double* T, const double* e, double e_s);

/* Energy moments of the calibration chains at block temperatures T[nblk]
 * (the energy matching of Sec. 2.1 / 2.2.2, with the fluctuation identity
 * for its derivative): chain c (c < chains) of phi[c][H*W] runs sweeps
 * s = 1 .. n_eq + n_meas with random-stream tag `tag` and realization index
 * c; after each of the last n_meas sweeps, E_b (Eq. 1 over the bonds block b
 * owns, FP64 from scratch) enters the sums. Out (each nblk, any may be NULL):
 * mean_e[b] = <E_b> / N_b (0 if N_b = 0), var_E[b] = <E_b^2> - <E_b>^2,
 * cov_r[b] = <E_b E_{b+1}> - <E_b><E_{b+1}> (block to the right; 0 on the last
 * block column), cov_d[b] = the same with the block below (0 on the last row).
 * Averages run over the n_meas sweeps and the chains. phi is updated in place. */
void orc_energy_moments(const orc_model* m, double* phi, const uint8_t* mask, const double* T,
                        int32_t n_eq, int32_t n_meas, int32_t chains, uint32_t tag,
                        const int64_t* Nb, double* mean_e, double* var_E, double* cov_r,
                        double* cov_d);

/* Per-block temperatures by damped Newton steps on the energy match:
 * iteration k (k < n_newton) gives untargeted blocks the median of the
 * targeted T, runs the chains (fresh from phi_init at k = 0, continued after)
 * with tag 1 + k, and from y_b = <E_b>/N_b and d y_b / d beta_b = -Var(E_b)/N_b
 * (fluctuation identity) moves every targeted block to
 *   beta_b + (y_b - e_s,b) N_b / Var(E_b)
 * (T doubled if that beta is <= 0; without variance, T doubled or halved
 * towards e_s,b), the new T kept within a factor 2 of the old one and within
 * [T_lo, T_hi]. Starts at T0. T_out: final temperatures, untargeted blocks at
 * the median. trace (NULL or n_newton * nblk): the T_b each iteration ran at. */
void orc_calibrate_newton(const orc_model* m, const double* phi_init, const uint8_t* mask,
                          const double* Es, const int64_t* Nsp, const int64_t* Nb, int32_t n_eq,
                          int32_t n_meas, int32_t n_newton, int32_t chains, double T_lo,
                          double T_hi, double T0, double* T_out, double* trace);

/* Median of the temperatures of targeted blocks (Sec. 2.2.2 fallback). */
double orc_median_targeted(int32_t nblk, const double* T, const int64_t* Nsp);

/* Sec. 3.2, Eqs. 3-4 over the gap sites. */
void orc_scores(int64_t n, const float* pred, const float* truth, const uint8_t* mask,
                double* aae, double* rase);

/* ---- 3-D grids (space-time extension named in Sec. 4) ----
 * Sites (z, y, x) of a D x H x W grid, index i = (z H + y) W + x, colour
 * (x + y + z) mod 2, cubic blocks of side lb numbered ((z/lb) nby + y/lb) nbx
 * + x/lb. Every site owns its +x, +y and +z bonds (6-neighbour MPR
 * Hamiltonian, open boundaries). Everything else (random numbers keyed by
 * the site index, Metropolis + over-relaxation, the stop rule, calibration)
 * is the 2-D method; D = 1 gives back the 2-D functions' results. Arrays are
 * D*H*W (sites) or nblk = nbx nby nbz (blocks). */
void orc3_model_init(orc_model* m, int32_t D, int32_t H, int32_t W, int32_t lb, double q,
                     double J, uint64_t seed, uint32_t slice);
void orc3_block_stats(const orc_model* m, const double* phi, const uint8_t* mask, double* Es,
                      int64_t* Nsp, int64_t* Nb, double* mean_angle, int64_t* n_gap,
                      int64_t* n_sample, double* global_mean);
void orc3_block_energy(const orc_model* m, const double* phi, double* E);
void orc3_update_site(const orc_model* m, double* phi, const uint8_t* mask, int64_t i, double T,
                      uint32_t t, uint32_t tag, uint32_t r, orc_diag* d);
void orc3_halfstep(const orc_model* m, double* phi, const uint8_t* mask, int colour,
                   const double* T_blk, const uint8_t* active, uint32_t t, uint32_t tag,
                   uint32_t r, orc_diag* diag);
void orc3_init_block_mean(const orc_model* m, double* phi, const uint8_t* mask,
                          const double* mean_angle, const int64_t* n_sample, double global_mean);
int orc3_simulate_one(const orc_model* m, double* phi, const uint8_t* mask, const double* T_blk,
                      const double* Es, const int64_t* Nsp, const int64_t* Nb,
                      const int64_t* n_gap, int32_t n_max, uint32_t r, int32_t* stop_sweep,
                      double* e_trace);
void orc3_calibrate(const orc_model* m, const double* phi_init, const uint8_t* mask,
                    const double* Es, const int64_t* Nsp, const int64_t* Nb, int32_t n_eq,
                    int32_t n_meas, int32_t n_bisect, int32_t chains, double T_lo, double T_hi,
                    double* T_out);

#ifdef __cplusplus
}
#endif
#endif
