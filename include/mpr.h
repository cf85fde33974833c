/*
 * libmpr — SV-MPR gap filling on one GB300 (sm_103a).
 *
 * Spatially variable modified-planar-rotator gap filling of Lach & Zukovic,
 * "Fast gap-filling of massive data by local-equilibrium conditional
 * simulations on GPU" (arXiv 2212.01317): block-specific temperatures
 * (Sec. 2.2.2, "BST"), checkerboard conditional Monte Carlo of Eq. 1 over the
 * gap sites only, a per-block stop at local equilibrium, and the conditional
 * mean back-transformed to the data scale (Sec. 2.1, Sec. 3.2).
 *
 * Conventions for every entry point:
 *   - Grids are row-major H x W; site (y,x) has linear index y*W + x and
 *     checkerboard colour (x + y) & 1. Blocks are l_b x l_b squares, block
 *     id b = (y / l_b) * nbx + x / l_b with nbx = ceil(W / l_b); edge blocks
 *     may be partial.
 *   - mask[i] != 0 marks a gap (prediction site); mask[i] == 0 a sample.
 *   - Pointer arguments may be host or device memory (detected with
 *     cudaPointerGetAttributes); device pointers must be on the context's
 *     device. Inputs are copied; the caller keeps ownership of every buffer it
 *     passes. Outputs are written into caller-allocated buffers of the stated
 *     size.
 *   - All work is issued on the context's CUDA stream (mpr_options.cuda_stream,
 *     NULL = the legacy default stream). Calls that return host-visible data
 *     synchronise that stream before returning.
 *   - No call throws; each returns an mpr_status and records a message that
 *     mpr_last_error() returns until the next call on the same context.
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef MPR_H
#define MPR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPR_ABI_VERSION 1

typedef struct mpr_ctx mpr_ctx; /* opaque; owns every device buffer it uses */

typedef enum {
    MPR_OK = 0,
    MPR_EINVAL = 1,      /* bad argument: sizes, pointers, option values */
    MPR_ENOMEM = 2,      /* device or host allocation failed */
    MPR_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    MPR_ENOSAMPLES = 4,  /* no nearest-neighbour sample pair anywhere: Eq. 2 undefined */
    MPR_ETIMEOUT = 5,    /* a bounded device-side wait gave up (reported, not hung) */
    MPR_ESTATE = 6       /* call out of order (e.g. predict before simulate) */
} mpr_status;

typedef enum { MPR_STORE_F32 = 0, MPR_STORE_BF16 = 1, MPR_STORE_F16 = 2 } mpr_storage;
typedef enum { MPR_INIT_BLOCK_MEAN = 0, MPR_INIT_RANDOM = 1 } mpr_init;
/* Local-equilibrium stop of a (block, realization) pair (Sec. 3.4):
 * CROSS: the first sweep t >= 1 at which the block's specific energy e_b(t)
 *   has reached e_s,b from the side it started on;
 * WINDOW: from sweep n_fit + n_f on, every n_f sweeps, the least-squares
 *   slope of e_b over the last n_fit sweeps is tested; the block stops once
 *   the slope no longer points from e_b(0) towards e_s,b (the drift has
 *   ended). Blocks without sample bonds follow the closing rule in both. */
typedef enum { MPR_STOP_CROSS = 0, MPR_STOP_WINDOW = 1 } mpr_stop_rule;

typedef struct {
    int32_t height, width; /* H, W >= 1, each <= 32768 */
    int32_t block;         /* l_b >= 1 (Sec. 2.2.2 block side) */
} mpr_grid;

typedef struct {
    double q;            /* Eq. 1 modification parameter, 0 < q <= 1/2 (default 0.5) */
    double J;            /* Eq. 1 coupling, J > 0 (default 1) */
    uint64_t seed;       /* Philox key (seed_lo, seed_hi ^ slice_id) */
    uint32_t slice_id;   /* distinguishes random streams of independent fields */
    int32_t n_max;       /* sweep cap per realization (default 200), <= 65535 */
    int32_t n_eq;        /* calibration: equilibration sweeps per iteration (25) */
    int32_t n_meas;      /* calibration: measured sweeps per iteration (20) */
    int32_t n_bisect;    /* calibration: bisection iterations (24), <= 65534 */
    int32_t cal_chains;  /* calibration: independent chains averaged (1) */
    float t_lo, t_hi;    /* calibration bracket (1e-4, 2) */
    int32_t overrelax;   /* 1: Metropolis then over-relaxation per site (default 1) */
    int32_t init;        /* mpr_init (default MPR_INIT_BLOCK_MEAN, Sec. 3.3.3) */
    int32_t storage;     /* mpr_storage of the realizations' gap angles (default F32).
                            BF16 / F16 halve the state; arithmetic stays FP32 and the
                            block energies FP64; proposals and reflections are rounded
                            to the stored type before their energy is taken, so the
                            incremental block energies stay exact for the stored state.
                            Sample angles and the calibration chains stay FP32. */
    int32_t group;       /* realizations interleaved per site: 0 = auto, 2 or 8 */
    int32_t profile;     /* 1: time every sweep-kernel launch with CUDA events (default 0) */
    int32_t cal_mode;    /* calibration launch: 0 auto (= 1), 1 one CUDA graph of per-half-step
                            launches, 2 one persistent cooperative kernel with grid barriers,
                            3 every kernel launched from the host (profilers see each one;
                            with profile = 1 every half-step is timed) */
    int32_t wait_ms;     /* limit of a device-side grid-barrier wait (default 2000 ms);
                            a wait that gives up makes the call return MPR_ETIMEOUT */
    int32_t barrier_test; /* test hook: extra arrivals the grid barrier waits for (default 0);
                             > 0 makes every wait give up after wait_ms */
    int32_t cal_method;  /* 0 bisection (default), 1 damped Newton steps on beta_b with
                            d<e_b>/d beta_b = -Var(E_b)/N_b (see mpr_energy_moments),
                            2 the unconditional curve: T_b = T0_b, where the data-free curve
                            e(T) reaches e_s,b (see mpr_get_energy_curve; no simulation of
                            the field) */
    int32_t n_newton;    /* Newton iterations (default 6), each n_eq + n_meas sweeps */
    float t_init;        /* Newton starting temperature (default 0.1) */
    int32_t sim_graph;   /* 1: mpr_simulate runs its sweep loop as one CUDA graph (a device-side
                            loop; full grids, no per-launch timing; ignored when profile = 1) */
    int32_t cal_points;  /* temperatures tried per block and calibration iteration: 1 bisection
                            (default), 2 trisection (the two on the two lanes of a realization
                            pair; n_bisect iterations shrink each bracket 3x; 16 of them leave
                            it narrower than 24 bisection steps), 4 or 8 (k-section on the lanes
                            of a lane group, lane r of the chains at point r mod k: each
                            iteration shrinks the bracket (k + 1)x; 8 iterations of 8 points
                            equal 16 trisection steps) */
    int32_t sim_tail;    /* running (block, realization) pairs below which mpr_simulate runs the
                            rest of its sweep loop (half-steps and stop tests, separated by
                            bounded grid-wide barriers) as one cooperative launch; 0: never
                            (default: measured slower than the per-launch loop with
                            programmatic launches; ignored by sim_graph and where cooperative
                            launch is unavailable) */
    int32_t sweep_form;  /* realizations' half-step: -1 automatic (default: while many pairs
                            run, two realization pairs per warp when the blocks hold at most 96
                            gap sites per colour on average, else one warp per pair; four warps
                            per pair when few remain), 0, 1, 2: always one, two or four warps
                            per pair, 3: two pairs per warp (16 lanes each), 4: the staged
                            half-step (the other colour's (cos, sin) of q phi staged in shared
                            memory per tile of at most 16 x 32 sites, one thread per gap site
                            and realization pair; batches of lane groups of eight only, other
                            batches take form 0) */
    int32_t pair_tail;   /* running (block, realization) pairs at or below which mpr_simulate runs
                            the rest of its sweep loop as one launch with one CTA per realization
                            pair (each pair's remaining sweeps and stop tests in its CTA, CTA
                            barriers between the phases); 0: never; values above 4096 act as
                            4096 (the default: 0.65 ms of 23.8 ms saved per 1024^2 bench step);
                            sim_tail > 0 takes precedence */
    int32_t sweep_form_bulk; /* with sweep_form = -1: the half-step form while the running
                                count is unknown (-1 the built-in choice by gap sites per block,
                                else 0, 3 or 4 as in sweep_form, e.g. an earlier mpr_autotune's
                                choice): mpr_simulate's first 8 sweeps (its loop reads the count
                                two chunks of four sweeps late), every sweep of the graph form
                                and of mpr_sim_sweep; afterwards the built-in choice */
    int32_t stop_rule;   /* mpr_stop_rule (default MPR_STOP_CROSS) */
    int32_t n_fit;       /* MPR_STOP_WINDOW: sweeps in the least-squares window (default 20) */
    int32_t n_f;         /* MPR_STOP_WINDOW: sweeps between two window tests (default 5) */
    float cal_warm;      /* 0: off (default). w > 1 (at most 100): warm start of the calibration
                            from the unconditional curve (see mpr_get_energy_curve): the first
                            iteration's cal_points points lie evenly on [T0_b / w, T0_b w]; the
                            k-point rule then keeps [t_lo, first point], the span between two
                            points, or [last point, t_hi], and the other n_bisect - 1
                            iterations k-section it. Needs cal_points >= 2, cal_method 0, a
                            cal_mode other than 2, and the curve's first temperature / w above
                            t_lo and its last one * w below t_hi (the default curve and bracket
                            allow w < 1.6) */
    int32_t alloc_test;  /* test hook: > 0 makes the context's alloc_test-th device allocation
                            (counting from 1, those of create included) fail with MPR_ENOMEM
                            without calling the allocator; the call that needed it returns
                            MPR_ENOMEM and a later call allocates again (default 0) */
    int32_t cal_continue; /* -1 (default): every calibration iteration restarts its chains from
                             the initial state and runs n_eq + n_meas sweeps. >= 0: only the
                             first does; later iterations continue each (chain, point) lane
                             from the state the previous iteration left at its previous
                             temperature, with cal_continue equilibration sweeps before the
                             n_meas measured ones. Needs cal_method 0 and a cal_mode other
                             than 2 */
    int32_t cal_sweep;   /* form of the calibration's half-steps (cal_mode 1 and 3): 0 (default)
                            picks by size: one warp per (block, realization pair) when a
                            colour's list needs 2^20 or more threads in the other form and the
                            grid holds at least 64 such units per SM, else one thread per (gap
                            entry, realization pair); 1 always the latter, 2 always the former.
                            Both compute the same moves from the same random numbers; only the
                            FP32 order of the block sums differs */
    void* cuda_stream;   /* cudaStream_t to issue work on (NULL = default stream) */
} mpr_options;

typedef struct {
    int64_t kernel_launches;        /* kernels this context launched so far */
    int64_t sim_halfstep_launches;  /* half-step launches made by simulate */
    int64_t cal_halfstep_launches;  /* half-step launches made by calibrate */
    double sim_halfstep_ms;         /* summed device time of those launches (profile = 1) */
    double cal_halfstep_ms;         /* cal_mode 1: time of the whole calibration graph;
                                       cal_mode 3: summed time of the half-step launches */
    int64_t sim_tail_launches;      /* stop-tail launches (pair_tail or sim_tail) made by
                                       simulate with profile = 1 */
    int64_t sim_tail_updates;       /* site updates those launches ran (of gap_updates) */
    double sim_tail_ms;             /* their device time, stop tests included */
} mpr_profile;

typedef struct {
    int32_t height, width, block, nbx, nby, nblk;
    int64_t n_gap;              /* |G_P| */
    int64_t n_gap_colour[2];    /* gap sites per checkerboard colour */
    double zmin, zmax;          /* Sec. 2.1 transform range (over samples) */
    int32_t degenerate;         /* 1 if zmax == zmin: predictions are the constant */
    int32_t calibrated;         /* temperatures set (calibrated or given) */
    int64_t realizations;       /* realizations accumulated into the mean so far */
    int32_t batch;              /* realizations in the current step-wise batch */
    int32_t group;              /* lane-group width in use */
    int64_t gap_updates;        /* Metropolis+OR site updates run by simulate so far */
    int64_t cal_gap_updates;    /* site updates run by calibrate so far */
    int64_t device_bytes;       /* device memory held by the context */
    int32_t n_slices;           /* fields in the context (1 for mpr_create) */
} mpr_info;

/* Fills *opt with the defaults listed above. */
void mpr_default_options(mpr_options* opt);

/* Sec. 2.1 transform and Eq. 2 per block (Sec. 2.2.2).
 * mask: H*W uint8 (host or device), != 0 = gap. values: H*W float (host or
 * device), read at sample sites only (gap entries may hold anything, NaN
 * included). Computes z_min/z_max over the samples, the angle of every
 * sample, each block's sample energy E_s,b over the sample-sample bonds it
 * owns (a site owns its right and down bond), N_SP,b, N_b and the block's
 * sample mean angle, and builds the gap-site lists. opt may be NULL
 * (defaults). On success *out receives a new context.
 * Errors: EINVAL (sizes, NULL pointers, options), ENOMEM, ECUDA,
 * ENOSAMPLES (no sample pair on the grid and at least one gap site). */
mpr_status mpr_create(const mpr_grid* grid, const uint8_t* mask, const float* values,
                      const mpr_options* opt, mpr_ctx** out);

/* ---- many fields in one context (the batched form) ----
 * mpr_create_batch: n independent fields (time slices) of any sizes, each
 * with its own mask and values (host or device pointers, row-major H_s*W_s;
 * all grids[k].block equal), packed into one canvas of whole blocks so that
 * every kernel launch of the context runs all of them: the calibration, each
 * sweep's half-steps and stop test, the accumulation. No bond joins two
 * fields; every field keeps its own transform range (Sec. 2.1), its own
 * median for blocks without sample bonds (Sec. 2.2.2), its own stop
 * bookkeeping, and its own random streams (key word 1 = seed_hi ^ (slice_id
 * + k), site index within the field), so field k computes what mpr_create
 * on it with slice_id + k computes. Canvas-level calls (state, stop,
 * temperatures, block statistics) use the canvas layout given by
 * mpr_get_slice_layout; mpr_predict writes the whole canvas (0 outside the
 * fields). Errors: EINVAL (sizes, the canvas would exceed 32768 sites a side
 * or 2^22 blocks), ENOSAMPLES (a field with gaps but no sample pair), ENOMEM,
 * ECUDA. The persistent calibration (cal_mode 2) takes one field only.
 * mpr_predict_batch: outs[k] (H_s*W_s floats, host or device) for every
 *   field; truths: NULL or n pointers; aae_rase: NULL or 2n doubles (host),
 *   AAE and RASE (Eqs. 3-4) of every field.
 * Host buffers (pinned or pageable) of either call move as one contiguous
 * copy per field through a device staging buffer the size of the largest
 * field (allocated for the call, freed after it); device buffers are copied
 * into or out of the canvas directly.
 * mpr_get_slice_layout: rects[4n] (host) = (y0, x0, H_s, W_s) of every field
 *   in the canvas. */
mpr_status mpr_create_batch(int32_t n, const mpr_grid* grids, const uint8_t* const* masks,
                            const float* const* values, const mpr_options* options,
                            mpr_ctx** out);
mpr_status mpr_predict_batch(mpr_ctx* ctx, float* const* outs, const float* const* truths,
                             double* aae_rase);
mpr_status mpr_get_slice_layout(const mpr_ctx* ctx, int32_t* rects);

/* Releases every resource of ctx (NULL is a no-op). Its device memory goes
 * back to the library's memory pool, where the next context reuses it. */
void mpr_destroy(mpr_ctx* ctx);

/* Device memory: contexts (2-D and 3-D) allocate from one stream-ordered pool
 * per device, owned by the library, which keeps freed memory cached so that
 * creating and destroying a context per field costs no cudaMalloc / cudaFree.
 * mpr_release_cached_memory returns the cached (unused) part of every pool
 * to the device; memory of live contexts is not affected. Never fails. */
void mpr_release_cached_memory(void);

/* Message of the last failed call on ctx ("" if none); valid until the next call. */
const char* mpr_last_error(const mpr_ctx* ctx);
const char* mpr_status_string(mpr_status s);

mpr_status mpr_get_info(const mpr_ctx* ctx, mpr_info* info);

/* Launch counts and, with mpr_options.profile = 1, the device time of the
 * half-step kernel measured with CUDA events on the context's stream around
 * each launch. Synchronises the stream. */
mpr_status mpr_get_profile(mpr_ctx* ctx, mpr_profile* out);

/* Per-block temperatures by energy matching (Sec. 2.1, applied per block in
 * Sec. 2.2.2): bisection on T_b in [t_lo, t_hi]; every iteration re-initialises
 * the gap sites, runs n_eq + n_meas sweeps of cal_chains chains at the current
 * midpoints and keeps the half of each bracket on the side of e_s,b. Blocks
 * without sample bonds take the median of the other blocks' temperatures.
 * With cal_method = 1 the bisection is replaced by n_newton damped Newton
 * steps on beta_b (see mpr_energy_moments): iteration k runs the chains
 * (fresh at k = 0, continued after) with tag 1 + k at the current T, and
 * every targeted block moves to beta_b + (y_b - e_s,b) N_b / Var(E_b), the
 * new T kept within a factor 2 of the old one and within [t_lo, t_hi] (T
 * doubled when that beta is <= 0; without variance, doubled or halved
 * towards e_s,b). Starts at t_init. With cal_warm > 1 the first iteration's
 * points come from the unconditional curve (see cal_warm); with
 * cal_method = 2 T_b is read off that curve without simulating the field.
 * block_T_out: NULL or nblk floats (host or device), row-major blocks.
 * Errors: EINVAL, ECUDA. A degenerate field (z_max == z_min) skips the
 * iterations and sets every T_b to t_lo. */
mpr_status mpr_calibrate(mpr_ctx* ctx, float* block_T_out);

/* Sets the block temperatures directly (nblk floats > 0, host or device). */
mpr_status mpr_set_temperatures(mpr_ctx* ctx, const float* block_T);
mpr_status mpr_get_temperatures(mpr_ctx* ctx, float* block_T_out);

/* ---- the unconditional e(T) curve ----
 * Plain MPR (Sec. 2.1) matches e_s against the specific energy of the
 * simulated grid. On a lattice without data that energy depends on T alone:
 * the unconditional curve e(T). The library measures it the way the
 * calibration measures a block: a data-free 64 x 64 lattice (open
 * boundaries), every angle started at pi, n_eq sweeps, then
 * E / N_bonds (N_bonds = 2 * 64 * 63) averaged over n_meas sweeps (the
 * context's n_eq, n_meas, q, J and over-relaxation); temperature k is
 * realization k of the random-stream tag 0xFFFE under the fixed key (0, 0),
 * so the curve depends on those five parameters only and is measured once
 * per process for each set of them. The measured curve has MPR_CURVE_POINTS
 * temperatures, geometric from 0.002 to 1.25 (as floats). T0_b is the temperature at which the
 * curve's non-decreasing envelope (each e raised to the largest before it)
 * reaches e_s,b, by linear interpolation, clamped to the first and last point.
 * The curve feeds cal_warm and cal_method = 2.
 *
 * mpr_get_energy_curve: measures the curve if the context has none, then
 * copies its n points into T_out (floats) and e_out (doubles), host or
 * device, each with room for `capacity`; *n_out = n. Errors: EINVAL (a NULL
 * pointer, capacity < n), ECUDA.
 * mpr_set_energy_curve: replaces the context's curve by n caller points
 * (2 <= n <= 64; host or device): T > 0, finite and strictly increasing,
 * e finite. Copied. Errors: EINVAL. */
#define MPR_CURVE_POINTS 40
mpr_status mpr_get_energy_curve(mpr_ctx* ctx, float* T_out, double* e_out, int32_t capacity,
                                int32_t* n_out);
mpr_status mpr_set_energy_curve(mpr_ctx* ctx, const float* T, const double* e, int32_t n);

/* ---- differentiable energy matching ----
 * The calibration (Sec. 2.1, applied per block in Sec. 2.2.2) matches the
 * chains' mean specific block energy y_b = <E_b>/N_b to e_s,b. For the Gibbs
 * law exp(-sum_b beta_b E_b) its derivative is the fluctuation identity
 *   d y_a / d beta_b = -Cov(E_a, E_b) / N_a,
 * exact for one block and for blocks whose gap sites' bonds all belong to
 * their own block; at block edges (a site's left / up bond owned by the
 * neighbouring block, updated at its own block's beta) it is an
 * approximation. Covariances beyond the four neighbouring blocks are
 * taken as 0.
 * mpr_energy_moments: sets the block inverse temperatures to beta[nblk]
 *   (host or device floats > 0, as mpr_set_temperatures with T = 1/beta),
 *   then runs the cal_chains calibration chains for n_eq + n_meas sweeps
 *   with random-stream tag `tag` (1 ... 65534): fresh from the block-mean
 *   start when restart != 0 (equal tags and restarts give common random
 *   numbers), else continuing the chains of the last call or calibration.
 *   Out (each nblk doubles, host or device, any may be NULL): mean_e = y_b,
 *   var_E = Var(E_b), cov_r = Cov(E_b, E_{b+1}) (block to the right; 0 on
 *   the last block column), cov_d = Cov(E_b, E_{b+nbx}) (0 on the last
 *   block row); averages over the n_meas measured sweeps and the chains,
 *   FP64. The moments stay in the context for mpr_energy_vjp.
 * mpr_energy_vjp: grad_beta[b] = sum_a grad_e[a] d y_a / d beta_b with the
 *   moments of the last mpr_energy_moments (nblk doubles each, host or device).
 * Errors: ESTATE (a realization batch is open; no moments yet), EINVAL, ECUDA. */
mpr_status mpr_energy_moments(mpr_ctx* ctx, const float* beta, int32_t n_eq, int32_t n_meas,
                              int32_t tag, int32_t restart, double* mean_e, double* var_E,
                              double* cov_r, double* cov_d);
mpr_status mpr_energy_vjp(mpr_ctx* ctx, const double* grad_e, double* grad_beta);

/* ---- site-specific temperatures (SST, Sec. 2.2.3) ----
 * mpr_smooth_temperatures: every site starts from its block's temperature
 *   (after mpr_calibrate or mpr_set_temperatures), then n_s times every
 *   site's T is replaced by the mean over the square of side 2 r_s + 1
 *   centred on it, coordinates clamped to the grid (sums in FP64, stored as
 *   FP32). Realizations run after this use the site temperatures in their
 *   Metropolis tests; the stop test is unchanged (block energies against
 *   e_s,b). T_site_out: NULL or H*W floats (host or device), row-major.
 *   0 <= r_s <= 4096, 0 <= n_s <= 1000.
 * mpr_set_site_temperatures: H*W positive floats (host or device), or NULL
 *   to return to the block temperatures. mpr_calibrate and
 *   mpr_set_temperatures also return to the block temperatures.
 * mpr_get_site_temperatures: H*W floats.
 * Errors: ESTATE (no block temperatures yet, a batch is open, or no site
 * temperatures to get), EINVAL, ECUDA. */
mpr_status mpr_smooth_temperatures(mpr_ctx* ctx, int32_t r_s, int32_t n_s, float* T_site_out);
mpr_status mpr_set_site_temperatures(mpr_ctx* ctx, const float* T_site);
mpr_status mpr_get_site_temperatures(mpr_ctx* ctx, float* T_site);

/* Runs n_realizations more local-equilibrium conditional simulations
 * (Sec. 2.2.2 block temperatures, Sec. 3.3.3 block-mean start, Sec. 3.4 stop)
 * and adds their final states to the running mean. Realization indices
 * continue from earlier calls, so calling it twice with R equals one call
 * with 2R. The sweeps run as a kernel per phase over the worklist of running
 * (block, realization pair) units; once at most pair_tail (block, realization)
 * pairs run, the rest runs in one launch with one CTA per realization pair
 * (options sim_graph, sim_tail and sweep_form choose other schedules; every
 * schedule computes the same states up to the order of the FP32 energy sums).
 * Errors: ESTATE (no temperatures yet), EINVAL (n < 1), ENOMEM, ECUDA,
 * ETIMEOUT (sim_tail only: a grid-barrier wait gave up). */
mpr_status mpr_simulate(mpr_ctx* ctx, int32_t n_realizations);

/* Conditional mean back-transformed (Sec. 2.1, Sec. 3.2): out[H*W] (host or
 * device) receives the predictions at gap sites and the input values at
 * sample sites, bit for bit. truth: NULL or H*W values; when given,
 * aae_rase[2] (host) receives AAE and RASE over the gap sites (Eqs. 3-4).
 * Errors: ESTATE (no realization accumulated), EINVAL, ECUDA. */
mpr_status mpr_predict(mpr_ctx* ctx, float* out, const float* truth, double* aae_rase);

/* ---- launch-shape autotuning ----
 * mpr_autotune times the realizations' half-step decompositions on trial
 * batches of n_realizations realizations (their first n_sweeps sweeps, every
 * block running, CUDA events on the context's stream) and keeps the fastest
 * for the context's later simulations while their running count is unknown
 * (sweep_form = -1; see sweep_form_bulk: mpr_simulate's first 8 sweeps, so
 * n_sweeps = 8 times exactly the sweeps the choice governs; afterwards the
 * built-in choice). Candidates k:
 *   0: G = 8, one warp per (block, realization pair) unit (sweep form 0);
 *   1: G = 8, two units per warp (form 3);
 *   2: G = 8, the staged half-step on tiles of at most 16 x 32 sites (form 4);
 *   3: G = 2, one warp per unit (form 0).
 * G is the lane-group width (realizations interleaved per site). The results
 * do not depend on the choice (the random streams are keyed by realization,
 * not by lane or form). The trial batches are discarded: nothing is
 * accumulated or counted. Needs temperatures; no batch may be open.
 * out->ms[k]: time of candidate k; out->trial_ms: the whole call.
 * Errors: ESTATE, EINVAL, ENOMEM, ECUDA. */
typedef struct {
    int32_t group;   /* chosen lane-group width */
    int32_t form;    /* chosen half-step form (0, 3 or 4) */
    float ms[4];     /* timed candidates */
    float trial_ms;  /* device time of all trial batches */
} mpr_tuning;
mpr_status mpr_autotune(mpr_ctx* ctx, int32_t n_realizations, int32_t n_sweeps, mpr_tuning* out);

/* ---- realizations split across processes ----
 * The realizations of one field are independent chains (Sec. 2.1) that
 * differ only in their random numbers, which are keyed by the realization
 * index. A job can therefore give each process a disjoint range of indices
 * and add up the per-site sums of the final states; the mean of the sum
 * equals the mean a single process would have accumulated over all ranges.
 * mpr_set_realization_base: the next realization run gets index r_first
 *   (>= 0); later realizations continue from it. Only between batches.
 *   Errors: ESTATE (a batch is open), EINVAL.
 * mpr_get_accumulator: sum_out[H*W] (host or device, row-major) receives
 *   sum_r phi_r at every gap site (transformed scale, radians) and 0 at
 *   sample sites; *n_realizations (may be NULL) the count accumulated.
 * mpr_set_accumulator: replaces the sums and the count (n_realizations >= 0)
 *   with the caller's, e.g. the element-wise sum over processes; sample
 *   entries are ignored. mpr_predict then divides by n_realizations.
 *   Errors: ESTATE (a batch is open), EINVAL, ECUDA. */
mpr_status mpr_set_realization_base(mpr_ctx* ctx, int64_t r_first);
mpr_status mpr_get_accumulator(mpr_ctx* ctx, double* sum_out, int64_t* n_realizations);
mpr_status mpr_set_accumulator(mpr_ctx* ctx, const double* sum_in, int64_t n_realizations);

/* ---- block statistics (Eq. 2 per block), host or device outputs, each nblk long;
 *      any pointer may be NULL. ---- */
mpr_status mpr_get_block_stats(mpr_ctx* ctx, double* Es, int32_t* Nsp, int32_t* Nb,
                               float* mean_angle, int32_t* n_gap);

/* ---- step-wise simulation: the pieces mpr_simulate is made of ----
 * mpr_sim_begin: allocates a batch of n realizations (indices continue from
 *   the accumulated count), initialises their gap sites, computes e_b(0) and
 *   the t = 0 stops. mpr_sim_sweep: runs up to n_sweeps sweeps (colour 0 then
 *   colour 1 half-step, block energies, stop decisions) and writes the number
 *   of (block, realization) pairs still running to *n_active (may be NULL).
 *   mpr_sim_end: adds the batch's states to the running mean. */
mpr_status mpr_sim_begin(mpr_ctx* ctx, int32_t n_realizations);
mpr_status mpr_sim_sweep(mpr_ctx* ctx, int32_t n_sweeps, int64_t* n_active);
mpr_status mpr_sim_end(mpr_ctx* ctx);

/* ---- sampling variant of the conditional mean ----
 * Sec. 2.1 predicts with the mean of the conditional distribution; mpr_simulate
 * estimates it from independent realizations, each stopped at local
 * equilibrium. This variant takes it from n_chains chains instead: each
 * starts like a realization (init option; realization indices continue from
 * the accumulated count), runs n_equil sweeps with every block active (no
 * stop test), then n_samples further sweeps, and its state after each of
 * those is one sample added to the running mean (which mpr_predict reads,
 * together with any realizations). Random streams: chain j is realization
 * r_next + j, tag 0, sweeps t = 1 .. n_equil + n_samples. Needs temperatures
 * and no open batch; n_chains >= 1, n_equil >= 0, n_samples >= 1,
 * n_equil + n_samples <= 65535. Errors: EINVAL, ESTATE, ECUDA, ENOMEM. */
mpr_status mpr_sample_chains(mpr_ctx* ctx, int32_t n_chains, int32_t n_equil, int32_t n_samples);

/* One checkerboard half-step (Sec. 2.2.2) of every realization of the batch:
 * Metropolis (+ over-relaxation) on the gap sites of `colour` whose block is
 * running, with the random-number tag `tag` (0 = simulation, 1 + k =
 * calibration iteration k) and sweep index t. No energies, no stop test. */
mpr_status mpr_halfstep(mpr_ctx* ctx, int32_t colour, int32_t t, int32_t tag);

/* Angles of realization r of the batch as a full H*W float grid (host or
 * device); sample sites carry their transformed angle. set_state reads gap
 * sites only. */
mpr_status mpr_get_state(mpr_ctx* ctx, int32_t r, float* angles);
mpr_status mpr_set_state(mpr_ctx* ctx, int32_t r, const float* angles);

/* Stop bookkeeping of the batch, [batch][nblk] row-major (host or device):
 * stop sweep (-1 = running) and running flag (1 = running). Either may be NULL.
 * set_running overwrites the running flags (1 byte per entry). */
mpr_status mpr_get_stop(mpr_ctx* ctx, int32_t* stop_sweep, uint8_t* running);
mpr_status mpr_set_running(mpr_ctx* ctx, const uint8_t* running);

/* Specific energies e_b = E_b / N_b that the stop test last used, [batch][nblk]
 * doubles (host or device): E_b summed by the sweep kernels (FP32 bond terms,
 * FP64 block sums) at t = 0 (mpr_sim_begin) and after every sweep in which the
 * block was running; entries of stopped blocks keep their last value. */
mpr_status mpr_get_block_e(mpr_ctx* ctx, double* e);

/* Block energies E_b (Eq. 1 over the bonds each block owns) of realization r
 * of the batch, recomputed from scratch in FP64; nblk doubles (host or device). */
mpr_status mpr_block_energy(mpr_ctx* ctx, int32_t r, double* E);

/* ---- block statistics without allocation ----
 * The paper has no counterpart to this entry point; it serves callers that
 * must not allocate device memory at the time they call: a service that
 * reserves all device memory up front for its own pool, code on a
 * latency-critical path that cannot pay for the device-wide synchronisation
 * cudaFree performs, or code running under memory pressure that must not fail
 * on an allocation. It computes what mpr_create computes for the block
 * statistics of one field (Sec. 2.1 range, Eq. 2 per block) but allocates
 * nothing: it works in a fixed scratch array of about 1.25 MiB that the
 * library keeps on every device that loads it, until the process exits.
 *   mask, values: H*W device arrays (as mpr_create); Es, Nsp, Nb, mean_angle,
 *   n_gap: nblk device arrays (as mpr_get_block_stats); zrange: 2 device
 *   doubles (z_min, z_max; both 0 without samples). Every pointer must be
 *   device memory of the current device, or managed memory: host pointers
 *   and device memory of another GPU are rejected before anything runs.
 *   The grid may have at most MPR_NOALLOC_MAX_BLOCKS blocks; larger grids
 *   return MPR_EINVAL without touching the outputs.
 *   Work is queued on cuda_stream (NULL = default stream) and not awaited.
 *   Every call looks up the scratch array's device address (a lookup that
 *   allocates nothing, and stays right after a device reset). The module that
 *   holds the array may be loaded onto a device only at its first use (lazy
 *   module loading), and loading it takes device memory: make one warm-up
 *   call on each device at start-up, before reserving the pool and before
 *   any stream capture, so that no later call needs memory.
 *   All calls share the one scratch array: calls that may overlap on the GPU
 *   (different streams, or different host threads) race and must be
 *   serialised by the caller.
 * Errors: EINVAL (sizes, parameters, NULL or host pointers), ECUDA. */
#define MPR_NOALLOC_MAX_BLOCKS 65536
mpr_status mpr_block_stats_noalloc(const mpr_grid* grid, const uint8_t* mask, const float* values,
                                   double q, double J, double* Es, int32_t* Nsp, int32_t* Nb,
                                   float* mean_angle, int32_t* n_gap, double* zrange,
                                   void* cuda_stream);

/* ---- 3-D grids (the space / space-time extension of Sec. 4) ----
 * A D x H x W grid, site (z, y, x) at index (z H + y) W + x, 6-neighbour
 * bonds of Eq. 1 with open boundaries, cubic blocks of side `block`
 * numbered ((z/lb) nby + y/lb) nbx + x/lb; every site owns its +x, +y, +z
 * bonds; checkerboard colour (x + y + z) mod 2. Everything else is the 2-D
 * method: Sec. 2.1 transform, Eq. 2 per block, per-block bisection
 * (calibration options as mpr_options), local-equilibrium realizations
 * from the block-mean start with the per-block stop (Sec. 3.4), the mean
 * back-transformed. Random numbers: counter (site index, t | tag << 16,
 * r / 2, 0), words 2 (r mod 2) and 2 (r mod 2) + 1, key (seed_lo, seed_hi ^
 * slice_id). FP32 state; the storage, group, cal_mode / cal_method /
 * cal_warm, SST, sim_graph and sweep_form options do not apply; stop_rule must be
 * MPR_STOP_CROSS (else EINVAL). Realizations of one call carry indices
 * r_next, r_next + 1, ... with r_next the accumulated count rounded up to
 * even. Arrays are D*H*W (sites, row-major) or nblk (blocks); pointers
 * host or device. Errors: as the 2-D calls. */
typedef struct {
    int32_t depth, height, width; /* D, H, W >= 1, D*H*W < 2^31 */
    int32_t block;                /* l_b >= 1 */
} mpr_grid3;

typedef struct {
    int32_t depth, height, width, block, nblk;
    int64_t n_gap;
    double zmin, zmax;
    int64_t realizations, gap_updates, cal_gap_updates;
} mpr3_info;

typedef struct mpr3_ctx mpr3_ctx;

mpr_status mpr3_create(const mpr_grid3* grid, const uint8_t* mask, const float* values,
                       const mpr_options* options, mpr3_ctx** out);
void mpr3_destroy(mpr3_ctx* ctx);
const char* mpr3_last_error(const mpr3_ctx* ctx);
mpr_status mpr3_get_info(const mpr3_ctx* ctx, mpr3_info* info);
/* Launch counts and, with mpr_options.profile = 1, the device time of the
 * realizations' half-steps (CUDA events around each sweep's two half-step
 * launches) and of the calibration's iterations (around all of them).
 * Synchronises the stream. */
mpr_status mpr3_get_profile(mpr3_ctx* ctx, mpr_profile* out);
mpr_status mpr3_get_block_stats(mpr3_ctx* ctx, double* Es, int32_t* Nsp, int32_t* Nb,
                                float* mean_angle, int32_t* n_gap);
mpr_status mpr3_calibrate(mpr3_ctx* ctx, float* block_T_out);
mpr_status mpr3_set_temperatures(mpr3_ctx* ctx, const float* block_T);
mpr_status mpr3_simulate(mpr3_ctx* ctx, int32_t n_realizations);
mpr_status mpr3_predict(mpr3_ctx* ctx, float* out, const float* truth, double* aae_rase);
/* step-wise pieces (as the 2-D ones): a batch, one half-step, state access */
mpr_status mpr3_sim_begin(mpr3_ctx* ctx, int32_t n_realizations);
mpr_status mpr3_halfstep(mpr3_ctx* ctx, int32_t colour, int32_t t, int32_t tag);
mpr_status mpr3_get_state(mpr3_ctx* ctx, int32_t r, float* angles);
mpr_status mpr3_set_state(mpr3_ctx* ctx, int32_t r, const float* angles);
mpr_status mpr3_sim_end(mpr3_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MPR_H */
