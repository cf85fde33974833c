// C-ABI of libmpr (include/mpr.h): context lifetime, device memory, and the
// order of kernel launches for create / calibrate / simulate / predict.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <vector>

#include "mpr.h"
#include "mpr_curve.h"
#include "mpr_internal.h"
#include "mpr_launch.h"
#include "mpr_memory.h"

using namespace mpr;

struct mpr_ctx {
    mpr_options opt{};
    Geom g{};
    Model m{};
    Rng rng{};
    cudaStream_t s = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only to record graphs
    int device = 0, n_sm = 152;
    std::string err;

    double zmin = 0, zmax = 0;   // slice 0
    int degenerate = 0;
    // fields packed into the canvas (one for mpr_create)
    int n_slices = 1;
    std::vector<int4> h_rect;    // (y0, x0, H, W) per slice
    std::vector<double> h_zmin, h_zmax;
    std::vector<int32_t> h_degen;
    int4* d_rect = nullptr;
    int4* d_blk = nullptr;
    int32_t* d_of_block = nullptr;
    uint32_t* d_key1 = nullptr;
    double* d_zmin = nullptr;
    double* d_zmax = nullptr;
    int32_t* d_degen = nullptr;
    Slices sl{};
    int64_t n_gap[2] = {0, 0};
    std::vector<int64_t> h_ngap;   // gap sites per slice
    int calibrated = 0;

    std::vector<void*> owned;  // every device allocation, freed at destroy
    int64_t device_bytes = 0;
    int64_t n_allocs = 0;      // allocations seen by the alloc_test hook

    // field
    float* values = nullptr;
    uint8_t* mask = nullptr;
    float* dang = nullptr;
    uint2* list[2] = {nullptr, nullptr};
    int32_t* start[2] = {nullptr, nullptr};
    int32_t* split[2] = {nullptr, nullptr};
    double* Es = nullptr;
    double* es = nullptr;   // E_s,b / N_SP,b
    double* inb = nullptr;  // 1 / N_b
    int32_t *Nsp = nullptr, *Nb = nullptr, *nsamp = nullptr, *ngap_c[2] = {nullptr, nullptr},
            *ngap = nullptr;
    // Blocks that calibrate: sample bonds (a target) and gap sites; 0 for the
    // others, which take the median (a block with sample bonds and no gap
    // site has e_b = e_s,b exactly and nothing to fill).
    int32_t* Nsp_cal = nullptr;
    double* ssum = nullptr;
    float* init_angle = nullptr;
    float *T = nullptr, *beta = nullptr, *lo = nullptr, *hi = nullptr;
    float *T2 = nullptr, *beta2 = nullptr;   // trisection's second point
    float *Tk = nullptr, *betak = nullptr;   // [points][nblk] of the 4- or 8-point calibration
    double* ebark = nullptr;                 // [points][nblk]
    double* ebar2 = nullptr;
    // The unconditional e(T) curve (measured or set on first use).
    float* curve_T = nullptr;
    double* curve_e = nullptr;
    int curve_n = 0;
    float* T_site = nullptr;     // [H*W] site temperatures (SST), allocated on first use
    float* beta_site = nullptr;  // [H*W] 1 / T_site
    int sst = 0;                 // 1: realizations use the site temperatures
    double* msum = nullptr;      // [4][nblk] sums of E, E^2, E E_right, E E_down
    double* mom = nullptr;       // [4][nblk] moments of the last energy-moment run
    bool chains_valid = false;   // the batch state holds the calibration chains
    bool moments_valid = false;
    cudaGraphConditionalHandle sim_cond = 0;   // set while a sweep loop is being captured
    bool sim_capture = false;                  // a sweep loop is being captured
    double* ebar = nullptr;
    double* sum = nullptr;  // [2][H][Wh] running sums of gap angles
    float* out_buf = nullptr;
    float* truth_buf = nullptr;
    double* err_buf = nullptr;
    unsigned long long* counters = nullptr;      // [0] running pairs, [1] site updates
    unsigned long long* h_counters = nullptr;    // pinned mirror
    uint32_t* mm = nullptr;

    // batch (step-wise simulation or calibration chains)
    int G = 1, groups = 0, Rp = 0, R = 0, r_off = 0;
    uint32_t r_even = 0;
    int t = 0;
    int batch_open = 0;
    int storage = 0;             // element type of the batch state (an mpr_storage)
    void* ang = nullptr;
    size_t ang_cap = 0;          // bytes
    double* eacc = nullptr;
    double* ecur = nullptr;      // [nblk][Rp] current E_b of every (block, realization)
    double* ecur0 = nullptr;     // [nblk][Rp] calibration: E_b of the start state
    uint8_t* running = nullptr;
    int32_t* stop = nullptr;
    int8_t* sigma = nullptr;
    double* e_last = nullptr;
    int32_t* tcount = nullptr;
    uint32_t* work = nullptr;    // [2][nblk * groups] worklists of running items, by sweep parity
    uint32_t work_stride = 0;
    size_t blk_cap = 0, lane_cap = 0, work_cap = 0;
    Control* ctl = nullptr;      // device loop state
    Control* h_ctl = nullptr;    // pinned mirror
    int grid_cache[2][3][4] = {};  // full grid of k_sweep by (G = 2 / 8, storage, form)
    // The WINDOW stop rule's ring of e_b (allocated when the rule is chosen).
    double* whist = nullptr;
    size_t whist_cap = 0;          // elements
    // The staged half-step's tiles (built at the first batch that uses them).
    Tiles tiles{};
    float* stab = nullptr;         // [2][H][Wh] staging table
    int32_t* tstart[2] = {nullptr, nullptr};
    uint2* tlist[2] = {nullptr, nullptr};
    int tile_grid = 0;             // resident CTAs of the staged kernel (by storage at build)
    int tile_grid_storage = -1;
    unsigned long long bound = ~0ull;  // upper bound of the running pairs (from the last read)
    int tuned_form = -1;         // autotuned half-step form (-1: the built-in choice)
    bool tuning_tiles = false;   // an autotune trial of the staged form is running
    bool energy_dirty = false;
    GridBarrier* bar = nullptr;  // grid barrier of the persistent calibration
    float* med = nullptr;
    int coop = 0;                // device supports cooperative launch

    int64_t realizations = 0;   // accumulated into sum
    int64_t r_next = 0;         // index of the next realization
    int64_t gap_updates = 0, cal_updates = 0;

    // instrumentation
    int64_t launches = 0;                        // kernels launched by this context
    std::vector<cudaEvent_t> ev_pool;            // recycled events
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_sim, ev_cal;  // pending pairs
    double sim_halfstep_ms = 0.0, cal_halfstep_ms = 0.0;
    int64_t sim_halfstep_launches = 0, cal_halfstep_launches = 0;
    double sim_tail_ms = 0.0;                    // stop-tail launches (profile = 1)
    int64_t sim_tail_launches = 0, sim_tail_updates = 0;
};

namespace {

// An NVTX range around an entry point (create, calibrate, simulate, sample,
// predict, autotune), so that profilers can attribute kernels to the phase
// that launched them; without a profiler attached it costs a pointer check.
struct PhaseRange {
    explicit PhaseRange(const char* name) { nvtxRangePushA(name); }
    ~PhaseRange() { nvtxRangePop(); }
    PhaseRange(const PhaseRange&) = delete;
    PhaseRange& operator=(const PhaseRange&) = delete;
};

mpr_status fail(mpr_ctx* c, mpr_status st, const char* fmt, ...) {
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

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MPR_ENOMEM : MPR_ECUDA,        \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,     \
                        __LINE__);                                                            \
    } while (0)

#define CKL()                                                                                 \
    do {                                                                                      \
        ++ctx->launches;                                                                      \
        cudaError_t e_ = cudaPeekAtLastError();                                               \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, MPR_ECUDA, "kernel launch failed: %s (%s:%d)",                   \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                          \
    } while (0)

#define TRY(expr)                                    \
    do {                                             \
        mpr_status st_ = (expr);                     \
        if (st_ != MPR_OK) return st_;               \
    } while (0)

template <class T>
mpr_status dalloc(mpr_ctx* ctx, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    // Test hook: the alloc_test-th allocation of the context is refused.
    if (ctx->opt.alloc_test > 0 && ++ctx->n_allocs == ctx->opt.alloc_test)
        return fail(ctx, MPR_ENOMEM, "allocation %d of %zu bytes refused by the alloc_test hook",
                    ctx->opt.alloc_test, count * sizeof(T));
    void* q = nullptr;
    cudaError_t e = pool_alloc(&q, count * sizeof(T), ctx->device, ctx->s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, MPR_ENOMEM, "allocation of %zu bytes failed: %s", count * sizeof(T),
                    cudaGetErrorString(e));
    }
    ctx->owned.push_back(q);
    ctx->device_bytes += (int64_t)(count * sizeof(T));
    *p = static_cast<T*>(q);
    return MPR_OK;
}

void dfree(mpr_ctx* ctx, void* p) {
    if (!p) return;
    auto it = std::find(ctx->owned.begin(), ctx->owned.end(), p);
    if (it != ctx->owned.end()) ctx->owned.erase(it);
    pool_free(p, ctx->s);
}

// Lane-group width: 2 (one realization pair per group) for up to two lanes
// or when asked, else 8 (four pairs per group).
int pick_group(int lanes, int requested) {
    if (requested == 2 || requested == 8) return requested;
    return lanes <= 2 ? 2 : 8;
}

mpr_status check_opts(mpr_ctx* ctx, const mpr_options& o) {
    if (!(o.q > 0.0 && o.q <= 0.5)) return fail(ctx, MPR_EINVAL, "q must be in (0, 1/2]");
    if (!(o.J > 0.0)) return fail(ctx, MPR_EINVAL, "J must be > 0");
    if (o.n_max < 1 || o.n_max > 65535) return fail(ctx, MPR_EINVAL, "n_max must be in [1, 65535]");
    if (o.n_eq < 0 || o.n_meas < 1 || o.n_eq + o.n_meas > 65535)
        return fail(ctx, MPR_EINVAL, "n_eq >= 0, n_meas >= 1, n_eq + n_meas <= 65535");
    if (o.n_bisect < 0 || o.n_bisect > 65534) return fail(ctx, MPR_EINVAL, "n_bisect in [0, 65534]");
    if (o.cal_chains < 1 || o.cal_chains > 4096) return fail(ctx, MPR_EINVAL, "cal_chains in [1, 4096]");
    if (!(o.t_lo > 0.0f && o.t_hi > o.t_lo)) return fail(ctx, MPR_EINVAL, "need 0 < t_lo < t_hi");
    if (o.storage != MPR_STORE_F32 && o.storage != MPR_STORE_BF16 && o.storage != MPR_STORE_F16)
        return fail(ctx, MPR_EINVAL, "unknown storage %d", o.storage);
    if (o.group != 0 && o.group != 2 && o.group != 8)
        return fail(ctx, MPR_EINVAL, "group must be 0, 2 or 8");
    if (o.init != MPR_INIT_BLOCK_MEAN && o.init != MPR_INIT_RANDOM)
        return fail(ctx, MPR_EINVAL, "unknown init mode");
    if (o.cal_mode < 0 || o.cal_mode > 3) return fail(ctx, MPR_EINVAL, "cal_mode must be 0 ... 3");
    if (o.wait_ms < 1) return fail(ctx, MPR_EINVAL, "wait_ms must be >= 1");
    if (o.barrier_test < 0) return fail(ctx, MPR_EINVAL, "barrier_test must be >= 0");
    if (o.alloc_test < 0) return fail(ctx, MPR_EINVAL, "alloc_test must be >= 0");
    if (o.cal_method < 0 || o.cal_method > 2) return fail(ctx, MPR_EINVAL, "cal_method must be 0, 1 or 2");
    if (o.cal_points != 1 && o.cal_points != 2 && o.cal_points != 4 && o.cal_points != 8)
        return fail(ctx, MPR_EINVAL, "cal_points must be 1, 2, 4 or 8");
    if (o.sim_tail < 0) return fail(ctx, MPR_EINVAL, "sim_tail must be >= 0");
    if (o.pair_tail < 0) return fail(ctx, MPR_EINVAL, "pair_tail must be >= 0");
    if (o.sweep_form < -1 || o.sweep_form > 4)
        return fail(ctx, MPR_EINVAL, "sweep_form must be -1, 0, 1, 2, 3 or 4");
    if (o.n_newton < 0 || o.n_newton > 65533) return fail(ctx, MPR_EINVAL, "n_newton in [0, 65533]");
    if (o.sweep_form_bulk != -1 && o.sweep_form_bulk != 0 && o.sweep_form_bulk != 3 &&
        o.sweep_form_bulk != 4)
        return fail(ctx, MPR_EINVAL, "sweep_form_bulk must be -1, 0, 3 or 4");
    if (o.stop_rule != MPR_STOP_CROSS && o.stop_rule != MPR_STOP_WINDOW)
        return fail(ctx, MPR_EINVAL, "unknown stop rule");
    if (o.n_fit < 2 || o.n_fit > 64 || o.n_f < 1 || o.n_f > 1024)
        return fail(ctx, MPR_EINVAL, "need 2 <= n_fit <= 64 and 1 <= n_f <= 1024");
    if (o.cal_method == 1 && !(o.t_init > o.t_lo && o.t_init < o.t_hi))
        return fail(ctx, MPR_EINVAL, "need t_lo < t_init < t_hi");
    if (o.cal_sweep < 0 || o.cal_sweep > 2)
        return fail(ctx, MPR_EINVAL, "cal_sweep must be 0, 1 or 2");
    if (o.cal_continue < -1 || o.cal_continue > 65535 - o.n_meas)
        return fail(ctx, MPR_EINVAL, "cal_continue must be -1 or in [0, 65535 - n_meas]");
    if (o.cal_continue >= 0 && (o.cal_method != 0 || o.cal_mode == 2))
        return fail(ctx, MPR_EINVAL, "continued calibration chains need cal_method 0 and a "
                                     "cal_mode other than 2");
    if (!(o.cal_warm == 0.0f || (o.cal_warm > 1.0f && o.cal_warm <= 100.0f)))
        return fail(ctx, MPR_EINVAL, "cal_warm must be 0 or in (1, 100]");
    if (o.cal_warm > 0.0f && (o.cal_points < 2 || o.cal_method != 0 || o.cal_mode == 2))
        return fail(ctx, MPR_EINVAL,
                    "the warm start (cal_warm) needs cal_points >= 2, cal_method 0 and a cal_mode "
                    "other than 2");
    return MPR_OK;
}

// Copies n bytes from a host or device pointer into device memory on the stream.
mpr_status copy_in(mpr_ctx* ctx, void* dst, const void* src, size_t n) {
    CK(cudaMemcpyAsync(dst, src, n, cudaMemcpyDefault, ctx->s));
    return MPR_OK;
}

mpr_status copy_out(mpr_ctx* ctx, void* dst, const void* src, size_t n) {
    CK(cudaMemcpyAsync(dst, src, n, cudaMemcpyDefault, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    return MPR_OK;
}

size_t storage_bytes(int storage) { return storage == MPR_STORE_F32 ? 4 : 2; }

// Per-batch buffers sized for `lanes` realization lanes, state elements of
// type `storage`.
mpr_status ensure_batch(mpr_ctx* ctx, int lanes, int requested_group, int storage) {
    const Geom& g = ctx->g;
    const int G = pick_group(lanes, requested_group);
    const int groups = (lanes + G - 1) / G;
    const int Rp = groups * G;
    const size_t ang_need = (size_t)groups * 2 * g.H * g.Wh * G * storage_bytes(storage);
    if (ang_need > ctx->ang_cap) {
        dfree(ctx, ctx->ang);
        ctx->ang = nullptr;
        ctx->ang_cap = 0;
        uint8_t* p = nullptr;
        TRY(dalloc(ctx, &p, ang_need));
        ctx->ang = p;
        ctx->ang_cap = ang_need;
    }
    const size_t blk_need = (size_t)g.nblk * Rp;
    if (blk_need > ctx->blk_cap) {
        for (void* p : {(void*)ctx->eacc, (void*)ctx->running, (void*)ctx->stop, (void*)ctx->sigma,
                        (void*)ctx->e_last, (void*)ctx->ecur, (void*)ctx->ecur0})
            dfree(ctx, p);
        ctx->eacc = nullptr; ctx->running = nullptr; ctx->stop = nullptr; ctx->sigma = nullptr;
        ctx->e_last = nullptr; ctx->ecur = nullptr; ctx->ecur0 = nullptr;
        ctx->blk_cap = 0;
        TRY(dalloc(ctx, &ctx->eacc, 2 * blk_need));   // two per-sweep buffers
        TRY(dalloc(ctx, &ctx->ecur, blk_need));
        TRY(dalloc(ctx, &ctx->ecur0, blk_need));
        TRY(dalloc(ctx, &ctx->e_last, blk_need));
        TRY(dalloc(ctx, &ctx->running, blk_need));
        TRY(dalloc(ctx, &ctx->stop, blk_need));
        TRY(dalloc(ctx, &ctx->sigma, blk_need));
        ctx->blk_cap = blk_need;
    }
    if ((size_t)Rp * ctx->n_slices > ctx->lane_cap) {
        dfree(ctx, ctx->tcount);
        ctx->tcount = nullptr;
        ctx->lane_cap = 0;
        TRY(dalloc(ctx, &ctx->tcount, (size_t)Rp * ctx->n_slices));
        ctx->lane_cap = (size_t)Rp * ctx->n_slices;
    }
    // Worklist units: one realization pair of one block (Rp / 2 per block).
    const size_t work_need = (size_t)g.nblk * (Rp / 2);
    if (work_need > ctx->work_cap) {
        dfree(ctx, ctx->work);
        ctx->work = nullptr;
        ctx->work_cap = 0;
        TRY(dalloc(ctx, &ctx->work, 2 * work_need));
        ctx->work_cap = work_need;
    }
    ctx->work_stride = (uint32_t)work_need;
    if (ctx->opt.stop_rule == MPR_STOP_WINDOW) {
        const size_t wneed = (size_t)ctx->opt.n_fit * blk_need;
        if (wneed > ctx->whist_cap) {
            dfree(ctx, ctx->whist);
            ctx->whist = nullptr;
            ctx->whist_cap = 0;
            TRY(dalloc(ctx, &ctx->whist, wneed));
            ctx->whist_cap = wneed;
        }
    }
    ctx->storage = storage;
    ctx->bound = ~0ull;
    ctx->G = G;
    ctx->groups = groups;
    ctx->Rp = Rp;
    CK(cudaMemsetAsync(ctx->eacc, 0, 2 * blk_need * sizeof(double), ctx->s));
    CK(cudaMemsetAsync(ctx->ctl, 0, sizeof(Control), ctx->s));
    return MPR_OK;
}

SweepArgs sweep_args(mpr_ctx* ctx, int colour, bool simulate) {
    SweepArgs a{};
    a.g = ctx->g;
    a.m = ctx->m;
    a.rng = ctx->rng;
    a.sl = ctx->sl;
    a.colour = colour;
    a.list = ctx->list[colour];
    a.start = ctx->start[colour];
    a.split = ctx->split[colour];
    a.ang = ctx->ang;
    a.dang = ctx->dang;
    a.beta = ctx->beta;
    a.beta_site = (simulate && ctx->sst) ? ctx->beta_site : nullptr;
    a.running = simulate ? ctx->running : nullptr;
    a.eacc = ctx->eacc;
    a.ecur = ctx->ecur;
    a.work = simulate ? ctx->work : nullptr;
    a.work_stride = ctx->work_stride;
    a.ctl = ctx->ctl;
    a.R = ctx->R;
    a.Rp = ctx->Rp;
    a.groups = ctx->groups;
    a.r_base = ctx->r_even;
    a.energy = 1;
    if (ctx->tiles.n > 0) {
        a.tl = ctx->tiles;
        a.tl.start = ctx->tstart[colour];
        a.tl.list = ctx->tlist[colour];
        a.tl.stab = ctx->stab;
    }
    return a;
}

// The stop rule of the realizations' stop tests.
StopWindow stop_window(const mpr_ctx* ctx) {
    StopWindow w{};
    w.rule = ctx->opt.stop_rule;
    w.n_fit = ctx->opt.n_fit;
    w.n_f = ctx->opt.n_f;
    w.hist = ctx->whist;
    w.stride = (size_t)ctx->g.nblk * ctx->Rp;
    return w;
}

// The staged half-step (form 4) needs lane groups of eight and its tiles.
bool tile_form_ok(const mpr_ctx* ctx) { return ctx->G == 8 && ctx->tiles.n > 0; }

// The options, the autotuner's choice or its trial ask for the staged half-step.
bool tiles_wanted(const mpr_ctx* ctx) {
    return ctx->opt.sweep_form == 4 || ctx->tuned_form == 4 || ctx->tuning_tiles ||
           (ctx->opt.sweep_form < 0 && ctx->opt.sweep_form_bulk == 4);
}

// Tiles, tile-major lists and staging table of the staged half-step, built
// once per context.
mpr_status ensure_tiles(mpr_ctx* ctx) {
    if (ctx->tiles.n > 0) return MPR_OK;
    const Geom& g = ctx->g;
    Tiles t = tile_shape(g);
    const size_t plane = (size_t)g.H * g.Wh;
    int32_t* cnt[2] = {nullptr, nullptr};
    TRY(dalloc(ctx, &ctx->stab, 2 * plane));
    for (int c = 0; c < 2; ++c) {
        TRY(dalloc(ctx, &ctx->tstart[c], (size_t)t.n + 1));
        TRY(dalloc(ctx, &ctx->tlist[c], (size_t)std::max<int64_t>(1, ctx->n_gap[c])));
        TRY(dalloc(ctx, &cnt[c], (size_t)t.n));
    }
    launch_stage_table(g, ctx->mask, ctx->dang, ctx->stab, ctx->s);
    launch_tile_count(g, t, ctx->d_of_block, ctx->mask, cnt[0], cnt[1], ctx->s);
    launch_scan(cnt[0], t.n, ctx->tstart[0], ctx->s);
    launch_scan(cnt[1], t.n, ctx->tstart[1], ctx->s);
    launch_tile_lists(g, t, ctx->d_of_block, ctx->mask, ctx->tstart[0], ctx->tstart[1],
                      ctx->tlist[0], ctx->tlist[1], ctx->s);
    ctx->launches += 5;
    CKL();
    dfree(ctx, cnt[0]);
    dfree(ctx, cnt[1]);
    ctx->tiles = t;
    return MPR_OK;
}

int tile_grid(mpr_ctx* ctx) {
    if (ctx->tile_grid_storage != ctx->storage) {
        ctx->tile_grid = ctx->n_sm * tile_blocks_per_sm(ctx->storage);
        ctx->tile_grid_storage = ctx->storage;
    }
    const int64_t items = (int64_t)ctx->tiles.n * ctx->groups;
    return (int)std::max<int64_t>(1, std::min<int64_t>(ctx->tile_grid, items));
}


// Running pairs per SM below which the half-step takes four warps per
// realization pair (form 2), and a grid no larger than the running pairs can
// fill. (Measured on the 1024² bench batch: two warps per pair below 32 to
// 512 pairs per SM made the batch 0.1 to 0.7 ms slower, one warp throughout
// ties with this choice; the stop tail costs launches, not passes.)
constexpr unsigned long long kForm2PairsPerSm = 4;
// Mean gap entries per block and colour at or below which two realization
// pairs share a warp (form 3). Measured: 1024^2, l_b = 16, 64 entries:
// simulate 23.10 -> 21.24 ms; 4096^2, l_b = 32, about 307 entries: 127.3 ->
// 131.4 ms.
constexpr double kHalfFormEntries = 96.0;

int sweep_form(mpr_ctx* ctx) {
    if (ctx->opt.sweep_form == 4) return tile_form_ok(ctx) ? 4 : 0;
    if (ctx->opt.sweep_form >= 0) return ctx->opt.sweep_form;
    if (ctx->bound < (unsigned long long)ctx->n_sm * kForm2PairsPerSm) return 2;
    // An autotuned (or asked-for) form holds while the running count is
    // unknown: the sweeps the autotuner's trial reproduces (a fresh batch, no
    // count read yet), which in the per-launch loop are its first two chunks
    // of four sweeps. (On the 256-field batch two pairs per warp ran the first
    // 8 sweeps 3.9 % faster, and the whole run 1.3 % slower when the form was
    // held for as long as 7/8 of the pairs ran, the count read late.)
    const int bulk = ctx->tuned_form >= 0 ? ctx->tuned_form : ctx->opt.sweep_form_bulk;
    if (bulk >= 0 && ctx->bound == ~0ull) {
        if (bulk == 4) return tile_form_ok(ctx) ? 4 : 0;
        return bulk;
    }
    const double per_block = (double)(ctx->n_gap[0] + ctx->n_gap[1]) / (2.0 * ctx->g.nblk);
    return per_block <= kHalfFormEntries ? 3 : 0;
}

int sweep_grid(mpr_ctx* ctx, int form) {
    int& full = ctx->grid_cache[ctx->G == 2 ? 0 : 1][ctx->storage][form];
    if (full == 0) full = ctx->n_sm * sweep_blocks_per_sm(ctx->G, ctx->storage, form);
    const unsigned long long ipc = (unsigned long long)sweep_items_per_cta(ctx->G, form);
    // (bound is ~0 while unknown: round up without overflowing)
    const unsigned long long need = ctx->bound / ipc + (ctx->bound % ipc != 0 ? 1 : 0);
    return (int)std::max<unsigned long long>(1, std::min<unsigned long long>(full, need));
}

// One realization half-step of the batch in sweep form `form` (4: staged).
void launch_halfstep(mpr_ctx* ctx, const SweepArgs& a, int form) {
    if (form == 4) {
        launch_sweep_tile(a, ctx->storage, tile_grid(ctx), ctx->s);
        return;
    }
    launch_sweep(a, ctx->G, ctx->storage, form, sweep_grid(ctx, form), ctx->s);
}

// Grid of the stop kernels: a thread per (item, lane) or per item, at most
// `per_sm` CTAs per SM (the kernels loop). The closing kernel's CTAs each take
// one ticket from a single counter, so it runs on fewer CTAs (two per SM);
// the targeted part has no such counter.
constexpr int kTargetedCtasPerSm = 8;
constexpr int kClosingCtasPerSm = 2;

int stop_grid(mpr_ctx* ctx, int64_t per_item, int per_sm) {
    const int64_t items = std::min<int64_t>((int64_t)ctx->g.nblk * (ctx->Rp / 2),
                                            (int64_t)std::min<unsigned long long>(ctx->bound, 1ull << 40));
    const int64_t n = std::max<int64_t>(1, items * per_item);
    return (int)std::min<int64_t>((n + 255) / 256, (int64_t)ctx->n_sm * per_sm);
}

cudaEvent_t get_event(mpr_ctx* ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// E_b of the batch's current state from scratch, into ecur: E_s,b plus every
// bond that touches a gap site (every lane of every block: the pass ignores
// the running flags). Clears eacc.
mpr_status energy_pass(mpr_ctx* ctx) {
    launch_ecur_reset(ctx->g.nblk, ctx->Rp, ctx->Es, ctx->ecur, ctx->eacc, ctx->s);
    CKL();
    for (int c = 0; c < 2; ++c) {
        SweepArgs a = sweep_args(ctx, c, false);
        a.R = ctx->Rp;
        launch_energy(a, ctx->G, ctx->storage, ctx->n_sm, ctx->s);
        CKL();
    }
    return MPR_OK;
}

// E_b(0) when every realization starts from the same state (the block-mean
// start, Sec. 3.3.3): the bond sums of the first lane group only, copied to
// the other lanes.
mpr_status energy_pass_shared_start(mpr_ctx* ctx) {
    launch_ecur_reset(ctx->g.nblk, ctx->Rp, ctx->Es, ctx->ecur, ctx->eacc, ctx->s);
    CKL();
    for (int c = 0; c < 2; ++c) {
        SweepArgs a = sweep_args(ctx, c, false);
        a.R = ctx->Rp;
        a.groups = 1;
        launch_energy(a, ctx->G, ctx->storage, ctx->n_sm, ctx->s);
        CKL();
    }
    launch_ecur_broadcast(ctx->g.nblk, ctx->Rp, ctx->G, ctx->ecur, ctx->s);
    CKL();
    return MPR_OK;
}

// After a stream synchronisation: fold the recorded pairs into the totals.
void collect_events(mpr_ctx* ctx) {
    for (int which = 0; which < 2; ++which) {
        auto& v = which ? ctx->ev_cal : ctx->ev_sim;
        double& acc = which ? ctx->cal_halfstep_ms : ctx->sim_halfstep_ms;
        for (auto& pr : v) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) acc += ms;
            else cudaGetLastError();
            ctx->ev_pool.push_back(pr.first);
            ctx->ev_pool.push_back(pr.second);
        }
        v.clear();
    }
}

mpr_status init_batch_state(mpr_ctx* ctx) {
    const int random = ctx->opt.init == MPR_INIT_RANDOM;
    for (int c = 0; c < 2; ++c) {
        launch_init(ctx->g, ctx->sl, ctx->list[c], ctx->n_gap[c], c, ctx->init_angle, ctx->ang,
                    ctx->storage, ctx->G, ctx->Rp, random, ctx->rng, ctx->r_even, ctx->s);
        CKL();
    }
    return MPR_OK;
}

// After the running flags were overwritten: per-realization counts of running
// targeted blocks and the worklist of units (lane groups of G lanes; the
// realizations' worklist uses pairs) with a running lane.
__global__ void k_rebuild(int nblk, int groups, int G, int Rp, const int32_t* of_block,
                          const int32_t* Nsp, const uint8_t* running, int32_t* tcount, Control* ctl,
                          uint32_t* work_all, uint32_t work_stride) {
    const int64_t n = (int64_t)nblk * groups;
    const uint32_t par = ctl->t & 1u;
    uint32_t* work = work_all + (size_t)par * work_stride;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < n;
         it += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(it / groups), grp = (int)(it % groups);
        bool any = false;
        for (int g = 0; g < G; ++g) {
            const int r = grp * G + g;
            if (!running[(size_t)b * Rp + r]) continue;
            any = true;
            if (Nsp[b] > 0) atomicAdd(&tcount[of_block[b] * Rp + r], 1);
        }
        if (any) work[atomicAdd(&ctl->n_work[par], 1u)] = (uint32_t)it;
    }
}

__global__ void k_fill_valid(uint8_t* running, int64_t n, int Rp, int r_off, int R) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t % Rp);
        running[t] = (r >= r_off && r < r_off + R) ? 1 : 0;
    }
}

// One sweep of the batch: colour 0, colour 1, block energies, stop tests,
// next worklist. Everything the kernels need comes from device memory.
mpr_status sweep_once(mpr_ctx* ctx) {
    const Geom& g = ctx->g;
    // With profiling on, one event pair spans the sweep's two half-steps
    // (launched back to back), so the events do not split them.
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ctx->opt.profile) {
        e0 = get_event(ctx);
        e1 = get_event(ctx);
        if (e0) cudaEventRecord(e0, ctx->s);
    }
    // The device's sweep index is the host's count plus one (the stop test at
    // t = 0 set it to 1, and every sweep's closing CTA advances it), so the
    // kernels take it as an argument instead of a dependent read; a captured
    // loop body reads it on the device.
    const int t_known = ctx->sim_capture ? -1 : ctx->t + 1;
    for (int c = 0; c < 2; ++c) {
        const int form = sweep_form(ctx);
        SweepArgs a = sweep_args(ctx, c, true);
        a.t_fixed = t_known > 0 ? t_known : 0;
        launch_halfstep(ctx, a, form);
        CKL();
        ++ctx->sim_halfstep_launches;
    }
    if (e0 && e1) {
        cudaEventRecord(e1, ctx->s);
        ctx->ev_sim.emplace_back(e0, e1);
    }
    // The stop kernels see the worklist's units as lane groups of two.
    const StopWindow win = stop_window(ctx);
    launch_stop_targeted(2, ctx->Rp / 2, ctx->Rp, ctx->d_of_block,
                         stop_grid(ctx, 2, kTargetedCtasPerSm),
                         ctx->ctl, ctx->work,
                         ctx->work_stride, ctx->es, ctx->inb, ctx->Nsp, ctx->eacc, ctx->ecur,
                         ctx->sigma, ctx->running, ctx->stop, ctx->tcount, ctx->e_last, t_known,
                         ctx->s, &win);
    CKL();
    launch_stop_rest(g.nblk, ctx->Rp / 2, 2, ctx->Rp, ctx->opt.n_max, ctx->d_of_block,
                     stop_grid(ctx, 1, kClosingCtasPerSm), ctx->ctl, ctx->work, ctx->work, ctx->work_stride, ctx->Nsp,
                     ctx->running, ctx->stop, ctx->tcount, ctx->sim_cond, t_known, ctx->s);
    CKL();
    ctx->t += 1;
    return MPR_OK;
}

// E_b of every (block, realization) recomputed from the state (after the
// state was overwritten through the API).
mpr_status refresh_energies(mpr_ctx* ctx) {
    TRY(energy_pass(ctx));
    ctx->energy_dirty = false;
    return MPR_OK;
}

// One bisection iteration k (Sec. 2.1 energy matching per block): midpoints
// and median fallback, fresh start, E_b from scratch, n_eq + n_meas sweeps
// with the energies of the last n_meas summed, bisection step. With cond != 0
// the last kernel also sets the graph's loop condition.
// One calibration half-step of colour c at sweep index sw (k_sweep_flat),
// timed with events when asked and profiling is on.
mpr_status flat_halfstep(mpr_ctx* ctx, int c, int sw, bool timed) {
    SweepArgs a = sweep_args(ctx, c, false);
    a.t_fixed = sw;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed && ctx->opt.profile) {
        e0 = get_event(ctx);
        e1 = get_event(ctx);
        if (e0) cudaEventRecord(e0, ctx->s);
    }
    launch_sweep_flat(a, ctx->G, ctx->n_gap[c], ctx->s);
    CKL();
    if (e0 && e1) {
        cudaEventRecord(e1, ctx->s);
        ctx->ev_cal.emplace_back(e0, e1);
    }
    ++ctx->cal_halfstep_launches;
    return MPR_OK;
}

// The calibration chains (fresh from the block-mean start, or continued) run
// n_eq + n_meas sweeps at the current beta with random-stream tag `tag`; the
// block-energy moments of the measured sweeps land in ctx->mom.
mpr_status moments_run(mpr_ctx* ctx, uint32_t tag, bool restart, int n_eq, int n_meas) {
    const Geom& g = ctx->g;
    const int chains = ctx->opt.cal_chains;
    if (restart || !ctx->chains_valid || ctx->storage != MPR_STORE_F32 || ctx->R != chains) {
        ctx->r_off = 0;
        ctx->r_even = 0;
        TRY(ensure_batch(ctx, chains, ctx->opt.group, MPR_STORE_F32));
        ctx->R = chains;
        launch_fill_samples(g, ctx->mask, ctx->dang, ctx->ang, MPR_STORE_F32, ctx->G,
                            ctx->groups, ctx->s);
        CKL();
        TRY(init_batch_state(ctx));
        ctx->chains_valid = true;
    }
    launch_set_tag(ctx->ctl, tag, ctx->s);
    CKL();
    TRY(energy_pass(ctx));
    CK(cudaMemsetAsync(ctx->msum, 0, 4 * (size_t)g.nblk * sizeof(double), ctx->s));
    for (int sw = 1; sw <= n_eq + n_meas; ++sw) {
        for (int c = 0; c < 2; ++c) TRY(flat_halfstep(ctx, c, sw, true));
        launch_cal_step(g.nblk, ctx->Rp, chains, n_eq, sw, ctx->ctl, ctx->inb, ctx->eacc,
                        ctx->ecur, ctx->ebar, ctx->s);
        CKL();
        if (sw > n_eq) {
            launch_cal_moments(g.nblk, g.nbx, ctx->Rp, chains, ctx->ecur, ctx->msum, ctx->s);
            CKL();
        }
    }
    launch_moments_final(g.nblk, g.nbx, 1.0 / ((double)n_meas * (double)chains), ctx->Nb,
                         ctx->msum, ctx->mom, ctx->s);
    CKL();
    ctx->moments_valid = true;
    ctx->cal_updates += (int64_t)(n_eq + n_meas) * chains * (ctx->n_gap[0] + ctx->n_gap[1]);
    return MPR_OK;
}

// Damped Newton calibration (cal_method 1).
mpr_status calibration_newton(mpr_ctx* ctx) {
    const Geom& g = ctx->g;
    const mpr_options& o = ctx->opt;
    launch_newton_init(g.nblk, o.t_init, o.t_lo, o.t_hi, ctx->T, ctx->lo, ctx->hi, ctx->s);
    CKL();
    for (int k = 0; k < o.n_newton; ++k) {
        launch_cal_fill(ctx->sl, g.nbx, ctx->Nsp_cal, ctx->T, ctx->beta, ctx->s);   // median, beta
        CKL();
        TRY(moments_run(ctx, (uint32_t)(1 + k), k == 0, o.n_eq, o.n_meas));
        launch_newton_update(g.nblk, ctx->es, ctx->Nsp_cal, ctx->Nb, ctx->mom, ctx->T, (double)o.t_lo,
                             (double)o.t_hi, ctx->s);
        CKL();
    }
    launch_cal_fill(ctx->sl, g.nbx, ctx->Nsp_cal, ctx->T, ctx->beta, ctx->s);
    CKL();
    return MPR_OK;
}

// Temperatures of the default unconditional curve: geometric from
// kCurveTmin to kCurveTmax.
constexpr double kCurveTmin = 0.002, kCurveTmax = 1.25;

// Measured curves, kept for the process: the curve depends on q, J, the
// over-relaxation switch, n_eq and n_meas only (its random streams use the
// fixed key (0, 0)), so every context with the same parameters reads the
// same numbers, and the kernel runs once per parameter set.
struct CurveEntry {
    double q, J;
    int overrelax, n_eq, n_meas;
    float T[MPR_CURVE_POINTS];
    double e[MPR_CURVE_POINTS];
};
std::mutex g_curve_mu;
std::deque<CurveEntry> g_curves;

// The context's e(T) curve: set by the caller, or the default curve
// (MPR_CURVE_POINTS temperatures, the calibration's n_eq and n_meas),
// measured on the context's stream unless this process measured it before.
mpr_status ensure_curve(mpr_ctx* ctx) {
    if (!ctx->curve_T) TRY(dalloc(ctx, &ctx->curve_T, (size_t)kCurveMaxPoints));
    if (!ctx->curve_e) TRY(dalloc(ctx, &ctx->curve_e, (size_t)kCurveMaxPoints));
    if (ctx->curve_n > 0) return MPR_OK;
    const mpr_options& o = ctx->opt;
    std::lock_guard<std::mutex> lock(g_curve_mu);
    const CurveEntry* hit = nullptr;
    for (const CurveEntry& c : g_curves)
        if (c.q == o.q && c.J == o.J && c.overrelax == ctx->m.overrelax && c.n_eq == o.n_eq &&
            c.n_meas == o.n_meas)
            hit = &c;
    CurveEntry fresh{};
    if (!hit) {
        fresh.q = o.q;
        fresh.J = o.J;
        fresh.overrelax = ctx->m.overrelax;
        fresh.n_eq = o.n_eq;
        fresh.n_meas = o.n_meas;
        for (int k = 0; k < MPR_CURVE_POINTS; ++k)
            fresh.T[k] = (float)(kCurveTmin * std::pow(kCurveTmax / kCurveTmin,
                                                       (double)k / (double)(MPR_CURVE_POINTS - 1)));
        CK(cudaMemcpyAsync(ctx->curve_T, fresh.T, sizeof(fresh.T), cudaMemcpyHostToDevice, ctx->s));
        launch_energy_curve(ctx->curve_T, MPR_CURVE_POINTS, o.n_eq, o.n_meas, ctx->m, 0ull,
                            ctx->curve_e, ctx->s);
        CKL();
        CK(cudaMemcpyAsync(fresh.e, ctx->curve_e, sizeof(fresh.e), cudaMemcpyDeviceToHost, ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
        g_curves.push_back(fresh);
    } else {
        CK(cudaMemcpyAsync(ctx->curve_T, hit->T, sizeof(hit->T), cudaMemcpyHostToDevice, ctx->s));
        CK(cudaMemcpyAsync(ctx->curve_e, hit->e, sizeof(hit->e), cudaMemcpyHostToDevice, ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
    }
    ctx->curve_n = MPR_CURVE_POINTS;
    return MPR_OK;
}

// The calibration's warp-form half-step needs this many (block, chain pair)
// units per SM (two waves of 32 resident warps) before it replaces the flat
// form on a long list.
constexpr int kCalWarpUnitsPerSm = 64;

// warm_first: the iteration's points come from the curve (launch_warm_points)
// instead of the bracket. first: the iteration is the calibration's first
// (with cal_continue >= 0 only the first restarts the chains; the others
// continue them and run cal_continue equilibration sweeps instead of n_eq).
mpr_status calibration_iteration(mpr_ctx* ctx, double inv_count, cudaGraphConditionalHandle cond,
                                 bool timed, bool warm_first = false, bool first = true) {
    const Geom& g = ctx->g;
    const mpr_options& o = ctx->opt;
    const int pts = o.cal_points;
    if (warm_first) {
        launch_warm_points(g.nblk, pts, ctx->Nsp_cal, ctx->es, ctx->curve_T, ctx->curve_e,
                           ctx->curve_n, (double)o.cal_warm, ctx->T, ctx->T2, ctx->Tk, ctx->ctl,
                           ctx->s);
        CKL();
    }
    if (pts > 2) {
        if (!warm_first) {
            launch_kpts_mid(g.nblk, pts, ctx->Nsp_cal, ctx->lo, ctx->hi, ctx->Tk, ctx->ctl, ctx->s);
            CKL();
        }
        for (int p = 0; p < pts; ++p) {
            launch_cal_fill(ctx->sl, g.nbx, ctx->Nsp_cal, ctx->Tk + (size_t)p * g.nblk,
                            ctx->betak + (size_t)p * g.nblk, ctx->s);
            CKL();
        }
    } else if (pts == 2) {
        if (!warm_first) {
            launch_kcal_mid(g.nblk, ctx->Nsp_cal, ctx->lo, ctx->hi, ctx->T, ctx->T2, ctx->ctl,
                            ctx->s);
            CKL();
        }
        launch_cal_fill(ctx->sl, g.nbx, ctx->Nsp_cal, ctx->T2, ctx->beta2, ctx->s);
        CKL();
    } else {
        launch_cal_mid(g.nblk, ctx->Nsp_cal, ctx->lo, ctx->hi, ctx->T, ctx->ctl, ctx->s);
        CKL();
    }
    if (pts <= 2) {
        launch_cal_fill(ctx->sl, g.nbx, ctx->Nsp_cal, ctx->T, ctx->beta, ctx->s);
        CKL();
    }
    const size_t blk = (size_t)g.nblk * ctx->Rp;
    const bool restart = first || o.cal_continue < 0;
    if (restart) {
        TRY(init_batch_state(ctx));
        // Every restart is from the same state, so E_b of the start (computed
        // once, before the first iteration) is copied. Continued chains keep
        // their state and the E_b the last sweep's fold left in ecur.
        CK(cudaMemcpyAsync(ctx->ecur, ctx->ecur0, blk * sizeof(double),
                           cudaMemcpyDeviceToDevice, ctx->s));
    }
    CK(cudaMemsetAsync(ctx->eacc, 0, 2 * blk * sizeof(double), ctx->s));
    // Sweep sw's changes go to eacc buffer sw & 1; the colour-0 launch of
    // sweep sw + 1 folds them (extra CTAs), the last sweep's fold runs alone.
    const int n_eq = restart ? o.n_eq : o.cal_continue;
    const int n_sw = n_eq + o.n_meas;
    // Half-step form: one thread per (entry, pair) while a colour's list is a
    // few waves, one warp per (block, pair) unit for longer lists that also
    // hold enough units to fill the GPU with warps (a large field of few
    // blocks would leave it a fraction of a wave of long-running warps).
    const int64_t flat_threads = std::max(ctx->n_gap[0], ctx->n_gap[1]) * (ctx->G / 2);
    const int64_t units = (int64_t)g.nblk * ctx->groups * (ctx->G / 2);
    const bool warp_form =
        o.cal_sweep == 2 || (o.cal_sweep == 0 && flat_threads >= (1 << 20) &&
                             units >= (int64_t)kCalWarpUnitsPerSm * ctx->n_sm);
    for (int sw = 1; sw <= n_sw; ++sw) {
        for (int c = 0; c < 2; ++c) {
            SweepArgs a = sweep_args(ctx, c, false);
            a.t_fixed = sw;
            a.eacc = ctx->eacc + (size_t)(sw & 1) * blk;
            a.beta_odd = pts == 2 ? ctx->beta2 : nullptr;
            a.beta_pts = pts > 2 ? ctx->betak : nullptr;
            a.n_pts = pts;
            FoldArgs f{};
            if (c == 0 && sw > 1) {
                f.ctas = (g.nblk + 255) / 256;
                f.nblk = g.nblk;
                f.Rp = ctx->Rp;
                f.chains = o.cal_chains;
                f.points = pts;
                f.ebar_odd = ctx->ebar2;
                f.ebar_pts = ctx->ebark;
                f.measure = (sw - 1) > n_eq;
                f.inb = ctx->inb;
                f.eacc = ctx->eacc + (size_t)((sw - 1) & 1) * blk;
                f.ecur = ctx->ecur;
                f.ebar = ctx->ebar;
            }
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (timed && ctx->opt.profile) {
                e0 = get_event(ctx);
                e1 = get_event(ctx);
                if (e0) cudaEventRecord(e0, ctx->s);
            }
            if (warp_form) launch_sweep_cal(a, ctx->G, ctx->s, f.ctas ? &f : nullptr);
            else launch_sweep_flat(a, ctx->G, ctx->n_gap[c], ctx->s, f.ctas ? &f : nullptr);
            CKL();
            if (e0 && e1) {
                cudaEventRecord(e1, ctx->s);
                ctx->ev_cal.emplace_back(e0, e1);
            }
            ++ctx->cal_halfstep_launches;
        }
    }
    launch_cal_step(g.nblk, ctx->Rp, o.cal_chains, n_eq, n_sw, ctx->ctl, ctx->inb,
                    ctx->eacc + (size_t)(n_sw & 1) * blk, ctx->ecur, ctx->ebar, ctx->s, pts,
                    ctx->ebar2, ctx->ebark);
    CKL();
    if (pts > 2)
        launch_kpts_update(g.nblk, pts, inv_count, ctx->es, ctx->Nsp_cal, ctx->Tk, ctx->lo,
                           ctx->hi, ctx->ebark, ctx->ctl, o.n_bisect, cond, ctx->s);
    else if (pts == 2)
        launch_kcal_update(g.nblk, inv_count, ctx->es, ctx->Nsp_cal, ctx->T, ctx->T2, ctx->lo, ctx->hi,
                           ctx->ebar, ctx->ebar2, ctx->ctl, o.n_bisect, cond, ctx->s);
    else
        launch_cal_update(g.nblk, inv_count, ctx->es, ctx->Nsp_cal, ctx->T, ctx->lo, ctx->hi,
                          ctx->ebar, ctx->ctl, o.n_bisect, cond, ctx->s);
    CKL();
    return MPR_OK;
}

// All iterations in one cooperative launch (mpr_persist.cu). Returns MPR_OK,
// MPR_ETIMEOUT (a barrier wait gave up), or `fallback` set when the launch was
// refused (then nothing ran and the graph path can take over).
mpr_status calibration_persistent(mpr_ctx* ctx, double inv_count, bool* fallback) {
    *fallback = false;
    const Geom& g = ctx->g;
    const mpr_options& o = ctx->opt;
    const int per_sm = cal_persistent_blocks_per_sm(ctx->G);
    if (!ctx->coop || per_sm < 1) {
        *fallback = true;
        return MPR_OK;
    }
    CalPersistArgs a{};
    a.sw = sweep_args(ctx, 0, false);
    a.sw.energy = 1;
    for (int c = 0; c < 2; ++c) {
        a.list[c] = ctx->list[c];
        a.start[c] = ctx->start[c];
        a.split[c] = ctx->split[c];
        a.n_list[c] = ctx->n_gap[c];
    }
    const size_t blk = (size_t)g.nblk * ctx->Rp;
    a.eacc2[0] = ctx->eacc;
    a.eacc2[1] = ctx->eacc + blk;
    a.Es = ctx->Es;
    a.es = ctx->es;
    a.inb = ctx->inb;
    a.Nsp = ctx->Nsp_cal;
    a.T = ctx->T;
    a.beta = ctx->beta;
    a.lo = ctx->lo;
    a.hi = ctx->hi;
    a.ebar = ctx->ebar;
    a.init_angle = ctx->init_angle;
    a.chains = o.cal_chains;
    a.n_eq = o.n_eq;
    a.n_meas = o.n_meas;
    a.n_bisect = o.n_bisect;
    a.random_init = o.init == MPR_INIT_RANDOM;
    a.inv_count = inv_count;
    a.bar = ctx->bar;
    a.spin_limit = (unsigned long long)o.wait_ms * 10000ull;   // ~100 ns per poll
    a.med = ctx->med;
    GridBarrier hb{0u, 0u, 0u, (unsigned int)o.barrier_test};
    CK(cudaMemcpyAsync(ctx->bar, &hb, sizeof(hb), cudaMemcpyHostToDevice, ctx->s));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (o.profile) {
        e0 = get_event(ctx);
        e1 = get_event(ctx);
        if (e0) cudaEventRecord(e0, ctx->s);
    }
    const cudaError_t le = launch_cal_persistent(a, ctx->G, ctx->n_sm * per_sm, ctx->s);
    if (le != cudaSuccess) {
        cudaGetLastError();
        if (e0) ctx->ev_pool.push_back(e0);
        if (e1) ctx->ev_pool.push_back(e1);
        *fallback = true;
        return MPR_OK;
    }
    ++ctx->launches;
    ctx->cal_halfstep_launches += 1;
    if (e0 && e1) {
        cudaEventRecord(e1, ctx->s);
        ctx->ev_cal.emplace_back(e0, e1);
    }
    CK(cudaMemcpyAsync(&hb, ctx->bar, sizeof(hb), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    if (hb.err)
        return fail(ctx, MPR_ETIMEOUT,
                    "calibration: a grid-barrier wait gave up after %d ms; the calibration "
                    "did not complete", o.wait_ms);
    return MPR_OK;
}

// The calibration's remaining n_iter iterations (up to n_bisect in all) as
// one CUDA graph: a device-side WHILE loop whose body is one iteration
// (captured once); the update kernel ends it once ctl->k reaches n_bisect.
// One launch, no host round trip per iteration.
mpr_status calibration_graph(mpr_ctx* ctx, double inv_count, int n_iter) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    mpr_status st = MPR_OK;
    cudaGraphConditionalHandle cond = 0;
    cudaGraphNodeParams p = {};
    cudaGraphNode_t node = nullptr;
    cudaGraph_t body = nullptr, captured = nullptr;
    const int64_t launches0 = ctx->launches, hs0 = ctx->cal_halfstep_launches;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) goto cuda_fail;
    if (cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
        goto cuda_fail;
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = cond;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p) != cudaSuccess) goto cuda_fail;
    body = p.conditional.phGraph_out[0];
    // Record on the private stream (the caller's may be the legacy default
    // stream, which cannot be captured); launch on the caller's stream.
    if (cudaStreamBeginCaptureToGraph(ctx->cap, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        goto cuda_fail;
    {
        cudaStream_t user = ctx->s;
        ctx->s = ctx->cap;
        st = calibration_iteration(ctx, inv_count, cond, false, false,
                                   ctx->opt.n_bisect - n_iter == 0);
        ctx->s = user;
    }
    if (cudaStreamEndCapture(ctx->cap, &captured) != cudaSuccess && st == MPR_OK) goto cuda_fail;
    if (st != MPR_OK) goto done;
    // The body ran once at capture time only as a recording; the loop runs
    // it n_bisect times.
    {
        const int64_t per_iter_launches = ctx->launches - launches0;
        const int64_t per_iter_hs = ctx->cal_halfstep_launches - hs0;
        ctx->launches = launches0 + per_iter_launches * n_iter;
        ctx->cal_halfstep_launches = hs0 + per_iter_hs * n_iter;
    }
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) goto cuda_fail;
    if (ctx->opt.profile) {
        e0 = get_event(ctx);
        e1 = get_event(ctx);
        if (e0) cudaEventRecord(e0, ctx->s);
    }
    if (cudaGraphLaunch(exec, ctx->s) != cudaSuccess) goto cuda_fail;
    if (e0 && e1) {
        cudaEventRecord(e1, ctx->s);
        ctx->ev_cal.emplace_back(e0, e1);
    }
    goto done;
cuda_fail: {
        cudaError_t e = cudaGetLastError();
        st = fail(ctx, MPR_ECUDA, "calibration graph: %s", cudaGetErrorString(e));
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(ctx->cap, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t tmp = nullptr;
            cudaStreamEndCapture(ctx->cap, &tmp);
            if (tmp && tmp != body) cudaGraphDestroy(tmp);
        }
    }
done:
    if (exec) {
        cudaStreamSynchronize(ctx->s);
        cudaGraphExecDestroy(exec);
    }
    if (graph) cudaGraphDestroy(graph);
    return st;
}

}  // namespace

// ------------------------------------------------------------------ public --
extern "C" {

void mpr_default_options(mpr_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->q = 0.5;
    o->J = 1.0;
    o->seed = 0;
    o->slice_id = 0;
    o->n_max = 200;
    o->n_eq = 25;
    o->n_meas = 20;
    o->n_bisect = 24;
    o->cal_chains = 1;
    o->t_lo = 1e-4f;
    o->t_hi = 2.0f;
    o->overrelax = 1;
    o->init = MPR_INIT_BLOCK_MEAN;
    o->storage = MPR_STORE_F32;
    o->group = 0;
    o->profile = 0;
    o->cal_mode = 0;
    o->wait_ms = 2000;
    o->barrier_test = 0;
    o->cal_method = 0;
    o->n_newton = 6;
    o->t_init = 0.1f;
    o->sim_graph = 0;
    o->cal_points = 1;
    o->sim_tail = 0;
    o->sweep_form = -1;
    o->pair_tail = 4096;
    o->sweep_form_bulk = -1;
    o->stop_rule = MPR_STOP_CROSS;
    o->n_fit = 20;
    o->n_f = 5;
    o->cal_warm = 0.0f;
    o->alloc_test = 0;
    o->cal_continue = -1;
    o->cal_sweep = 0;
    o->cuda_stream = nullptr;
}

const char* mpr_status_string(mpr_status s) {
    switch (s) {
        case MPR_OK: return "ok";
        case MPR_EINVAL: return "invalid argument";
        case MPR_ENOMEM: return "out of memory";
        case MPR_ECUDA: return "CUDA error";
        case MPR_ENOSAMPLES: return "no sample pair";
        case MPR_ETIMEOUT: return "device wait timed out";
        case MPR_ESTATE: return "call out of order";
    }
    return "unknown status";
}

const char* mpr_last_error(const mpr_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

void mpr_release_cached_memory(void) { pool_trim(); }

void mpr_destroy(mpr_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->s);
    for (auto& pr : ctx->ev_sim) ctx->ev_pool.insert(ctx->ev_pool.end(), {pr.first, pr.second});
    for (auto& pr : ctx->ev_cal) ctx->ev_pool.insert(ctx->ev_pool.end(), {pr.first, pr.second});
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    for (void* p : ctx->owned) pool_free(p, ctx->s);
    cudaStreamSynchronize(ctx->s);
    pinned_release(ctx->h_counters);   // h_ctl lies in the same slot
    delete ctx;
}

}  // extern "C"

namespace {

// Canvas mask: 1 gap / 0 sample inside every slice's field (any nonzero
// input is a gap), 2 everywhere else.
__global__ void k_mask_normalize(Geom g, Slices sl, uint8_t* __restrict__ mask) {
    const int64_t n = (int64_t)g.H * g.W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / g.W), x = (int)(i % g.W);
        const int s = sl.of_block[(y / g.lb) * g.nbx + x / g.lb];
        bool inside = false;
        if (s >= 0) {
            const int4 rc = sl.rect[s];
            inside = y < rc.x + rc.z && x < rc.y + rc.w;
        }
        mask[i] = inside ? (mask[i] != 0 ? MASK_GAP : 0) : MASK_ABSENT;
    }
}

struct SliceDesc {
    int y0, x0, H, W;
};


// Host memory (pinned or pageable), as opposed to device or managed memory.
bool is_host_pointer(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

// Copies a caller's h x w field (contiguous rows, es-byte elements) into the
// canvas at element offset `off` (to_canvas) or out of it. Device or managed
// memory: one row-strided copy. Host memory goes through `stage`, a device
// buffer of at least h w es bytes, so that the host link carries one
// contiguous copy: a row-strided copy straight from or to host memory moves
// one row (a few KB) per transfer and measured a few GB/s (0.2-0.3 s for the
// 1.3 GB of the 256-field batch's inputs).
mpr_status canvas_copy(mpr_ctx* ctx, bool to_canvas, void* canvas, size_t off, const void* in,
                       void* out, int h, int w, size_t es, void* stage) {
    const size_t pitch = (size_t)ctx->g.W * es, row = (size_t)w * es;
    uint8_t* c = static_cast<uint8_t*>(canvas) + off * es;
    if (to_canvas) {
        if (stage) {
            CK(cudaMemcpyAsync(stage, in, row * h, cudaMemcpyDefault, ctx->s));
            in = stage;
        }
        CK(cudaMemcpy2DAsync(c, pitch, in, row, row, h, cudaMemcpyDefault, ctx->s));
    } else {
        CK(cudaMemcpy2DAsync(stage ? stage : out, row, c, pitch, row, h, cudaMemcpyDefault, ctx->s));
        if (stage) CK(cudaMemcpyAsync(out, stage, row * h, cudaMemcpyDefault, ctx->s));
    }
    return MPR_OK;
}

// A device staging buffer for canvas_copy when one of the n pointers is host
// memory (nullptr otherwise): room for the largest of the context's fields.
mpr_status host_stage(mpr_ctx* ctx, const void* const* ptrs, int n, size_t es, uint8_t** stage) {
    *stage = nullptr;
    bool host = false;
    for (int k = 0; k < n && !host; ++k) host = is_host_pointer(ptrs[k]);
    if (!host) return MPR_OK;
    size_t big = 0;
    for (const int4& rc : ctx->h_rect) big = std::max(big, (size_t)rc.z * rc.w);
    return dalloc(ctx, stage, big * es);
}

// Allocation, slice tables, transform, Eq. 2 statistics and gap lists of a
// canvas holding `desc` fields; `upload` copies the inputs into ctx->values
// and ctx->mask (canvas layout; mask is normalised afterwards).
template <class Upload>
mpr_status create_impl(const mpr_options* opt_in, int H, int W, int lb,
                       const std::vector<SliceDesc>& desc, Upload upload, mpr_ctx** out) {
    mpr_ctx* ctx = new (std::nothrow) mpr_ctx();
    if (!ctx) return MPR_ENOMEM;
    auto bail = [&](mpr_status st) {
        mpr_destroy(ctx);
        return st;
    };
    if (opt_in) ctx->opt = *opt_in; else mpr_default_options(&ctx->opt);
    if (check_opts(ctx, ctx->opt) != MPR_OK) return bail(MPR_EINVAL);
    if (H < 1 || W < 1 || H > MAX_SIDE || W > MAX_SIDE || lb < 1) return bail(MPR_EINVAL);
    Geom& g = ctx->g;
    g.H = H;
    g.W = W;
    g.Wh = (W + 1) / 2;
    g.lb = lb;
    g.nbx = (W + lb - 1) / lb;
    g.nby = (H + lb - 1) / lb;
    if ((int64_t)g.nbx * g.nby > MAX_BLOCKS) return bail(MPR_EINVAL);
    g.nblk = g.nbx * g.nby;
    const int ns = (int)desc.size();
    ctx->n_slices = ns;
    ctx->m.q = (float)ctx->opt.q;
    ctx->m.J = (float)ctx->opt.J;
    ctx->m.inv_q = (float)(1.0 / ctx->opt.q);
    ctx->m.overrelax = ctx->opt.overrelax ? 1 : 0;
    ctx->rng.key0 = (uint32_t)(ctx->opt.seed & 0xffffffffu);
    ctx->rng.key1 = (uint32_t)(ctx->opt.seed >> 32) ^ ctx->opt.slice_id;
    for (int r = 0; r < 10; ++r) ctx->rng.rk0[r] = ctx->rng.key0 + (uint32_t)r * 0x9E3779B9u;
    ctx->s = (cudaStream_t)ctx->opt.cuda_stream;

    if (cudaGetDevice(&ctx->device) != cudaSuccess) return bail(MPR_ECUDA);
    if (cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess)
        return bail(MPR_ECUDA);
    cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
    if (ctx->n_sm < 1) ctx->n_sm = 1;

    const int64_t n = (int64_t)H * W;
    const size_t plane = (size_t)H * g.Wh;
    mpr_status st;
#define ST(x) do { st = (x); if (st != MPR_OK) return bail(st); } while (0)
    ST(dalloc(ctx, &ctx->values, n));
    ST(dalloc(ctx, &ctx->mask, n));
    ST(dalloc(ctx, &ctx->dang, 2 * plane));
    ST(dalloc(ctx, &ctx->sum, 2 * plane));
    ST(dalloc(ctx, &ctx->Es, g.nblk));
    ST(dalloc(ctx, &ctx->msum, 4 * (size_t)g.nblk));
    ST(dalloc(ctx, &ctx->mom, 4 * (size_t)g.nblk));
    ST(dalloc(ctx, &ctx->es, g.nblk));
    ST(dalloc(ctx, &ctx->inb, g.nblk));
    ST(dalloc(ctx, &ctx->Nsp, g.nblk));
    ST(dalloc(ctx, &ctx->Nsp_cal, g.nblk));
    ST(dalloc(ctx, &ctx->Nb, g.nblk));
    ST(dalloc(ctx, &ctx->nsamp, g.nblk));
    ST(dalloc(ctx, &ctx->ngap_c[0], g.nblk));
    ST(dalloc(ctx, &ctx->ngap_c[1], g.nblk));
    ST(dalloc(ctx, &ctx->ngap, g.nblk));
    ST(dalloc(ctx, &ctx->ssum, g.nblk));
    ST(dalloc(ctx, &ctx->init_angle, g.nblk));
    ST(dalloc(ctx, &ctx->T, g.nblk));
    ST(dalloc(ctx, &ctx->beta, g.nblk));
    ST(dalloc(ctx, &ctx->lo, g.nblk));
    ST(dalloc(ctx, &ctx->hi, g.nblk));
    ST(dalloc(ctx, &ctx->ebar, g.nblk));
    ST(dalloc(ctx, &ctx->T2, g.nblk));
    ST(dalloc(ctx, &ctx->beta2, g.nblk));
    ST(dalloc(ctx, &ctx->ebar2, g.nblk));
    ST(dalloc(ctx, &ctx->start[0], g.nblk + 1));
    ST(dalloc(ctx, &ctx->start[1], g.nblk + 1));
    ST(dalloc(ctx, &ctx->split[0], g.nblk));
    ST(dalloc(ctx, &ctx->split[1], g.nblk));
    ST(dalloc(ctx, &ctx->counters, 4));
    ST(dalloc(ctx, &ctx->mm, 2 * (size_t)ns));
    ST(dalloc(ctx, &ctx->err_buf, 2 * (size_t)ns));
    ST(dalloc(ctx, &ctx->ctl, 1));
    ST(dalloc(ctx, &ctx->bar, 1));
    ST(dalloc(ctx, &ctx->med, 1));
    ST(dalloc(ctx, &ctx->d_rect, ns));
    ST(dalloc(ctx, &ctx->d_blk, ns));
    ST(dalloc(ctx, &ctx->d_of_block, g.nblk));
    ST(dalloc(ctx, &ctx->d_key1, ns));
    ST(dalloc(ctx, &ctx->d_zmin, ns));
    ST(dalloc(ctx, &ctx->d_zmax, ns));
    ST(dalloc(ctx, &ctx->d_degen, ns));
    cudaDeviceGetAttribute(&ctx->coop, cudaDevAttrCooperativeLaunch, ctx->device);
    {
        // One pinned slot: the four counters, then the Control mirror.
        static_assert(64 + sizeof(Control) <= kPinnedSlot, "pinned slot too small");
        uint8_t* slot = static_cast<uint8_t*>(pinned_slot());
        if (!slot) return bail(MPR_ENOMEM);
        ctx->h_counters = reinterpret_cast<unsigned long long*>(slot);
        ctx->h_ctl = reinterpret_cast<Control*>(slot + 64);
    }

    // Slice tables: rectangles, block rectangles, slice of every block, keys.
    std::vector<int4> rect(ns), blk(ns);
    std::vector<int32_t> of_block(g.nblk, -1);
    std::vector<uint32_t> key1(ns);
    for (int k = 0; k < ns; ++k) {
        const SliceDesc& d = desc[k];
        rect[k] = make_int4(d.y0, d.x0, d.H, d.W);
        const int by0 = d.y0 / lb, bx0 = d.x0 / lb;
        const int nby = (d.H + lb - 1) / lb, nbx = (d.W + lb - 1) / lb;
        blk[k] = make_int4(by0, bx0, nby, nbx);
        for (int by = by0; by < by0 + nby; ++by)
            for (int bx = bx0; bx < bx0 + nbx; ++bx) of_block[(size_t)by * g.nbx + bx] = k;
        key1[k] = (uint32_t)(ctx->opt.seed >> 32) ^ (ctx->opt.slice_id + (uint32_t)k);
    }
    ctx->h_rect = rect;
    if (cudaMemcpyAsync(ctx->d_rect, rect.data(), ns * sizeof(int4), cudaMemcpyHostToDevice, ctx->s) ||
        cudaMemcpyAsync(ctx->d_blk, blk.data(), ns * sizeof(int4), cudaMemcpyHostToDevice, ctx->s) ||
        cudaMemcpyAsync(ctx->d_of_block, of_block.data(), g.nblk * 4, cudaMemcpyHostToDevice,
                        ctx->s) ||
        cudaMemcpyAsync(ctx->d_key1, key1.data(), ns * 4, cudaMemcpyHostToDevice, ctx->s))
        return bail(MPR_ECUDA);
    ctx->sl = Slices{ns,          rect[0],     key1[0],    ctx->d_rect, ctx->d_blk, ctx->d_of_block,
                     ctx->d_key1, ctx->d_zmin, ctx->d_zmax, ctx->d_degen};

    {
        const mpr_status us = upload(ctx);
        if (us != MPR_OK) return bail(us);
    }
    k_mask_normalize<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, ctx->s>>>(
        g, ctx->sl, ctx->mask);
    ++ctx->launches;
    // z_min / z_max over the samples of every slice.
    {
        std::vector<uint32_t> mm(2 * (size_t)ns);
        for (int k = 0; k < ns; ++k) { mm[2 * k] = 0xffffffffu; mm[2 * k + 1] = 0u; }
        if (cudaMemcpyAsync(ctx->mm, mm.data(), mm.size() * 4, cudaMemcpyHostToDevice, ctx->s) !=
            cudaSuccess)
            return bail(MPR_ECUDA);
        launch_minmax(g, ctx->d_of_block, ctx->values, ctx->mask, ctx->mm, ctx->s);
        ++ctx->launches;
        if (cudaMemcpyAsync(mm.data(), ctx->mm, mm.size() * 4, cudaMemcpyDeviceToHost, ctx->s) !=
                cudaSuccess ||
            cudaStreamSynchronize(ctx->s) != cudaSuccess)
            return bail(MPR_ECUDA);
        ctx->h_zmin.assign(ns, 0.0);
        ctx->h_zmax.assign(ns, 0.0);
        ctx->h_degen.assign(ns, 1);
        for (int k = 0; k < ns; ++k) {
            if (mm[2 * k] == 0xffffffffu) continue;   // no sample in the slice
            ctx->h_zmin[k] = (double)ord2f(mm[2 * k]);
            ctx->h_zmax[k] = (double)ord2f(mm[2 * k + 1]);
            ctx->h_degen[k] = !(ctx->h_zmax[k] > ctx->h_zmin[k]);
        }
        ctx->zmin = ctx->h_zmin[0];
        ctx->zmax = ctx->h_zmax[0];
        ctx->degenerate = 1;     // every slice constant: nothing to calibrate
        for (int k = 0; k < ns; ++k) ctx->degenerate &= ctx->h_degen[k];
        if (cudaMemcpyAsync(ctx->d_zmin, ctx->h_zmin.data(), ns * 8, cudaMemcpyHostToDevice, ctx->s) ||
            cudaMemcpyAsync(ctx->d_zmax, ctx->h_zmax.data(), ns * 8, cudaMemcpyHostToDevice, ctx->s) ||
            cudaMemcpyAsync(ctx->d_degen, ctx->h_degen.data(), ns * 4, cudaMemcpyHostToDevice,
                            ctx->s))
            return bail(MPR_ECUDA);
    }
    launch_layout(g, ctx->sl, ctx->values, ctx->mask, ctx->dang, ctx->s);
    launch_block_stats(g, ctx->sl, ctx->values, ctx->mask, ctx->opt.q, ctx->opt.J, ctx->Es,
                       ctx->Nsp, ctx->Nb, ctx->ssum, ctx->nsamp, ctx->ngap_c[0], ctx->ngap_c[1],
                       ctx->s);
    launch_scan(ctx->ngap_c[0], g.nblk, ctx->start[0], ctx->s);
    launch_scan(ctx->ngap_c[1], g.nblk, ctx->start[1], ctx->s);
    ctx->launches += 4;
    if (cudaPeekAtLastError() != cudaSuccess) return bail(MPR_ECUDA);

    // Host-side bookkeeping: list sizes, initial angles, sample-pair check.
    std::vector<int32_t> s0(g.nblk + 1), s1(g.nblk + 1), nsp(g.nblk), nsm(g.nblk), ng0(g.nblk),
        ng1(g.nblk), nbv(g.nblk);
    std::vector<double> ssum(g.nblk), esv(g.nblk);
    if (cudaMemcpyAsync(s0.data(), ctx->start[0], s0.size() * 4, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(s1.data(), ctx->start[1], s1.size() * 4, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(nsp.data(), ctx->Nsp, nsp.size() * 4, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(nsm.data(), ctx->nsamp, nsm.size() * 4, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(ng0.data(), ctx->ngap_c[0], ng0.size() * 4, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(ng1.data(), ctx->ngap_c[1], ng1.size() * 4, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(ssum.data(), ctx->ssum, ssum.size() * 8, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(esv.data(), ctx->Es, esv.size() * 8, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaMemcpyAsync(nbv.data(), ctx->Nb, nbv.size() * 4, cudaMemcpyDeviceToHost, ctx->s) ||
        cudaStreamSynchronize(ctx->s))
        return bail(MPR_ECUDA);
    ctx->n_gap[0] = s0[g.nblk];
    ctx->n_gap[1] = s1[g.nblk];
    // Per slice: sample pairs (Eq. 2 needs one), gap sites, global sample mean.
    std::vector<int64_t> pairs(ns, 0), samples(ns, 0);
    std::vector<double> gsum(ns, 0.0);
    ctx->h_ngap.assign(ns, 0);
    std::vector<float> init(g.nblk, 0.0f);
    std::vector<int32_t> ng(g.nblk);
    for (int b = 0; b < g.nblk; ++b) {
        ng[b] = ng0[b] + ng1[b];
        const int k = of_block[b];
        if (k < 0) continue;
        pairs[k] += nsp[b];
        samples[k] += nsm[b];
        gsum[k] += ssum[b];
        ctx->h_ngap[k] += ng[b];
    }
    for (int k = 0; k < ns; ++k)
        if (pairs[k] == 0 && ctx->h_ngap[k] > 0) {
            mpr_destroy(ctx);
            return MPR_ENOSAMPLES;
        }
    for (int b = 0; b < g.nblk; ++b) {
        const int k = of_block[b];
        if (k < 0) continue;
        const double gmean = samples[k] ? gsum[k] / (double)samples[k] : 0.0;
        init[b] = (float)(nsm[b] > 0 ? ssum[b] / (double)nsm[b] : gmean);
    }
    std::vector<double> es_h(g.nblk), inb_h(g.nblk);
    std::vector<int32_t> nsp_cal(g.nblk);
    for (int b = 0; b < g.nblk; ++b) {
        es_h[b] = nsp[b] > 0 ? esv[b] / (double)nsp[b] : 0.0;
        inb_h[b] = nbv[b] > 0 ? 1.0 / (double)nbv[b] : 0.0;
        nsp_cal[b] = ng[b] > 0 ? nsp[b] : 0;
    }
    ST(dalloc(ctx, &ctx->list[0], ctx->n_gap[0]));
    ST(dalloc(ctx, &ctx->list[1], ctx->n_gap[1]));
    if (cudaMemcpyAsync(ctx->init_angle, init.data(), g.nblk * 4, cudaMemcpyHostToDevice, ctx->s) ||
        cudaMemcpyAsync(ctx->es, es_h.data(), g.nblk * 8, cudaMemcpyHostToDevice, ctx->s) ||
        cudaMemcpyAsync(ctx->inb, inb_h.data(), g.nblk * 8, cudaMemcpyHostToDevice, ctx->s) ||
        cudaMemcpyAsync(ctx->ngap, ng.data(), g.nblk * 4, cudaMemcpyHostToDevice, ctx->s) ||
        cudaMemcpyAsync(ctx->Nsp_cal, nsp_cal.data(), g.nblk * 4, cudaMemcpyHostToDevice, ctx->s))
        return bail(MPR_ECUDA);
    launch_build_lists(g, ctx->d_of_block, ctx->mask, ctx->start[0], ctx->start[1], ctx->list[0],
                       ctx->list[1], ctx->split[0], ctx->split[1], ctx->s);
    ++ctx->launches;
    if (cudaMemsetAsync(ctx->sum, 0, 2 * plane * sizeof(double), ctx->s) ||
        cudaMemsetAsync(ctx->ctl, 0, sizeof(Control), ctx->s) ||
        cudaMemsetAsync(ctx->counters, 0, 4 * sizeof(unsigned long long), ctx->s) ||
        cudaPeekAtLastError() || cudaStreamSynchronize(ctx->s))
        return bail(MPR_ECUDA);
#undef ST
    *out = ctx;
    return MPR_OK;
}

}  // namespace

extern "C" {

mpr_status mpr_create(const mpr_grid* grid, const uint8_t* mask_in, const float* values_in,
                      const mpr_options* opt_in, mpr_ctx** out) {
    PhaseRange phase_range("mpr_create");
    if (!out) return MPR_EINVAL;
    *out = nullptr;
    if (!grid || !mask_in || !values_in) return MPR_EINVAL;
    const int H = grid->height, W = grid->width;
    if (H < 1 || W < 1 || H > MAX_SIDE || W > MAX_SIDE || grid->block < 1) return MPR_EINVAL;
    const size_t n = (size_t)H * W;
    auto upload = [&](mpr_ctx* ctx) -> mpr_status {
        if (copy_in(ctx, ctx->values, values_in, n * sizeof(float)) != MPR_OK) return MPR_ECUDA;
        return copy_in(ctx, ctx->mask, mask_in, n);
    };
    return create_impl(opt_in, H, W, grid->block, {SliceDesc{0, 0, H, W}}, upload, out);
}

mpr_status mpr_create_batch(int32_t n, const mpr_grid* grids, const uint8_t* const* masks,
                            const float* const* values, const mpr_options* opt_in,
                            mpr_ctx** out) {
    PhaseRange phase_range("mpr_create_batch");
    if (!out) return MPR_EINVAL;
    *out = nullptr;
    if (n < 1 || !grids || !masks || !values) return MPR_EINVAL;
    const int lb = grids[0].block;
    if (lb < 1) return MPR_EINVAL;
    for (int k = 0; k < n; ++k)
        if (grids[k].block != lb || grids[k].height < 1 || grids[k].width < 1 ||
            grids[k].height > MAX_SIDE || grids[k].width > MAX_SIDE || !masks[k] || !values[k])
            return MPR_EINVAL;
    // Shelf packing on a grid of L x L cells, L = l_b (2 l_b if l_b is odd,
    // so that every slice origin has y0 + x0 even): slices sorted by height,
    // placed left to right, a new shelf when the row is full.
    const int L = (lb % 2 == 0) ? lb : 2 * lb;
    auto up = [&](int v) { return (v + L - 1) / L * L; };
    std::vector<int> order(n);
    int64_t area = 0;
    int wmax = 0;
    for (int k = 0; k < n; ++k) {
        order[k] = k;
        area += (int64_t)up(grids[k].height) * up(grids[k].width);
        wmax = std::max(wmax, up(grids[k].width));
    }
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return grids[a].height > grids[b].height; });
    const int Wc = std::max(wmax, up((int)std::ceil(std::sqrt((double)area))));
    std::vector<SliceDesc> desc(n);
    int x = 0, y = 0, shelf = 0;
    for (int k : order) {
        const int hp = up(grids[k].height), wp = up(grids[k].width);
        if (x + wp > Wc) {
            y += shelf;
            x = 0;
            shelf = 0;
        }
        desc[k] = SliceDesc{y, x, grids[k].height, grids[k].width};
        x += wp;
        shelf = std::max(shelf, hp);
    }
    const int Hc = y + shelf;
    if (Hc > MAX_SIDE || Wc > MAX_SIDE) return MPR_EINVAL;
    auto upload = [&](mpr_ctx* ctx) -> mpr_status {
        const size_t nc = (size_t)ctx->g.H * ctx->g.W;
        if (cudaMemsetAsync(ctx->mask, 0, nc, ctx->s) != cudaSuccess ||
            cudaMemsetAsync(ctx->values, 0, nc * sizeof(float), ctx->s) != cudaSuccess)
            return MPR_ECUDA;
        uint8_t *sv = nullptr, *sm = nullptr;
        TRY(host_stage(ctx, reinterpret_cast<const void* const*>(values), n, sizeof(float), &sv));
        TRY(host_stage(ctx, reinterpret_cast<const void* const*>(masks), n, 1, &sm));
        mpr_status st = MPR_OK;
        for (int k = 0; k < n && st == MPR_OK; ++k) {
            const SliceDesc& d = desc[k];
            const size_t off = (size_t)d.y0 * ctx->g.W + d.x0;
            st = canvas_copy(ctx, true, ctx->values, off, values[k], nullptr, d.H, d.W,
                             sizeof(float), sv);
            if (st == MPR_OK)
                st = canvas_copy(ctx, true, ctx->mask, off, masks[k], nullptr, d.H, d.W, 1, sm);
        }
        dfree(ctx, sv);
        dfree(ctx, sm);
        return st;
    };
    return create_impl(opt_in, Hc, Wc, lb, desc, upload, out);
}

mpr_status mpr_get_info(const mpr_ctx* ctx, mpr_info* info) {
    if (!ctx || !info) return MPR_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->height = ctx->g.H;
    info->width = ctx->g.W;
    info->block = ctx->g.lb;
    info->nbx = ctx->g.nbx;
    info->nby = ctx->g.nby;
    info->nblk = ctx->g.nblk;
    info->n_gap = ctx->n_gap[0] + ctx->n_gap[1];
    info->n_gap_colour[0] = ctx->n_gap[0];
    info->n_gap_colour[1] = ctx->n_gap[1];
    info->zmin = ctx->zmin;
    info->zmax = ctx->zmax;
    info->degenerate = ctx->degenerate;
    info->calibrated = ctx->calibrated;
    info->realizations = ctx->realizations;
    info->batch = ctx->batch_open ? ctx->R : 0;
    info->group = ctx->G;
    info->gap_updates = ctx->gap_updates;
    info->cal_gap_updates = ctx->cal_updates;
    info->device_bytes = ctx->device_bytes;
    info->n_slices = ctx->n_slices;
    return MPR_OK;
}

mpr_status mpr_get_profile(mpr_ctx* ctx, mpr_profile* p) {
    if (!ctx || !p) return MPR_EINVAL;
    ctx->err.clear();
    CK(cudaStreamSynchronize(ctx->s));
    collect_events(ctx);
    std::memset(p, 0, sizeof(*p));
    p->kernel_launches = ctx->launches;
    p->sim_halfstep_launches = ctx->sim_halfstep_launches;
    p->cal_halfstep_launches = ctx->cal_halfstep_launches;
    p->sim_halfstep_ms = ctx->sim_halfstep_ms;
    p->cal_halfstep_ms = ctx->cal_halfstep_ms;
    p->sim_tail_launches = ctx->sim_tail_launches;
    p->sim_tail_updates = ctx->sim_tail_updates;
    p->sim_tail_ms = ctx->sim_tail_ms;
    return MPR_OK;
}

mpr_status mpr_get_block_stats(mpr_ctx* ctx, double* Es, int32_t* Nsp, int32_t* Nb,
                               float* mean_angle, int32_t* n_gap) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    const size_t nb = ctx->g.nblk;
    if (Es) TRY(copy_out(ctx, Es, ctx->Es, nb * 8));
    if (Nsp) TRY(copy_out(ctx, Nsp, ctx->Nsp, nb * 4));
    if (Nb) TRY(copy_out(ctx, Nb, ctx->Nb, nb * 4));
    if (mean_angle) TRY(copy_out(ctx, mean_angle, ctx->init_angle, nb * 4));
    if (n_gap) TRY(copy_out(ctx, n_gap, ctx->ngap, nb * 4));
    return MPR_OK;
}

mpr_status mpr_set_temperatures(mpr_ctx* ctx, const float* T) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    if (!T) return fail(ctx, MPR_EINVAL, "T is NULL");
    std::vector<float> h(ctx->g.nblk), bt(ctx->g.nblk);
    CK(cudaMemcpyAsync(h.data(), T, h.size() * 4, cudaMemcpyDefault, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    for (int b = 0; b < ctx->g.nblk; ++b) {
        if (!(h[b] > 0.0f) || !std::isfinite(h[b]))
            return fail(ctx, MPR_EINVAL, "temperature of block %d is not a positive number", b);
        bt[b] = 1.0f / h[b];
    }
    CK(cudaMemcpyAsync(ctx->T, h.data(), h.size() * 4, cudaMemcpyHostToDevice, ctx->s));
    CK(cudaMemcpyAsync(ctx->beta, bt.data(), bt.size() * 4, cudaMemcpyHostToDevice, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    ctx->calibrated = 1;
    ctx->sst = 0;
    return MPR_OK;
}

mpr_status mpr_get_temperatures(mpr_ctx* ctx, float* T) {
    if (!ctx || !T) return MPR_EINVAL;
    ctx->err.clear();
    if (!ctx->calibrated) return fail(ctx, MPR_ESTATE, "no temperatures yet");
    return copy_out(ctx, T, ctx->T, (size_t)ctx->g.nblk * 4);
}

mpr_status mpr_get_energy_curve(mpr_ctx* ctx, float* T_out, double* e_out, int32_t capacity,
                                int32_t* n_out) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    if (!T_out || !e_out || !n_out) return fail(ctx, MPR_EINVAL, "T_out, e_out and n_out are required");
    TRY(ensure_curve(ctx));
    if (capacity < ctx->curve_n)
        return fail(ctx, MPR_EINVAL, "capacity %d is below the curve's %d points", capacity,
                    ctx->curve_n);
    TRY(copy_out(ctx, T_out, ctx->curve_T, (size_t)ctx->curve_n * 4));
    TRY(copy_out(ctx, e_out, ctx->curve_e, (size_t)ctx->curve_n * 8));
    *n_out = ctx->curve_n;
    return MPR_OK;
}

mpr_status mpr_set_energy_curve(mpr_ctx* ctx, const float* T, const double* e, int32_t n) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    if (!T || !e) return fail(ctx, MPR_EINVAL, "T and e are required");
    if (n < 2 || n > kCurveMaxPoints)
        return fail(ctx, MPR_EINVAL, "a curve has 2 to %d points", kCurveMaxPoints);
    std::vector<float> hT(n);
    std::vector<double> he(n);
    CK(cudaMemcpyAsync(hT.data(), T, (size_t)n * 4, cudaMemcpyDefault, ctx->s));
    CK(cudaMemcpyAsync(he.data(), e, (size_t)n * 8, cudaMemcpyDefault, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    for (int k = 0; k < n; ++k) {
        if (!(hT[k] > 0.0f) || !std::isfinite(hT[k]) || !std::isfinite(he[k]))
            return fail(ctx, MPR_EINVAL, "curve point %d: T must be > 0 and finite, e finite", k);
        if (k > 0 && !(hT[k] > hT[k - 1]))
            return fail(ctx, MPR_EINVAL, "curve temperatures must increase strictly (point %d)", k);
    }
    if (!ctx->curve_T) TRY(dalloc(ctx, &ctx->curve_T, (size_t)kCurveMaxPoints));
    if (!ctx->curve_e) TRY(dalloc(ctx, &ctx->curve_e, (size_t)kCurveMaxPoints));
    CK(cudaMemcpyAsync(ctx->curve_T, hT.data(), (size_t)n * 4, cudaMemcpyHostToDevice, ctx->s));
    CK(cudaMemcpyAsync(ctx->curve_e, he.data(), (size_t)n * 8, cudaMemcpyHostToDevice, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    ctx->curve_n = n;
    return MPR_OK;
}

mpr_status mpr_calibrate(mpr_ctx* ctx, float* block_T_out) {
    PhaseRange phase_range("mpr_calibrate");
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    const Geom& g = ctx->g;
    const mpr_options& o = ctx->opt;
    ctx->batch_open = 0;
    if (ctx->degenerate) {
        std::vector<float> h(g.nblk, o.t_lo);
        CK(cudaMemcpyAsync(ctx->T, h.data(), h.size() * 4, cudaMemcpyHostToDevice, ctx->s));
        for (auto& v : h) v = 1.0f / o.t_lo;
        CK(cudaMemcpyAsync(ctx->beta, h.data(), h.size() * 4, cudaMemcpyHostToDevice, ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
        ctx->calibrated = 1;
        if (block_T_out) return copy_out(ctx, block_T_out, ctx->T, (size_t)g.nblk * 4);
        return MPR_OK;
    }
    const int chains = o.cal_chains;
    if (o.cal_method == 2) {
        // T_b where the unconditional curve reaches e_s,b; the median for
        // blocks without a target.
        TRY(ensure_curve(ctx));
        launch_curve_T(g.nblk, ctx->Nsp_cal, ctx->es, ctx->curve_T, ctx->curve_e, ctx->curve_n,
                       ctx->T, ctx->s);
        CKL();
        launch_cal_fill(ctx->sl, g.nbx, ctx->Nsp_cal, ctx->T, ctx->beta, ctx->s);
        CKL();
        ctx->calibrated = 1;
        ctx->sst = 0;
        if (block_T_out) TRY(copy_out(ctx, block_T_out, ctx->T, (size_t)g.nblk * 4));
        CK(cudaStreamSynchronize(ctx->s));
        return MPR_OK;
    }
    const bool warm = o.cal_warm > 0.0f && o.n_bisect > 0;
    if (warm) {
        TRY(ensure_curve(ctx));
        float ends[2];
        CK(cudaMemcpyAsync(&ends[0], ctx->curve_T, 4, cudaMemcpyDeviceToHost, ctx->s));
        CK(cudaMemcpyAsync(&ends[1], ctx->curve_T + ctx->curve_n - 1, 4, cudaMemcpyDeviceToHost,
                           ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
        if (!((double)ends[0] / o.cal_warm > o.t_lo && (double)ends[1] * o.cal_warm < o.t_hi))
            return fail(ctx, MPR_EINVAL,
                        "warm start: the curve's temperatures [%g, %g] widened by cal_warm = %g "
                        "leave the bracket (%g, %g)", ends[0], ends[1], o.cal_warm, o.t_lo, o.t_hi);
    }
    if (o.cal_method == 1) {
        TRY(calibration_newton(ctx));
        ctx->calibrated = 1;
        ctx->sst = 0;
        if (block_T_out) TRY(copy_out(ctx, block_T_out, ctx->T, (size_t)g.nblk * 4));
        CK(cudaStreamSynchronize(ctx->s));
        collect_events(ctx);
        return MPR_OK;
    }
    ctx->r_off = 0;
    ctx->r_even = 0;
    TRY(ensure_batch(ctx, chains * o.cal_points, o.group, MPR_STORE_F32));
    ctx->R = chains * o.cal_points;
    ctx->chains_valid = true;
    CK(cudaMemsetAsync(ctx->ebar2, 0, (size_t)g.nblk * sizeof(double), ctx->s));
    if (o.cal_points > 2) {
        if (!ctx->Tk) TRY(dalloc(ctx, &ctx->Tk, (size_t)8 * g.nblk));
        if (!ctx->betak) TRY(dalloc(ctx, &ctx->betak, (size_t)8 * g.nblk));
        if (!ctx->ebark) TRY(dalloc(ctx, &ctx->ebark, (size_t)8 * g.nblk));
        CK(cudaMemsetAsync(ctx->ebark, 0, (size_t)8 * g.nblk * sizeof(double), ctx->s));
    }
    launch_cal_init(g.nblk, o.t_lo, o.t_hi, ctx->lo, ctx->hi, ctx->ebar, ctx->ctl, ctx->s);
    CKL();
    const double inv_count = 1.0 / ((double)o.n_meas * (double)chains);
    launch_fill_samples(g, ctx->mask, ctx->dang, ctx->ang, MPR_STORE_F32, ctx->G, ctx->groups,
                        ctx->s);
    CKL();
    // auto and 1: graph; 2: persistent; 3: a launch per kernel from the host.
    bool fallback = o.cal_mode != 2;
    if (!fallback && (ctx->n_slices > 1 || o.cal_points != 1))
        return fail(ctx, MPR_EINVAL,
                    "the persistent calibration (cal_mode 2) takes one field and bisection");
    if (!fallback) {
        TRY(calibration_persistent(ctx, inv_count, &fallback));
        if (fallback && o.cal_mode == 2)
            return fail(ctx, MPR_ECUDA, "calibration: cooperative launch refused");
    }
    if (fallback && o.n_bisect > 0) {
        // E_b of the start state of every iteration.
        TRY(init_batch_state(ctx));
        TRY(energy_pass(ctx));
        CK(cudaMemcpyAsync(ctx->ecur0, ctx->ecur, (size_t)g.nblk * ctx->Rp * sizeof(double),
                           cudaMemcpyDeviceToDevice, ctx->s));
    }
    if (fallback) {
        if (o.n_bisect > 0 && o.cal_mode == 3) {
            for (int k = 0; k < o.n_bisect; ++k)
                TRY(calibration_iteration(ctx, inv_count, 0, true, warm && k == 0, k == 0));
        } else if (o.n_bisect > 0) {
            // A first iteration that differs from the others (the warm start's
            // points, or the only restart of continued chains) runs ahead of
            // the graph, whose body is one of the others.
            const bool ahead = warm || o.cal_continue >= 0;
            if (ahead) TRY(calibration_iteration(ctx, inv_count, 0, true, warm, true));
            const int rest = o.n_bisect - (ahead ? 1 : 0);
            if (rest > 0) TRY(calibration_graph(ctx, inv_count, rest));
        }
        launch_cal_mid(g.nblk, ctx->Nsp_cal, ctx->lo, ctx->hi, ctx->T, ctx->ctl, ctx->s);
        CKL();
        launch_cal_fill(ctx->sl, g.nbx, ctx->Nsp_cal, ctx->T, ctx->beta, ctx->s);
        CKL();
    }
    const int64_t cal_sweeps =
        o.n_bisect <= 0 ? 0
        : o.cal_continue < 0 ? (int64_t)o.n_bisect * (o.n_eq + o.n_meas)
                             : (int64_t)(o.n_eq + o.n_meas) +
                                   (int64_t)(o.n_bisect - 1) * (o.cal_continue + o.n_meas);
    ctx->cal_updates += cal_sweeps * chains * o.cal_points * (ctx->n_gap[0] + ctx->n_gap[1]);
    ctx->calibrated = 1;
    ctx->sst = 0;
    if (block_T_out) TRY(copy_out(ctx, block_T_out, ctx->T, (size_t)g.nblk * 4));
    CK(cudaStreamSynchronize(ctx->s));
    collect_events(ctx);
    return MPR_OK;
}

mpr_status mpr_sim_begin(mpr_ctx* ctx, int32_t n) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    if (n < 1) return fail(ctx, MPR_EINVAL, "n_realizations must be >= 1");
    if (!ctx->calibrated) return fail(ctx, MPR_ESTATE, "calibrate or set temperatures first");
    const int64_t r_base = ctx->r_next;
    if (r_base + n > (int64_t)0x1FFFFFFFF) return fail(ctx, MPR_EINVAL, "realization index overflow");
    ctx->r_off = (int)(r_base & 1);
    ctx->r_even = (uint32_t)(r_base - ctx->r_off);
    TRY(ensure_batch(ctx, n + ctx->r_off, ctx->opt.group, ctx->opt.storage));
    if (ctx->G == 8 && tiles_wanted(ctx)) TRY(ensure_tiles(ctx));
    ctx->R = n;
    ctx->chains_valid = false;
    ctx->t = 0;
    const int64_t nbr = (int64_t)ctx->g.nblk * ctx->Rp;
    k_fill_valid<<<(int)std::min<int64_t>((nbr + 255) / 256, 152 * 16), 256, 0, ctx->s>>>(
        ctx->running, nbr, ctx->Rp, ctx->r_off, ctx->R);
    CKL();
    launch_fill_samples(ctx->g, ctx->mask, ctx->dang, ctx->ang, ctx->storage, ctx->G, ctx->groups,
                        ctx->s);
    CKL();
    TRY(init_batch_state(ctx));
    CK(cudaMemsetAsync(ctx->tcount, 0, (size_t)ctx->Rp * ctx->n_slices * sizeof(int32_t), ctx->s));
    // E_b(0): bond energies of the initial state (no moves), t = 0 stops,
    // worklist of the first sweep.
    if (ctx->opt.init == MPR_INIT_RANDOM || ctx->groups == 1) TRY(energy_pass(ctx));
    else TRY(energy_pass_shared_start(ctx));
    launch_stop_init(ctx->g.nblk, ctx->Rp, ctx->d_of_block, ctx->es, ctx->inb, ctx->Nsp, ctx->ngap,
                     ctx->ecur,
                     ctx->sigma, ctx->running, ctx->stop, ctx->tcount, ctx->e_last, ctx->s);
    CKL();
    launch_stop_rest(ctx->g.nblk, ctx->Rp / 2, 2, ctx->Rp, ctx->opt.n_max, ctx->d_of_block,
                     stop_grid(ctx, 1, kClosingCtasPerSm), ctx->ctl, nullptr, ctx->work, ctx->work_stride, ctx->Nsp,
                     ctx->running, ctx->stop, ctx->tcount, 0, -1, ctx->s);
    CKL();
    ctx->energy_dirty = false;
    ctx->batch_open = 1;
    return MPR_OK;
}

mpr_status mpr_sim_sweep(mpr_ctx* ctx, int32_t n_sweeps, int64_t* n_active) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    if (!ctx->batch_open) return fail(ctx, MPR_ESTATE, "no open batch (mpr_sim_begin)");
    if (ctx->energy_dirty) TRY(refresh_energies(ctx));
    for (int i = 0; i < n_sweeps && ctx->t < ctx->opt.n_max; ++i) TRY(sweep_once(ctx));
    if (n_active) {
        CK(cudaMemcpyAsync(ctx->h_ctl, ctx->ctl, sizeof(Control), cudaMemcpyDeviceToHost, ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
        *n_active = (int64_t)ctx->h_ctl->n_running;
    }
    return MPR_OK;
}

mpr_status mpr_sim_end(mpr_ctx* ctx) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    if (!ctx->batch_open) return fail(ctx, MPR_ESTATE, "no open batch (mpr_sim_begin)");
    for (int c = 0; c < 2; ++c) {
        launch_accumulate(ctx->g, ctx->list[c], ctx->n_gap[c], c, ctx->ang, ctx->storage, ctx->G,
                          ctx->groups,
                          ctx->r_off, ctx->R, ctx->sum, ctx->s);
        CKL();
    }
    CK(cudaMemsetAsync(&ctx->counters[1], 0, sizeof(unsigned long long), ctx->s));
    launch_count_updates(ctx->g.nblk, ctx->Rp, ctx->stop, ctx->ngap, &ctx->counters[1], ctx->s);
    CKL();
    CK(cudaMemcpyAsync(ctx->h_counters + 1, ctx->counters + 1, sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    collect_events(ctx);
    ctx->gap_updates += (int64_t)ctx->h_counters[1];
    ctx->realizations += ctx->R;
    ctx->r_next += ctx->R;
    ctx->batch_open = 0;
    return MPR_OK;
}

mpr_status mpr_sample_chains(mpr_ctx* ctx, int32_t n_chains, int32_t n_equil, int32_t n_samples) {
    PhaseRange phase_range("mpr_sample_chains");
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    if (ctx->batch_open) return fail(ctx, MPR_ESTATE, "a batch is open");
    if (n_chains < 1 || n_equil < 0 || n_samples < 1 || (int64_t)n_equil + n_samples > 65535)
        return fail(ctx, MPR_EINVAL,
                    "need n_chains >= 1, n_equil >= 0, n_samples >= 1, n_equil + n_samples <= 65535");
    // The start state and realization indices of a batch of n_chains; the
    // stop test is not used: every (block, chain) of the batch runs.
    TRY(mpr_sim_begin(ctx, n_chains));
    const int64_t nbr = (int64_t)ctx->g.nblk * ctx->Rp;
    k_fill_valid<<<(int)std::min<int64_t>((nbr + 255) / 256, 152 * 16), 256, 0, ctx->s>>>(
        ctx->running, nbr, ctx->Rp, ctx->r_off, ctx->R);
    CKL();
    launch_set_tag(ctx->ctl, 0u, ctx->s);
    CKL();
    const unsigned long long bound = ctx->bound;
    ctx->bound = ~0ull;
    int form = ctx->opt.sweep_form >= 0 ? ctx->opt.sweep_form : 0;
    if (form == 4 && !tile_form_ok(ctx)) form = 0;
    mpr_status st = MPR_OK;
    for (int t = 1; t <= n_equil + n_samples && st == MPR_OK; ++t) {
        for (int c = 0; c < 2 && st == MPR_OK; ++c) {
            SweepArgs a = sweep_args(ctx, c, true);
            a.work = nullptr;   // every unit; the running flags (all set) decide
            a.energy = 0;
            a.t_fixed = t;
            launch_halfstep(ctx, a, form);
            ++ctx->launches;
            ++ctx->sim_halfstep_launches;
            if (cudaPeekAtLastError() != cudaSuccess)
                st = fail(ctx, MPR_ECUDA, "sample_chains: half-step launch failed");
        }
        if (t <= n_equil) continue;
        for (int c = 0; c < 2 && st == MPR_OK; ++c) {
            launch_accumulate(ctx->g, ctx->list[c], ctx->n_gap[c], c, ctx->ang, ctx->storage,
                              ctx->G, ctx->groups, ctx->r_off, ctx->R, ctx->sum, ctx->s);
            ++ctx->launches;
            if (cudaPeekAtLastError() != cudaSuccess)
                st = fail(ctx, MPR_ECUDA, "sample_chains: accumulate launch failed");
        }
    }
    ctx->bound = bound;
    ctx->batch_open = 0;
    ctx->energy_dirty = true;
    if (st != MPR_OK) return st;
    CK(cudaStreamSynchronize(ctx->s));
    ctx->gap_updates += (int64_t)n_chains * (n_equil + n_samples) * (ctx->n_gap[0] + ctx->n_gap[1]);
    ctx->realizations += (int64_t)n_chains * n_samples;
    ctx->r_next += n_chains;
    return MPR_OK;
}

// The whole sweep loop as one CUDA graph: a conditional WHILE node whose body
// is one sweep (two half-steps, the two stop kernels); the stop test's last
// CTA sets the loop condition on the device. Grids are the full ones (the
// running count is not known when the graph is recorded).
mpr_status simulate_graph(mpr_ctx* ctx) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    mpr_status st = MPR_OK;
    cudaGraphConditionalHandle cond = 0;
    cudaGraphNodeParams p = {};
    cudaGraphNode_t node = nullptr;
    cudaGraph_t body = nullptr, captured = nullptr;
    const int64_t launches0 = ctx->launches;
    const unsigned long long bound = ctx->bound;
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) goto cuda_fail;
    if (cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
        goto cuda_fail;
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = cond;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p) != cudaSuccess) goto cuda_fail;
    body = p.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(ctx->cap, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        goto cuda_fail;
    {
        cudaStream_t user = ctx->s;
        const int profile = ctx->opt.profile;
        ctx->s = ctx->cap;
        ctx->sim_cond = cond;
        ctx->sim_capture = true;
        ctx->opt.profile = 0;
        ctx->bound = ~0ull;
        st = sweep_once(ctx);
        ctx->opt.profile = profile;
        ctx->sim_cond = 0;
        ctx->sim_capture = false;
        ctx->s = user;
    }
    if (cudaStreamEndCapture(ctx->cap, &captured) != cudaSuccess && st == MPR_OK) goto cuda_fail;
    if (st != MPR_OK) goto done;
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) goto cuda_fail;
    if (cudaGraphLaunch(exec, ctx->s) != cudaSuccess) goto cuda_fail;
    goto done;
cuda_fail: {
        cudaError_t e = cudaGetLastError();
        st = fail(ctx, MPR_ECUDA, "simulate graph: %s", cudaGetErrorString(e));
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(ctx->cap, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t tmp = nullptr;
            cudaStreamEndCapture(ctx->cap, &tmp);
            if (tmp && tmp != body) cudaGraphDestroy(tmp);
        }
    }
done:
    if (exec) {
        cudaStreamSynchronize(ctx->s);
        cudaGraphExecDestroy(exec);
    }
    if (graph) cudaGraphDestroy(graph);
    ctx->bound = bound;
    if (st == MPR_OK) {
        // Sweeps done = the device sweep index minus one.
        CK(cudaMemcpyAsync(ctx->h_ctl, ctx->ctl, sizeof(Control), cudaMemcpyDeviceToHost, ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
        const int64_t per_sweep = ctx->launches - launches0;
        ctx->t = (int)ctx->h_ctl->t - 1;
        ctx->launches = launches0 + per_sweep * ctx->t;
    }
    return st;
}

// The rest of the sweep loop as one cooperative launch (the stop tail, when
// few pairs still run). *ran is false when the device or the grid does not
// allow the launch (then nothing ran and the per-launch loop goes on).
// Profiling of a stop-tail launch (profile = 1): its device time and the
// site updates it ran (the batch's updates after it minus those before it),
// kept apart from the per-launch half-steps' figures.
struct TailProfile {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
};

mpr_status tail_profile_begin(mpr_ctx* ctx, TailProfile& tp) {
    if (!ctx->opt.profile) return MPR_OK;
    tp.e0 = get_event(ctx);
    tp.e1 = get_event(ctx);
    if (!tp.e0 || !tp.e1) return fail(ctx, MPR_ECUDA, "cudaEventCreate failed");
    CK(cudaMemsetAsync(ctx->counters + 2, 0, 2 * sizeof(unsigned long long), ctx->s));
    launch_count_updates(ctx->g.nblk, ctx->Rp, ctx->stop, ctx->ngap, ctx->counters + 2, ctx->s,
                         ctx->ctl);
    CKL();
    CK(cudaEventRecord(tp.e0, ctx->s));
    return MPR_OK;
}

mpr_status tail_profile_end(mpr_ctx* ctx, TailProfile& tp) {
    if (!tp.e0) return MPR_OK;
    CK(cudaEventRecord(tp.e1, ctx->s));
    launch_count_updates(ctx->g.nblk, ctx->Rp, ctx->stop, ctx->ngap, ctx->counters + 3, ctx->s,
                         ctx->ctl);
    CKL();
    CK(cudaMemcpyAsync(ctx->h_counters + 4, ctx->counters + 2, 2 * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, ctx->s));
    return MPR_OK;
}

// After a synchronisation of the stream.
void tail_profile_collect(mpr_ctx* ctx, TailProfile& tp) {
    if (!tp.e0) return;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, tp.e0, tp.e1) == cudaSuccess) ctx->sim_tail_ms += ms;
    else cudaGetLastError();
    ctx->sim_tail_updates += (int64_t)(ctx->h_counters[5] - ctx->h_counters[4]);
    ++ctx->sim_tail_launches;
    ctx->ev_pool.push_back(tp.e0);
    ctx->ev_pool.push_back(tp.e1);
    tp.e0 = tp.e1 = nullptr;
}

// The arguments of the stop-tail launches: every sweep field, both colours'
// lists and the stop test's arrays.
SimTailArgs tail_args(mpr_ctx* ctx) {
    const mpr_options& o = ctx->opt;
    SimTailArgs a{};
    a.sw = sweep_args(ctx, 0, true);
    a.sw.energy = 1;
    for (int c = 0; c < 2; ++c) {
        a.list[c] = ctx->list[c];
        a.start[c] = ctx->start[c];
        a.split[c] = ctx->split[c];
    }
    StopArgs& st = a.st;
    st.G = 2;                       // the worklist's units: realization pairs
    st.groups = ctx->Rp / 2;
    st.Rp = ctx->Rp;
    st.nblk = ctx->g.nblk;
    st.n_max = o.n_max;
    st.of_block = ctx->d_of_block;
    st.es = ctx->es;
    st.inb = ctx->inb;
    st.Nsp = ctx->Nsp;
    st.eacc = ctx->eacc;
    st.ecur = ctx->ecur;
    st.sigma = ctx->sigma;
    st.running = ctx->running;
    st.stop = ctx->stop;
    st.tcount = ctx->tcount;
    st.e_last = ctx->e_last;
    st.win = stop_window(ctx);
    a.ctl = ctx->ctl;
    a.work_all = ctx->work;
    return a;
}

mpr_status simulate_tail(mpr_ctx* ctx, bool* ran) {
    *ran = false;
    const int per_sm = ctx->coop ? sim_tail_blocks_per_sm(ctx->G, ctx->storage) : 0;
    if (per_sm < 1) return MPR_OK;
    const mpr_options& o = ctx->opt;
    SimTailArgs a = tail_args(ctx);
    a.bar = ctx->bar;
    a.spin_limit = (unsigned long long)o.wait_ms * 10000ull;   // ~100 ns per poll
    GridBarrier hb{0u, 0u, 0u, (unsigned int)o.barrier_test};
    CK(cudaMemcpyAsync(ctx->bar, &hb, sizeof(hb), cudaMemcpyHostToDevice, ctx->s));
    TailProfile tp;
    TRY(tail_profile_begin(ctx, tp));
    // A grid sized for the pairs still running (16 warps per CTA, about two
    // units per warp at the switch): few CTAs make the grid barriers cheap.
    const unsigned long long want = std::max<unsigned long long>(8, ctx->bound / 32);
    const int grid = (int)std::min<unsigned long long>((unsigned long long)ctx->n_sm * per_sm, want);
    const cudaError_t le = launch_sim_tail(a, ctx->G, ctx->storage, grid, ctx->s);
    if (le != cudaSuccess) {
        cudaGetLastError();
        if (tp.e0) ctx->ev_pool.push_back(tp.e0);
        if (tp.e1) ctx->ev_pool.push_back(tp.e1);
        return MPR_OK;
    }
    *ran = true;
    ++ctx->launches;
    TRY(tail_profile_end(ctx, tp));
    CK(cudaMemcpyAsync(&hb, ctx->bar, sizeof(hb), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaMemcpyAsync(ctx->h_ctl, ctx->ctl, sizeof(Control), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    tail_profile_collect(ctx, tp);
    if (hb.err)
        return fail(ctx, MPR_ETIMEOUT,
                    "simulate: a grid-barrier wait gave up after %d ms; the batch did not "
                    "complete", o.wait_ms);
    // Sweeps run by the launch: from the host's count to the device's last.
    const int t_end = (int)ctx->h_ctl->t - 1;
    if (t_end > ctx->t) ctx->t = t_end;
    ctx->bound = ctx->h_ctl->n_running;
    return MPR_OK;
}

// The rest of the sweep loop with one CTA per realization pair (the stop
// tail, once every pair's running units fit one CTA's buffer).
mpr_status simulate_pair_tail(mpr_ctx* ctx) {
    const SimTailArgs a = tail_args(ctx);
    TailProfile tp;
    TRY(tail_profile_begin(ctx, tp));
    const cudaError_t le = launch_pair_tail(a, ctx->G, ctx->storage, ctx->Rp / 2, ctx->s);
    if (le != cudaSuccess) return fail(ctx, MPR_ECUDA, "stop tail: %s", cudaGetErrorString(le));
    ++ctx->launches;
    TRY(tail_profile_end(ctx, tp));
    CK(cudaMemcpyAsync(ctx->h_ctl, ctx->ctl, sizeof(Control), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    tail_profile_collect(ctx, tp);
    // Sweeps run by the launch: from the host's count to the device's last.
    const int t_end = (int)ctx->h_ctl->t - 1;
    if (t_end > ctx->t) ctx->t = t_end;
    ctx->bound = 0;
    return MPR_OK;
}

mpr_status mpr_simulate(mpr_ctx* ctx, int32_t n) {
    PhaseRange phase_range("mpr_simulate");
    if (!ctx) return MPR_EINVAL;
    TRY(mpr_sim_begin(ctx, n));
    if (ctx->opt.sim_graph && !ctx->opt.profile) {
        TRY(simulate_graph(ctx));
        return mpr_sim_end(ctx);
    }
    // Sweeps are queued in chunks; after each chunk the running count is
    // copied to pinned memory. The host checks the count of the chunk before
    // the one it just queued, so the GPU never waits for the host. Sweeps
    // queued after everything stopped find an empty worklist.
    const int chunk = 4;
    unsigned long long* flag = ctx->h_counters + 2;   // two pinned slots
    cudaEvent_t ev[2] = {get_event(ctx), get_event(ctx)};
    if (!ev[0] || !ev[1]) return fail(ctx, MPR_ECUDA, "cudaEventCreate failed");
    int c = 0;
    mpr_status st = MPR_OK;
    bool tail = ctx->opt.sim_tail > 0;
    // (every pair's units are at most the running count)
    const unsigned long long pair_below = (unsigned long long)std::min(ctx->opt.pair_tail, kPairTailCap);
    while (ctx->t < ctx->opt.n_max) {
        for (int i = 0; i < chunk && ctx->t < ctx->opt.n_max && st == MPR_OK; ++i) st = sweep_once(ctx);
        if (st != MPR_OK) break;
        if (cudaMemcpyAsync(flag + (c & 1), &ctx->ctl->n_running, sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, ctx->s) != cudaSuccess ||
            cudaEventRecord(ev[c & 1], ctx->s) != cudaSuccess) {
            st = fail(ctx, MPR_ECUDA, "simulate: copy of the running count failed");
            break;
        }
        if (c >= 1) {
            if (cudaEventSynchronize(ev[(c - 1) & 1]) != cudaSuccess) {
                st = fail(ctx, MPR_ECUDA, "simulate: event synchronisation failed");
                break;
            }
            // The running count never grows, so the count read here bounds
            // the work of every sweep queued from now on.
            ctx->bound = flag[(c - 1) & 1];
            if (ctx->bound == 0) break;
            // Few pairs left: the rest of the loop as one cooperative launch
            // (when asked for), or with one CTA per realization pair.
            if (!tail && ctx->bound <= pair_below) {
                st = simulate_pair_tail(ctx);
                break;
            }
            if (tail && ctx->bound < (unsigned long long)ctx->opt.sim_tail) {
                bool ran = false;
                st = simulate_tail(ctx, &ran);
                if (st != MPR_OK || ran) break;
                tail = false;
            }
        }
        ++c;
    }
    ctx->ev_pool.push_back(ev[0]);
    ctx->ev_pool.push_back(ev[1]);
    if (st != MPR_OK) return st;
    return mpr_sim_end(ctx);
}

mpr_status mpr_halfstep(mpr_ctx* ctx, int32_t colour, int32_t t, int32_t tag) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    if (!ctx->batch_open) return fail(ctx, MPR_ESTATE, "no open batch (mpr_sim_begin)");
    if (colour != 0 && colour != 1) return fail(ctx, MPR_EINVAL, "colour must be 0 or 1");
    if (t < 0 || t > 65535 || tag < 0 || tag > 65535)
        return fail(ctx, MPR_EINVAL, "t and tag must be in [0, 65535]");
    CK(cudaMemcpyAsync(ctx->h_ctl, ctx->ctl, sizeof(Control), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    Control saved = *ctx->h_ctl;
    ctx->h_ctl->t = (uint32_t)t;
    ctx->h_ctl->tag = (uint32_t)tag;
    CK(cudaMemcpyAsync(ctx->ctl, ctx->h_ctl, sizeof(Control), cudaMemcpyHostToDevice, ctx->s));
    SweepArgs a = sweep_args(ctx, colour, true);
    a.work = nullptr;       // every item; the running flags decide
    a.energy = 0;
    const unsigned long long bound = ctx->bound;
    ctx->bound = ~0ull;
    // The form the options ask for (the automatic choice: one warp per pair).
    int form = ctx->opt.sweep_form >= 0 ? ctx->opt.sweep_form : 0;
    if (form == 4 && !tile_form_ok(ctx)) form = 0;
    launch_halfstep(ctx, a, form);
    ctx->bound = bound;
    CKL();
    CK(cudaStreamSynchronize(ctx->s));
    *ctx->h_ctl = saved;
    CK(cudaMemcpyAsync(ctx->ctl, ctx->h_ctl, sizeof(Control), cudaMemcpyHostToDevice, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    ctx->energy_dirty = true;
    return MPR_OK;
}

mpr_status mpr_get_state(mpr_ctx* ctx, int32_t r, float* angles) {
    if (!ctx || !angles) return MPR_EINVAL;
    ctx->err.clear();
    if (!ctx->batch_open) return fail(ctx, MPR_ESTATE, "no open batch");
    if (r < 0 || r >= ctx->R) return fail(ctx, MPR_EINVAL, "r out of range");
    const size_t n = (size_t)ctx->g.H * ctx->g.W;
    if (!ctx->out_buf) TRY(dalloc(ctx, &ctx->out_buf, n));
    launch_get_state(ctx->g, ctx->mask, ctx->dang, ctx->ang, ctx->storage, ctx->G, r + ctx->r_off,
                     ctx->out_buf, ctx->s);
    CKL();
    return copy_out(ctx, angles, ctx->out_buf, n * 4);
}

mpr_status mpr_set_state(mpr_ctx* ctx, int32_t r, const float* angles) {
    if (!ctx || !angles) return MPR_EINVAL;
    ctx->err.clear();
    if (!ctx->batch_open) return fail(ctx, MPR_ESTATE, "no open batch");
    if (r < 0 || r >= ctx->R) return fail(ctx, MPR_EINVAL, "r out of range");
    const size_t n = (size_t)ctx->g.H * ctx->g.W;
    if (!ctx->truth_buf) TRY(dalloc(ctx, &ctx->truth_buf, n));
    TRY(copy_in(ctx, ctx->truth_buf, angles, n * 4));
    launch_set_state(ctx->g, ctx->mask, ctx->ang, ctx->storage, ctx->G, r + ctx->r_off,
                     ctx->truth_buf, ctx->s);
    CKL();
    CK(cudaStreamSynchronize(ctx->s));
    ctx->energy_dirty = true;
    return MPR_OK;
}

mpr_status mpr_get_stop(mpr_ctx* ctx, int32_t* stop_sweep, uint8_t* running) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    if (!ctx->batch_open) return fail(ctx, MPR_ESTATE, "no open batch");
    const int nb = ctx->g.nblk;
    std::vector<int32_t> hs((size_t)nb * ctx->Rp);
    std::vector<uint8_t> hr((size_t)nb * ctx->Rp);
    CK(cudaMemcpyAsync(hs.data(), ctx->stop, hs.size() * 4, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaMemcpyAsync(hr.data(), ctx->running, hr.size(), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    std::vector<int32_t> os((size_t)ctx->R * nb);
    std::vector<uint8_t> orr((size_t)ctx->R * nb);
    for (int r = 0; r < ctx->R; ++r)
        for (int b = 0; b < nb; ++b) {
            os[(size_t)r * nb + b] = hs[(size_t)b * ctx->Rp + r + ctx->r_off];
            orr[(size_t)r * nb + b] = hr[(size_t)b * ctx->Rp + r + ctx->r_off];
        }
    if (stop_sweep)
        CK(cudaMemcpyAsync(stop_sweep, os.data(), os.size() * 4, cudaMemcpyDefault, ctx->s));
    if (running) CK(cudaMemcpyAsync(running, orr.data(), orr.size(), cudaMemcpyDefault, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    return MPR_OK;
}

mpr_status mpr_get_block_e(mpr_ctx* ctx, double* e) {
    if (!ctx || !e) return MPR_EINVAL;
    ctx->err.clear();
    if (!ctx->batch_open) return fail(ctx, MPR_ESTATE, "no open batch");
    const int nb = ctx->g.nblk;
    std::vector<double> h((size_t)nb * ctx->Rp), o((size_t)ctx->R * nb);
    CK(cudaMemcpyAsync(h.data(), ctx->e_last, h.size() * 8, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    for (int r = 0; r < ctx->R; ++r)
        for (int b = 0; b < nb; ++b) o[(size_t)r * nb + b] = h[(size_t)b * ctx->Rp + r + ctx->r_off];
    CK(cudaMemcpyAsync(e, o.data(), o.size() * 8, cudaMemcpyDefault, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    return MPR_OK;
}

mpr_status mpr_set_running(mpr_ctx* ctx, const uint8_t* running) {
    if (!ctx || !running) return MPR_EINVAL;
    ctx->err.clear();
    if (!ctx->batch_open) return fail(ctx, MPR_ESTATE, "no open batch");
    const int nb = ctx->g.nblk;
    std::vector<uint8_t> in((size_t)ctx->R * nb), hr((size_t)nb * ctx->Rp, 0);
    CK(cudaMemcpyAsync(in.data(), running, in.size(), cudaMemcpyDefault, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    for (int r = 0; r < ctx->R; ++r)
        for (int b = 0; b < nb; ++b)
            hr[(size_t)b * ctx->Rp + r + ctx->r_off] = in[(size_t)r * nb + b] ? 1 : 0;
    CK(cudaMemcpyAsync(ctx->running, hr.data(), hr.size(), cudaMemcpyHostToDevice, ctx->s));
    CK(cudaMemsetAsync(ctx->tcount, 0, (size_t)ctx->Rp * ctx->n_slices * sizeof(int32_t), ctx->s));
    CK(cudaMemcpyAsync(ctx->h_ctl, ctx->ctl, sizeof(Control), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    const uint32_t par = ctx->h_ctl->t & 1u;
    CK(cudaMemsetAsync(&ctx->ctl->n_work[par], 0, sizeof(uint32_t), ctx->s));
    const int64_t items = (int64_t)nb * (ctx->Rp / 2);
    k_rebuild<<<(int)std::min<int64_t>((items + 255) / 256, 152 * 16), 256, 0, ctx->s>>>(
        nb, ctx->Rp / 2, 2, ctx->Rp, ctx->d_of_block, ctx->Nsp, ctx->running, ctx->tcount,
        ctx->ctl, ctx->work, ctx->work_stride);
    ctx->bound = ~0ull;
    CKL();
    CK(cudaStreamSynchronize(ctx->s));
    return MPR_OK;
}

mpr_status mpr_block_energy(mpr_ctx* ctx, int32_t r, double* E) {
    if (!ctx || !E) return MPR_EINVAL;
    ctx->err.clear();
    if (!ctx->batch_open) return fail(ctx, MPR_ESTATE, "no open batch");
    if (r < 0 || r >= ctx->R) return fail(ctx, MPR_EINVAL, "r out of range");
    double* d = nullptr;
    TRY(dalloc(ctx, &d, ctx->g.nblk));
    launch_block_energy(ctx->g, ctx->d_of_block, ctx->mask, ctx->dang, ctx->ang, ctx->storage,
                        ctx->G,
                        r + ctx->r_off, ctx->opt.q, ctx->opt.J, d, ctx->s);
    mpr_status st = MPR_OK;
    if (cudaPeekAtLastError() != cudaSuccess) st = fail(ctx, MPR_ECUDA, "block energy launch failed");
    if (st == MPR_OK) st = copy_out(ctx, E, d, (size_t)ctx->g.nblk * 8);
    dfree(ctx, d);
    ctx->device_bytes -= (int64_t)ctx->g.nblk * 8;
    return st;
}

mpr_status ensure_site_buffers(mpr_ctx* ctx) {
    const size_t n = (size_t)ctx->g.H * ctx->g.W;
    if (!ctx->T_site) TRY(dalloc(ctx, &ctx->T_site, n));
    if (!ctx->beta_site) TRY(dalloc(ctx, &ctx->beta_site, n));
    return MPR_OK;
}

mpr_status mpr_smooth_temperatures(mpr_ctx* ctx, int32_t r_s, int32_t n_s, float* T_site_out) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    if (!ctx->calibrated) return fail(ctx, MPR_ESTATE, "calibrate or set temperatures first");
    if (ctx->batch_open) return fail(ctx, MPR_ESTATE, "a batch is open");
    if (r_s < 0 || r_s > 4096 || n_s < 0 || n_s > 1000)
        return fail(ctx, MPR_EINVAL, "need 0 <= r_s <= 4096 and 0 <= n_s <= 1000");
    TRY(ensure_site_buffers(ctx));
    const size_t n = (size_t)ctx->g.H * ctx->g.W;
    double *Ts = nullptr, *tmp = nullptr;
    CK(cudaMallocAsync((void**)&Ts, n * sizeof(double), ctx->s));
    CK(cudaMallocAsync((void**)&tmp, n * sizeof(double), ctx->s));
    launch_sst(ctx->g, ctx->sl, ctx->T, r_s, n_s, Ts, tmp, ctx->T_site, ctx->beta_site, ctx->s);
    ctx->launches += 2 + 2 * n_s;
    const cudaError_t e = cudaPeekAtLastError();
    cudaFreeAsync(Ts, ctx->s);
    cudaFreeAsync(tmp, ctx->s);
    if (e != cudaSuccess) return fail(ctx, MPR_ECUDA, "smoothing: %s", cudaGetErrorString(e));
    ctx->sst = 1;
    if (T_site_out) return copy_out(ctx, T_site_out, ctx->T_site, n * 4);
    CK(cudaStreamSynchronize(ctx->s));
    return MPR_OK;
}

mpr_status mpr_set_site_temperatures(mpr_ctx* ctx, const float* T_site) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    if (ctx->batch_open) return fail(ctx, MPR_ESTATE, "a batch is open");
    if (!T_site) {
        ctx->sst = 0;
        return MPR_OK;
    }
    if (!ctx->calibrated) return fail(ctx, MPR_ESTATE, "calibrate or set temperatures first");
    const size_t n = (size_t)ctx->g.H * ctx->g.W;
    std::vector<float> h(n);
    CK(cudaMemcpyAsync(h.data(), T_site, n * 4, cudaMemcpyDefault, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    for (float v : h)
        if (!(v > 0.0f) || !std::isfinite(v)) return fail(ctx, MPR_EINVAL, "site temperatures must be > 0");
    TRY(ensure_site_buffers(ctx));
    CK(cudaMemcpyAsync(ctx->T_site, h.data(), n * 4, cudaMemcpyHostToDevice, ctx->s));
    launch_site_beta((int64_t)n, ctx->T_site, ctx->beta_site, ctx->s);
    CKL();
    CK(cudaStreamSynchronize(ctx->s));
    ctx->sst = 1;
    return MPR_OK;
}

mpr_status mpr_get_site_temperatures(mpr_ctx* ctx, float* T_site) {
    if (!ctx || !T_site) return MPR_EINVAL;
    ctx->err.clear();
    if (!ctx->sst) return fail(ctx, MPR_ESTATE, "no site temperatures");
    return copy_out(ctx, T_site, ctx->T_site, (size_t)ctx->g.H * ctx->g.W * 4);
}

mpr_status mpr_energy_moments(mpr_ctx* ctx, const float* beta, int32_t n_eq, int32_t n_meas,
                              int32_t tag, int32_t restart, double* mean_e, double* var_E,
                              double* cov_r, double* cov_d) {
    if (!ctx || !beta) return MPR_EINVAL;
    ctx->err.clear();
    if (ctx->batch_open) return fail(ctx, MPR_ESTATE, "a realization batch is open");
    if (n_eq < 0 || n_meas < 1 || n_eq + n_meas > 65535)
        return fail(ctx, MPR_EINVAL, "need n_eq >= 0, n_meas >= 1, n_eq + n_meas <= 65535");
    if (tag < 1 || tag > 65534) return fail(ctx, MPR_EINVAL, "tag must be in [1, 65534]");
    const int nb = ctx->g.nblk;
    std::vector<float> hb(nb), ht(nb);
    CK(cudaMemcpyAsync(hb.data(), beta, nb * 4, cudaMemcpyDefault, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    for (int b = 0; b < nb; ++b) {
        if (!(hb[b] > 0.0f) || !std::isfinite(hb[b]))
            return fail(ctx, MPR_EINVAL, "beta of block %d is not a positive number", b);
        ht[b] = 1.0f / hb[b];
    }
    CK(cudaMemcpyAsync(ctx->beta, hb.data(), nb * 4, cudaMemcpyHostToDevice, ctx->s));
    CK(cudaMemcpyAsync(ctx->T, ht.data(), nb * 4, cudaMemcpyHostToDevice, ctx->s));
    ctx->calibrated = 1;
    ctx->sst = 0;
    TRY(moments_run(ctx, (uint32_t)tag, restart != 0, n_eq, n_meas));
    double* outs[4] = {mean_e, var_E, cov_r, cov_d};
    for (int k = 0; k < 4; ++k)
        if (outs[k]) TRY(copy_out(ctx, outs[k], ctx->mom + (size_t)k * nb, (size_t)nb * 8));
    CK(cudaStreamSynchronize(ctx->s));
    collect_events(ctx);
    return MPR_OK;
}

mpr_status mpr_energy_vjp(mpr_ctx* ctx, const double* grad_e, double* grad_beta) {
    if (!ctx || !grad_e || !grad_beta) return MPR_EINVAL;
    ctx->err.clear();
    if (!ctx->moments_valid) return fail(ctx, MPR_ESTATE, "no energy moments yet");
    const size_t nb = (size_t)ctx->g.nblk;
    double* tmp = nullptr;
    CK(cudaMallocAsync((void**)&tmp, 2 * nb * sizeof(double), ctx->s));
    mpr_status st = copy_in(ctx, tmp, grad_e, nb * 8);
    if (st == MPR_OK) {
        launch_energy_vjp(ctx->g.nblk, ctx->g.nbx, ctx->Nb, ctx->mom, tmp, tmp + nb, ctx->s);
        ++ctx->launches;
        st = cudaPeekAtLastError() == cudaSuccess ? copy_out(ctx, grad_beta, tmp + nb, nb * 8)
                                                  : fail(ctx, MPR_ECUDA, "k_energy_vjp");
    }
    cudaFreeAsync(tmp, ctx->s);
    CK(cudaStreamSynchronize(ctx->s));
    return st;
}

mpr_status mpr_autotune(mpr_ctx* ctx, int32_t n_realizations, int32_t n_sweeps,
                        mpr_tuning* out) {
    PhaseRange phase_range("mpr_autotune");
    if (!ctx || !out) return MPR_EINVAL;
    ctx->err.clear();
    if (ctx->batch_open) return fail(ctx, MPR_ESTATE, "a batch is open");
    if (!ctx->calibrated) return fail(ctx, MPR_ESTATE, "calibrate or set temperatures first");
    if (n_realizations < 1 || n_sweeps < 1 || n_sweeps > 64)
        return fail(ctx, MPR_EINVAL, "need n_realizations >= 1 and 1 <= n_sweeps <= 64");
    std::memset(out, 0, sizeof(*out));
    const int saved_group = ctx->opt.group, saved_form = ctx->tuned_form;
    const int saved_profile = ctx->opt.profile;
    const int64_t saved[4] = {ctx->gap_updates, ctx->launches, ctx->sim_halfstep_launches,
                              ctx->realizations};
    const int cand[4][2] = {{8, 0}, {8, 3}, {8, 4}, {2, 0}};
    float best = 0.0f;
    int best_k = -1;
    mpr_status st = MPR_OK;
    ctx->opt.profile = 0;
    cudaEvent_t t0 = get_event(ctx), t1 = get_event(ctx);
    if (!t0 || !t1) return fail(ctx, MPR_ECUDA, "cudaEventCreate failed");
    cudaEventRecord(t0, ctx->s);
    // An untimed sweep first: the batch state's first touch (memory the pool
    // maps on first use) would otherwise be charged to the first candidate.
    ctx->opt.group = cand[0][0];
    ctx->tuned_form = cand[0][1];
    st = mpr_sim_begin(ctx, n_realizations);
    if (st == MPR_OK) {
        st = sweep_once(ctx);
        ctx->batch_open = 0;
    }
    for (int k = 0; k < 4 && st == MPR_OK; ++k) {
        ctx->opt.group = cand[k][0];
        ctx->tuned_form = cand[k][1];
        ctx->tuning_tiles = cand[k][1] == 4;
        // A trial batch: the first sweeps (every pair running), timed on the
        // stream; discarded afterwards (nothing is accumulated or counted).
        st = mpr_sim_begin(ctx, n_realizations);
        ctx->tuning_tiles = false;
        if (st != MPR_OK) break;
        if (cand[k][1] == 4 && !tile_form_ok(ctx)) {   // (lane groups of two: no staged form)
            ctx->batch_open = 0;
            out->ms[k] = -1.0f;
            continue;
        }
        cudaEvent_t e0 = get_event(ctx), e1 = get_event(ctx);
        if (!e0 || !e1) { st = fail(ctx, MPR_ECUDA, "cudaEventCreate failed"); break; }
        cudaEventRecord(e0, ctx->s);
        for (int i = 0; i < n_sweeps && st == MPR_OK; ++i) st = sweep_once(ctx);
        cudaEventRecord(e1, ctx->s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(ctx, MPR_ECUDA, "autotune sync");
        float ms = 0.0f;
        if (st == MPR_OK) cudaEventElapsedTime(&ms, e0, e1);
        ctx->ev_pool.push_back(e0);
        ctx->ev_pool.push_back(e1);
        ctx->batch_open = 0;
        out->ms[k] = ms;
        if (st == MPR_OK && (best_k < 0 || ms < best)) { best = ms; best_k = k; }
    }
    cudaEventRecord(t1, ctx->s);
    if (cudaEventSynchronize(t1) == cudaSuccess) cudaEventElapsedTime(&out->trial_ms, t0, t1);
    else cudaGetLastError();
    ctx->ev_pool.push_back(t0);
    ctx->ev_pool.push_back(t1);
    ctx->opt.profile = saved_profile;
    ctx->gap_updates = saved[0];
    ctx->launches = saved[1];
    ctx->sim_halfstep_launches = saved[2];
    ctx->realizations = saved[3];
    ctx->chains_valid = false;
    if (st != MPR_OK || best_k < 0) {
        ctx->opt.group = saved_group;
        ctx->tuned_form = saved_form;
        return st != MPR_OK ? st : fail(ctx, MPR_ECUDA, "autotune: no candidate ran");
    }
    ctx->opt.group = cand[best_k][0];
    ctx->tuned_form = cand[best_k][1];
    out->group = cand[best_k][0];
    out->form = cand[best_k][1];
    return MPR_OK;
}

mpr_status mpr_set_realization_base(mpr_ctx* ctx, int64_t r_first) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    if (ctx->batch_open) return fail(ctx, MPR_ESTATE, "a batch is open");
    if (r_first < 0 || r_first > (int64_t)0x1FFFFFFFF)
        return fail(ctx, MPR_EINVAL, "r_first out of range");
    ctx->r_next = r_first;
    return MPR_OK;
}

mpr_status mpr_get_accumulator(mpr_ctx* ctx, double* sum_out, int64_t* n_realizations) {
    if (!ctx) return MPR_EINVAL;
    ctx->err.clear();
    if (ctx->batch_open) return fail(ctx, MPR_ESTATE, "a batch is open");
    if (n_realizations) *n_realizations = ctx->realizations;
    if (!sum_out) return MPR_OK;
    const size_t n = (size_t)ctx->g.H * ctx->g.W;
    double* tmp = nullptr;
    CK(cudaMallocAsync((void**)&tmp, n * sizeof(double), ctx->s));
    launch_sum_to_grid(ctx->g, ctx->mask, ctx->sum, tmp, ctx->s);
    mpr_status st = cudaGetLastError() == cudaSuccess ? copy_out(ctx, sum_out, tmp, n * 8)
                                                      : fail(ctx, MPR_ECUDA, "k_sum_to_grid");
    cudaFreeAsync(tmp, ctx->s);
    CK(cudaStreamSynchronize(ctx->s));
    return st;
}

mpr_status mpr_set_accumulator(mpr_ctx* ctx, const double* sum_in, int64_t n_realizations) {
    if (!ctx || !sum_in) return MPR_EINVAL;
    ctx->err.clear();
    if (ctx->batch_open) return fail(ctx, MPR_ESTATE, "a batch is open");
    if (n_realizations < 0) return fail(ctx, MPR_EINVAL, "n_realizations must be >= 0");
    const size_t n = (size_t)ctx->g.H * ctx->g.W;
    double* tmp = nullptr;
    CK(cudaMallocAsync((void**)&tmp, n * sizeof(double), ctx->s));
    mpr_status st = copy_in(ctx, tmp, sum_in, n * 8);
    if (st == MPR_OK) {
        launch_grid_to_sum(ctx->g, ctx->mask, tmp, ctx->sum, ctx->s);
        if (cudaGetLastError() != cudaSuccess) st = fail(ctx, MPR_ECUDA, "k_grid_to_sum");
    }
    cudaFreeAsync(tmp, ctx->s);
    CK(cudaStreamSynchronize(ctx->s));
    if (st == MPR_OK) ctx->realizations = n_realizations;
    return st;
}

// Predictions of the whole canvas into ctx->out_buf; with a truth canvas in
// ctx->truth_buf the per-slice error sums land in ctx->err_buf.
mpr_status predict_canvas(mpr_ctx* ctx, bool with_truth) {
    const int64_t total_gap = ctx->n_gap[0] + ctx->n_gap[1];
    if (ctx->realizations == 0 && total_gap > 0)
        return fail(ctx, MPR_ESTATE, "no realization accumulated (mpr_simulate)");
    const size_t n = (size_t)ctx->g.H * ctx->g.W;
    if (!ctx->out_buf) TRY(dalloc(ctx, &ctx->out_buf, n));
    if (with_truth)
        CK(cudaMemsetAsync(ctx->err_buf, 0, 2 * (size_t)ctx->n_slices * sizeof(double), ctx->s));
    const double inv_r = ctx->realizations > 0 ? 1.0 / (double)ctx->realizations : 0.0;
    launch_predict(ctx->g, ctx->sl, ctx->values, ctx->mask, ctx->sum, inv_r, ctx->out_buf,
                   with_truth ? ctx->truth_buf : nullptr, ctx->err_buf, ctx->s);
    CKL();
    return MPR_OK;
}

mpr_status mpr_predict(mpr_ctx* ctx, float* out, const float* truth, double* aae_rase) {
    PhaseRange phase_range("mpr_predict");
    if (!ctx || !out) return MPR_EINVAL;
    ctx->err.clear();
    const size_t n = (size_t)ctx->g.H * ctx->g.W;
    if (truth) {
        if (!ctx->truth_buf) TRY(dalloc(ctx, &ctx->truth_buf, n));
        TRY(copy_in(ctx, ctx->truth_buf, truth, n * 4));
    }
    TRY(predict_canvas(ctx, truth != nullptr));
    TRY(copy_out(ctx, out, ctx->out_buf, n * 4));
    if (truth && aae_rase) {
        std::vector<double> h(2 * (size_t)ctx->n_slices);
        TRY(copy_out(ctx, h.data(), ctx->err_buf, h.size() * 8));
        double a = 0.0, r = 0.0;
        for (int k = 0; k < ctx->n_slices; ++k) { a += h[2 * k]; r += h[2 * k + 1]; }
        const int64_t total_gap = ctx->n_gap[0] + ctx->n_gap[1];
        aae_rase[0] = total_gap ? a / (double)total_gap : 0.0;
        aae_rase[1] = total_gap ? std::sqrt(r / (double)total_gap) : 0.0;
    }
    return MPR_OK;
}

mpr_status mpr_predict_batch(mpr_ctx* ctx, float* const* outs, const float* const* truths,
                             double* aae_rase) {
    PhaseRange phase_range("mpr_predict_batch");
    if (!ctx || !outs) return MPR_EINVAL;
    ctx->err.clear();
    const Geom& g = ctx->g;
    const size_t n = (size_t)g.H * g.W;
    for (int k = 0; k < ctx->n_slices; ++k)
        if (!outs[k] || (truths && !truths[k])) return fail(ctx, MPR_EINVAL, "NULL slice pointer");
    if (truths) {
        if (!ctx->truth_buf) TRY(dalloc(ctx, &ctx->truth_buf, n));
        CK(cudaMemsetAsync(ctx->truth_buf, 0, n * 4, ctx->s));
        uint8_t* st = nullptr;
        TRY(host_stage(ctx, reinterpret_cast<const void* const*>(truths), ctx->n_slices, 4, &st));
        mpr_status s2 = MPR_OK;
        for (int k = 0; k < ctx->n_slices && s2 == MPR_OK; ++k) {
            const int4 rc = ctx->h_rect[k];
            s2 = canvas_copy(ctx, true, ctx->truth_buf, (size_t)rc.x * g.W + rc.y, truths[k],
                             nullptr, rc.z, rc.w, 4, st);
        }
        dfree(ctx, st);
        TRY(s2);
    }
    TRY(predict_canvas(ctx, truths != nullptr));
    {
        uint8_t* st = nullptr;
        TRY(host_stage(ctx, reinterpret_cast<const void* const*>(outs), ctx->n_slices, 4, &st));
        mpr_status s2 = MPR_OK;
        for (int k = 0; k < ctx->n_slices && s2 == MPR_OK; ++k) {
            const int4 rc = ctx->h_rect[k];
            s2 = canvas_copy(ctx, false, ctx->out_buf, (size_t)rc.x * g.W + rc.y, nullptr, outs[k],
                             rc.z, rc.w, 4, st);
        }
        dfree(ctx, st);
        TRY(s2);
    }
    CK(cudaStreamSynchronize(ctx->s));
    if (truths && aae_rase) {
        std::vector<double> h(2 * (size_t)ctx->n_slices);
        TRY(copy_out(ctx, h.data(), ctx->err_buf, h.size() * 8));
        for (int k = 0; k < ctx->n_slices; ++k) {
            const int64_t ng = ctx->h_ngap[k];
            aae_rase[2 * k] = ng ? h[2 * k] / (double)ng : 0.0;
            aae_rase[2 * k + 1] = ng ? std::sqrt(h[2 * k + 1] / (double)ng) : 0.0;
        }
    }
    return MPR_OK;
}

mpr_status mpr_get_slice_layout(const mpr_ctx* ctx, int32_t* rects) {
    if (!ctx || !rects) return MPR_EINVAL;
    for (int k = 0; k < ctx->n_slices; ++k) {
        rects[4 * k] = ctx->h_rect[k].x;
        rects[4 * k + 1] = ctx->h_rect[k].y;
        rects[4 * k + 2] = ctx->h_rect[k].z;
        rects[4 * k + 3] = ctx->h_rect[k].w;
    }
    return MPR_OK;
}

}  // extern "C"
