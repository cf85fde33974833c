// Host-side launchers of the kernels in mpr_kernels.cu (stream-ordered, no sync).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "mpr_internal.h"

namespace mpr {

float ord2f(uint32_t u);

// One field (mask != 0: gap): mm[0..1] = order-preserving (min, max), pre-set.
void launch_minmax_field(const float* values, const uint8_t* mask, int64_t n, uint32_t* mm,
                         cudaStream_t s);
// mm: 2 per slice (order-preserving min, max), pre-set to (max, 0).
void launch_minmax(const Geom& g, const int32_t* of_block, const float* values,
                   const uint8_t* mask, uint32_t* mm, cudaStream_t s);
void launch_layout(const Geom& g, const Slices& sl, const float* values, const uint8_t* mask,
                   float* dang, cudaStream_t s);
void launch_block_stats(const Geom& g, const Slices& sl, const float* values, const uint8_t* mask,
                        double q, double J, double* Es, int32_t* Nsp, int32_t* Nb, double* ssum,
                        int32_t* nsamp, int32_t* ngap0, int32_t* ngap1, cudaStream_t s);
void launch_scan(const int32_t* cnt, int n, int32_t* out, cudaStream_t s);
void launch_build_lists(const Geom& g, const int32_t* of_block, const uint8_t* mask,
                        const int32_t* start0, const int32_t* start1, uint2* list0, uint2* list1,
                        int32_t* split0, int32_t* split1, cudaStream_t s);
// `storage` is an mpr_storage value (0 FP32, 1 BF16, 2 FP16): the element
// type of the batch state `ang`.
void launch_init(const Geom& g, const Slices& sl, const uint2* list, int64_t n_list, int colour,
                 const float* init_angle, void* ang, int storage, int G, int Rp, int random,
                 Rng rng, uint32_t r_even, cudaStream_t s);
void launch_fill_samples(const Geom& g, const uint8_t* mask, const float* dang, void* ang,
                         int storage, int G, int groups, cudaStream_t s);
// form 0, 1, 2: one, two or four warps per realization pair (more warps per
// pair as fewer items are left).
void launch_sweep(const SweepArgs& a, int G, int storage, int form, int grid, cudaStream_t s);
int sweep_blocks_per_sm(int G, int storage, int form);
int sweep_items_per_cta(int G, int form);
void launch_energy(const SweepArgs& a, int G, int storage, int n_sm, cudaStream_t s);
// fold: NULL, or the previous sweep's fold run by extra CTAs of this launch.
void launch_sweep_flat(const SweepArgs& a, int G, int64_t n_list, cudaStream_t s,
                       const FoldArgs* fold = nullptr);
// The same half-step of the calibration's chains in the warp form (one warp
// per (block, pair) unit).
void launch_sweep_cal(const SweepArgs& a, int G, cudaStream_t s, const FoldArgs* fold = nullptr);
void launch_ecur_broadcast(int nblk, int Rp, int G, double* ecur, cudaStream_t s);
void launch_ecur_reset(int nblk, int Rp, const double* Es, double* ecur, double* eacc,
                       cudaStream_t s);
// tcount is [n_slices][Rp]: running targeted blocks per slice and realization.
void launch_stop_init(int nblk, int Rp, const int32_t* of_block, const double* es,
                      const double* inb, const int32_t* Nsp, const int32_t* ngap, const double* ecur,
                      int8_t* sigma, uint8_t* running, int32_t* stop, int32_t* tcount,
                      double* e_last, cudaStream_t s);
void launch_stop_targeted(int G, int groups, int Rp, const int32_t* of_block, int grid,
                          Control* ctl, const uint32_t* work, uint32_t work_stride,
                          const double* es, const double* inb, const int32_t* Nsp, double* eacc,
                          double* ecur, const int8_t* sigma, uint8_t* running, int32_t* stop,
                          int32_t* tcount, double* e_last, int t_known, cudaStream_t s,
                          const StopWindow* win = nullptr);
// work == nullptr: every item (t = 0). Writes the next sweep's worklist into
// work_all and advances ctl->t.
void launch_stop_rest(int nblk, int groups, int G, int Rp, int n_max, const int32_t* of_block,
                      int grid, Control* ctl, const uint32_t* work, uint32_t* work_all,
                      uint32_t work_stride, const int32_t* Nsp, uint8_t* running, int32_t* stop,
                      const int32_t* tcount, cudaGraphConditionalHandle cond, int t_known,
                      cudaStream_t s);
// ctl != nullptr: updates so far, running pairs counted up to sweep ctl->t - 1.
void launch_count_updates(int nblk, int Rp, const int32_t* stop, const int32_t* ngap,
                          unsigned long long* total, cudaStream_t s, const Control* ctl = nullptr);
void launch_cal_init(int nblk, float t_lo, float t_hi, float* lo, float* hi, double* ebar,
                     Control* ctl, cudaStream_t s);
void launch_cal_mid(int nblk, const int32_t* Nsp, const float* lo, const float* hi, float* T,
                    Control* ctl, cudaStream_t s);
void launch_cal_fill(const Slices& sl, int nbx, const int32_t* Nsp, float* T, float* beta,
                     cudaStream_t s);
// points = 2: even lanes' energies go to ebar, odd lanes' to ebar_odd; points
// > 2: lane r's to ebar_pts[r mod points].
void launch_cal_step(int nblk, int Rp, int chains, int n_eq, int t_fixed, const Control* ctl,
                     const double* inb, double* eacc, double* ecur, double* ebar, cudaStream_t s,
                     int points = 1, double* ebar_odd = nullptr, double* ebar_pts = nullptr);
// k-point calibration (points = 4 or 8): the points of every bracket, and the
// bracket update from the points' mean energies (Tk, ebar_pts: [points][nblk]).
void launch_kpts_mid(int nblk, int points, const int32_t* Nsp, const float* lo, const float* hi,
                     float* Tk, Control* ctl, cudaStream_t s);
void launch_kpts_update(int nblk, int points, double inv_count, const double* es,
                        const int32_t* Nsp, const float* Tk, float* lo, float* hi,
                        double* ebar_pts, Control* ctl, int n_iter,
                        cudaGraphConditionalHandle cond, cudaStream_t s);
// Trisection (two temperatures per block per iteration).
void launch_kcal_mid(int nblk, const int32_t* Nsp, const float* lo, const float* hi, float* T0,
                     float* T1, Control* ctl, cudaStream_t s);
void launch_kcal_update(int nblk, double inv_count, const double* es, const int32_t* Nsp,
                        const float* T0, const float* T1, float* lo, float* hi, double* ebar0,
                        double* ebar1, Control* ctl, int n_iter, cudaGraphConditionalHandle cond,
                        cudaStream_t s);
void launch_cal_update(int nblk, double inv_count, const double* es, const int32_t* Nsp,
                       const float* T, float* lo, float* hi, double* ebar, Control* ctl,
                       int n_bisect, cudaGraphConditionalHandle cond, cudaStream_t s);
void launch_accumulate(const Geom& g, const uint2* list, int64_t n_list, int colour,
                       const void* ang, int storage, int G, int groups, int r_off, int R,
                       double* sum, cudaStream_t s);
void launch_sum_to_grid(const Geom& g, const uint8_t* mask, const double* sum, double* out,
                        cudaStream_t s);
void launch_grid_to_sum(const Geom& g, const uint8_t* mask, const double* in, double* sum,
                        cudaStream_t s);
// err: 2 per slice (sum |e|, sum e^2 over the slice's gap sites), pre-zeroed.
void launch_predict(const Geom& g, const Slices& sl, const float* values, const uint8_t* mask,
                    const double* sum, double inv_r, float* out, const float* truth, double* err,
                    cudaStream_t s);
void launch_get_state(const Geom& g, const uint8_t* mask, const float* dang, const void* ang,
                      int storage, int G, int r, float* out, cudaStream_t s);
void launch_set_state(const Geom& g, const uint8_t* mask, void* ang, int storage, int G, int r,
                      const float* in, cudaStream_t s);
void launch_block_energy(const Geom& g, const int32_t* of_block, const uint8_t* mask,
                         const float* dang, const void* ang, int storage, int G, int r, double q,
                         double J, double* E, cudaStream_t s);

// Sec. 2.2.3 site temperatures: Ts (FP64, H*W) smoothed from T_blk, then
// Tf = (float)Ts and beta = 1 / Tf; tmp is H*W doubles of scratch.
void launch_sst(const Geom& g, const Slices& sl, const float* T_blk, int r, int n_s, double* Ts,
                double* tmp, float* Tf, float* beta, cudaStream_t s);
void launch_site_beta(int64_t n, const float* Tf, float* beta, cudaStream_t s);

// Energy moments of the calibration chains and the Newton calibration.
void launch_cal_moments(int nblk, int nbx, int Rp, int chains, const double* ecur, double* S,
                        cudaStream_t s);
void launch_moments_final(int nblk, int nbx, double inv_n, const int32_t* Nb, const double* S,
                          double* M, cudaStream_t s);
void launch_newton_update(int nblk, const double* es, const int32_t* Nsp, const int32_t* Nb,
                          const double* M, float* T, double t_lo, double t_hi, cudaStream_t s);
void launch_newton_init(int nblk, float t_init, float t_lo, float t_hi, float* T, float* lo,
                        float* hi, cudaStream_t s);
void launch_energy_vjp(int nblk, int nbx, const int32_t* Nb, const double* M, const double* g,
                       double* out, cudaStream_t s);
void launch_set_tag(Control* ctl, uint32_t tag, cudaStream_t s);

// The realizations' stop tail as one cooperative launch (mpr_simtail.cu).
int sim_tail_blocks_per_sm(int G, int storage);
cudaError_t launch_sim_tail(const SimTailArgs& a, int G, int storage, int grid, cudaStream_t s);

// The realizations' stop tail with one CTA per realization pair
// (mpr_pairtail.cu); every pair's running units must fit kPairTailCap.
constexpr int kPairTailCap = 4096;
cudaError_t launch_pair_tail(const SimTailArgs& a, int G, int storage, int n_pairs,
                             cudaStream_t s);

// The staged half-step (mpr_tile.cu): tile shape of a geometry, the staging
// table, the tile-major lists (count, scan with launch_scan, then write), the
// kernel (G = 8 only) and its resident CTAs per SM.
Tiles tile_shape(const Geom& g);
void launch_stage_table(const Geom& g, const uint8_t* mask, const float* dang, float* stab,
                        cudaStream_t s);
void launch_tile_count(const Geom& g, const Tiles& tl, const int32_t* of_block,
                       const uint8_t* mask, int32_t* cnt0, int32_t* cnt1, cudaStream_t s);
void launch_tile_lists(const Geom& g, const Tiles& tl, const int32_t* of_block,
                       const uint8_t* mask, const int32_t* start0, const int32_t* start1,
                       uint2* list0, uint2* list1, cudaStream_t s);
int tile_blocks_per_sm(int storage);
void launch_sweep_tile(const SweepArgs& a, int storage, int grid, cudaStream_t s);

int cal_persistent_blocks_per_sm(int G);
cudaError_t launch_cal_persistent(const CalPersistArgs& a, int G, int grid, cudaStream_t s);

}  // namespace mpr
