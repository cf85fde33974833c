// Internal layouts shared by the sm_103a kernels and the C-ABI host code.
//
// Device memory of one context (one field):
//   dang   [2][H][Wh] float   sample angles per checkerboard colour (0 at gaps)
//   list_c [n_gap_c]  uint2   gap sites of colour c, block-major, row-major
//                             within a block: .x = y << 16 | x, .y = b << 10 | flags
//   start_c[nblk+1]   int32   list_c segment of every block
//   ang    [groups][2][H][Wh][G]  angles of the batch (FP32, FP16 or BF16):
//                             realization r = group * G + lane lives in lane
//                             r % G of group r / G; the FP32 form also holds
//                             the sample angles there, the 16-bit forms read
//                             samples from dang only
//   eacc   [nblk][Rp] double  per-sweep energy change of each block (Rp = groups * G)
//   ecur   [nblk][Rp] double  current block energy E_b
//   running[nblk][Rp] uint8   1 while block b of realization r still sweeps
// Wh = ceil(W/2); site (y,x) of colour c = (x+y)&1 sits at half index x >> 1.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mpr {

// Low bits of a list entry's .y word.
enum : uint32_t {
    NB_L = 1u << 0,   // left neighbour exists
    NB_R = 1u << 1,
    NB_U = 1u << 2,
    NB_D = 1u << 3,
    GAP_L = 1u << 4,  // left neighbour is a gap site
    GAP_R = 1u << 5,
    GAP_U = 1u << 6,
    GAP_D = 1u << 7,
    EDGE_L = 1u << 8, // left bond is owned by block b - 1 (x % l_b == 0, x > 0)
    EDGE_U = 1u << 9, // up bond is owned by block b - nbx (y % l_b == 0, y > 0)
};
constexpr int META_SHIFT = 10;
constexpr int MAX_BLOCKS = 1 << 22;
constexpr int MAX_SIDE = 32768;

struct Geom {
    int H, W, Wh, lb, nbx, nby, nblk;
};

struct Rng {
    uint32_t key0, key1;
    uint32_t rk0[10];          // round keys of key word 0: key0 + r * 0x9E3779B9
};

// Mask values of the canvas: 0 sample, 1 gap (prediction site), 2 absent
// (no site: the padding between the fields packed into one canvas).
constexpr uint8_t MASK_GAP = 1;
constexpr uint8_t MASK_ABSENT = 2;

// Independent fields (slices) packed into one canvas. A slice occupies a
// rectangle of whole blocks whose origin has y0 + x0 even (so a site's
// checkerboard colour is the same in the canvas and in its own field); the
// sites of the rectangle outside the field are absent. No bond joins two
// slices. Every slice keeps its own transform range, random-stream key and
// site numbering, so a slice of a batch computes what its field computes
// alone. A single field is the one-slice case.
struct Slices {
    int n;
    int4 rect0;                // rect[0] and key1[0], read from the kernel parameters
    uint32_t key1_0;           // when n == 1 (no table lookups on the hot path)
    const int4* rect;          // [n] (y0, x0, H_s, W_s): the field's sites in the canvas
    const int4* blk;           // [n] (by0, bx0, nby_s, nbx_s): the slice's blocks
    const int32_t* of_block;   // [nblk] slice of every block, -1 for padding blocks
    const uint32_t* key1;      // [n] Philox key word 1 (seed_hi ^ slice id)
    const double* zmin;        // [n] Sec. 2.1 range over the slice's samples
    const double* zmax;        // [n]
    const int32_t* degenerate; // [n] 1: z_max == z_min
};

// Slice s's rectangle and key word (the one-field case without a lookup).
__device__ __forceinline__ int4 slice_rect(const Slices& sl, int s) {
    return sl.n == 1 ? sl.rect0 : sl.rect[s];
}
__device__ __forceinline__ uint32_t slice_key1(const Slices& sl, int s) {
    return sl.n == 1 ? sl.key1_0 : sl.key1[s];
}
__device__ __forceinline__ int slice_of(const Slices& sl, int b) {
    return sl.n == 1 ? 0 : sl.of_block[b];
}

// Philox counter word 0 of a site: its index within its own field.
__host__ __device__ inline uint32_t local_index(const int4& rc, int y, int x) {
    return (uint32_t)(y - rc.x) * (uint32_t)rc.w + (uint32_t)(x - rc.y);
}

struct Model {
    float q, J, inv_q;
    int overrelax;
};

// Device-resident loop state of a batch. Kernels read the sweep index, the
// random-stream tag and the worklist size from here, so sweeps need no new
// launch parameters. The worklist is double-buffered by sweep parity: sweep t
// reads list t & 1, and its stop test writes list (t + 1) & 1.
struct Control {
    uint32_t t;                  // sweep index of the sweep in progress
    uint32_t tag;                // random-stream tag (0 realizations, 1 + k calibration)
    uint32_t k;                  // calibration iteration
    uint32_t n_work[2];          // worklist sizes by sweep parity
    uint32_t energy_dirty;       // state was overwritten: energies must be recomputed
    uint32_t ticket;             // CTAs of the closing stop kernel that have finished
    uint32_t t_tail;             // the pair-per-CTA stop tail: latest sweep index reached
    unsigned long long n_running;      // running (block, realization) pairs after the last stop test
    unsigned long long n_running_acc;  // the same, being counted by the stop test in progress
};

// Tiles of the staged half-step: every block is cut into tiles of th rows and
// tw columns (the last ones of a block partial), numbered block-major, then
// row-major within the block. Each colour has its own list of gap entries in
// tile order (within a tile: the block-edge entries first, then row-major)
// with segment starts per tile.
constexpr int kTileRows = 16;          // th = min(l_b, kTileRows)
constexpr int kTileCols = 32;          // tw = min(l_b, kTileCols)
constexpr int kTileStageRows = kTileRows + 2;
constexpr int kTileStageCols = kTileCols / 2 + 2;   // staged half-columns, at most

struct Tiles {
    int th, tw;                // tile rows / columns in sites
    int tpx, tpy;              // tiles per block across / down
    int n;                     // tiles of the canvas: nblk * tpx * tpy
    const int32_t* start;      // [n + 1] segments of this colour's tile list
    const uint2* list;         // gap entries of this colour, tile-major
    const float* stab;         // [2][H][Wh] staging table: the sample angle at a
                               // sample site, NaN at a gap site, -1 at an absent
                               // site and at the padding half-site of odd widths
};

// One half-step over the gap sites of one colour, for every running
// (block, realization pair) unit of the worklist.
struct SweepArgs {
    Geom g;
    Model m;
    Rng rng;                  // key0 (seed_lo); key1 comes from the slice table
    Slices sl;
    int colour;
    const uint2* list;        // gap entries of this colour
    const int32_t* start;     // [nblk + 1]
    const int32_t* split;     // [nblk] end of each block's edge entries
    void* ang;                // batch state [groups][2][H][Wh][G] (FP32, FP16 or BF16)
    const float* dang;        // [2][H][Wh] FP32 sample angles (0 at gaps)
    const float* beta;        // [nblk] 1 / T_b
    const float* beta_site;   // [H*W] 1 / T_i (site temperatures, Sec. 2.2.3) or nullptr
    const float* beta_odd;    // [nblk] 1 / T_b of odd lanes (trisection's second point) or nullptr
    const float* beta_pts;    // [n_pts][nblk] 1 / T of the k-point calibration (lane r takes
                              // point r mod n_pts) or nullptr
    int n_pts;
    const uint8_t* running;   // [nblk][Rp] or nullptr (= every lane r < R runs)
    double* eacc;             // [nblk][Rp] energy change of this sweep (moves)
    double* ecur;             // [nblk][Rp] E_b (the energy pass adds into it)
    const uint32_t* work;     // two worklists of units b * (Rp / 2) + pair, or nullptr = all units
    uint32_t work_stride;     // elements per worklist
    const Control* ctl;
    int R, Rp, groups;        // realizations in the batch, padded lanes, lane groups
    uint32_t r_base;          // global index of lane 0 (even)
    int energy;               // 1: accumulate energy increments of the moves
    int t_fixed;              // > 0: sweep index of this launch (else read from ctl)
    Tiles tl;                 // the staged half-step's tiles (tl.n == 0: not built)
};

// The WINDOW stop rule (Sec. 3.4: n_fit, n_f): e_b of the last n_fit sweeps
// of every (block, realization), a ring indexed by sweep mod n_fit.
struct StopWindow {
    int rule;                 // 0 CROSS, 1 WINDOW
    int n_fit, n_f;
    double* hist;             // [n_fit][nblk * Rp]
    size_t stride;            // nblk * Rp
};

// Per-(block, realization) bookkeeping of the stop test (Sec. 3.4 reading):
// the operands of the targeted and the closing parts of a sweep's test.
struct StopArgs {
    int G, groups, Rp, nblk, n_max;
    const int32_t* of_block;  // [nblk] slice of every block
    const double* es;         // [nblk] e_s,b
    const double* inb;       // [nblk] 1 / N_b
    const int32_t* Nsp;       // [nblk] sample bonds (0: not targeted)
    double* eacc;             // [nblk][Rp] the sweep's change (folded and cleared)
    double* ecur;             // [nblk][Rp] E_b
    const int8_t* sigma;      // [nblk][Rp] side of e_s,b at t = 0
    uint8_t* running;         // [nblk][Rp]
    int32_t* stop;            // [nblk][Rp] stop sweep
    int32_t* tcount;          // [n_slices][Rp] running targeted blocks
    double* e_last;           // [nblk][Rp] e_b after the last test
    StopWindow win;           // the stop rule (win.rule == 0: first crossing)
};

// The calibration's per-sweep fold (E_b += the sweep's change; the measured
// sweeps' e_b summed), run by extra CTAs of the next half-step's launch.
struct FoldArgs {
    int ctas;                 // CTAs of the launch that fold (0: none)
    int nblk, Rp, chains, measure;
    int points;               // 2: even / odd lanes are the trisection's two points
    const double* inb;        // [nblk] 1 / N_b
    double* eacc;             // [nblk][Rp] change of the sweep being folded (cleared)
    double* ecur;             // [nblk][Rp]
    double* ebar;             // [nblk] (even lanes when points == 2)
    double* ebar_odd;         // [nblk] odd lanes (points == 2)
    double* ebar_pts;         // [points][nblk] (points > 2: lane r adds to point r mod points)
};

// Grid-wide barrier state of a cooperative launch (zeroed before each launch).
struct GridBarrier {
    unsigned int arrive;   // CTAs arrived at the current barrier
    unsigned int gen;      // barriers completed
    unsigned int err;      // 1: a wait gave up (the launch returned early)
    unsigned int extra;    // test hook: arrivals awaited beyond the grid (0 normally)
};

// The simulation's stop tail as one cooperative launch: sweeps (two
// half-steps over the worklist, then the two parts of the stop test) until
// no pair runs or the sweep index passes n_max, phases separated by grid
// barriers; the barrier closing a sweep also advances the Control.
struct SimTailArgs {
    SweepArgs sw;              // colour-independent sweep fields
    const uint2* list[2];
    const int32_t* start[2];
    const int32_t* split[2];
    StopArgs st;
    Control* ctl;
    uint32_t* work_all;        // the two worklists (sw.work_stride apart)
    GridBarrier* bar;
    unsigned long long spin_limit;
};

// The persistent calibration kernel's arguments.
struct CalPersistArgs {
    SweepArgs sw;              // colour-independent sweep fields (ecur, ang, beta, ...)
    const uint2* list[2];
    const int32_t* start[2];
    const int32_t* split[2];
    int64_t n_list[2];
    double* eacc2[2];          // per-sweep energy changes, by sweep parity
    const double* Es;
    const double* es;
    const double* inb;
    const int32_t* Nsp;
    float* T;
    float* beta;
    float* lo;
    float* hi;
    double* ebar;
    const float* init_angle;
    int chains, n_eq, n_meas, n_bisect, random_init;
    double inv_count;
    GridBarrier* bar;
    unsigned long long spin_limit;
    float* med;                // median of the targeted blocks' T
};

}  // namespace mpr
