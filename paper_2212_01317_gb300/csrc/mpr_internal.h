// Internal layouts shared by the sm_103a kernels and the C-ABI host code.
//
// Device memory of one context (one field):
//   dang   [2][H][Wh] float   sample angles per checkerboard colour (0 at gaps)
//   dcs    [2][H][Wh] float2  (cos q*phi, sin q*phi) of sample sites
//   list_c [n_gap_c]  uint2   gap sites of colour c, block-major, row-major
//                             within a block: .x = y << 16 | x, .y = b << 10 | flags
//   start_c[nblk+1]   int32   list_c segment of every block
//   ang    [groups][2][H][Wh][G]  gap angles of the batch: realization
//                             r = group * G + lane lives in lane r % G of group
//                             r / G; sample entries are never read or written
//   eacc   [nblk][Rp] double  per-sweep sums of the bond energies that involve a
//                             gap site, owned by each block (Rp = groups * G)
//   running[nblk][Rp] uint8   1 while block b of realization r still sweeps
// Wh = ceil(W/2); site (y,x) of colour c = (x+y)&1 sits at half index x >> 1.
#pragma once
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
};

struct Model {
    float q, J, inv_q;
    int overrelax;
};

// One half-step over the gap sites of one colour, all realizations of a batch.
struct SweepArgs {
    Geom g;
    Model m;
    Rng rng;
    int colour;
    const uint2* list;        // gap entries of this colour
    const int32_t* start;     // [nblk + 1]
    float* ang;               // batch state (float storage)
    const float2* dcs;        // [2][H][Wh]
    const float* beta;        // [nblk] 1 / T_b
    const uint8_t* running;   // [nblk][Rp] or nullptr (= every block runs)
    double* eacc;             // [nblk][Rp]
    int R, Rp, groups;        // realizations in the batch, padded count, lane groups
    uint32_t r_base;          // global index of batch realization 0 (random stream)
    uint32_t t, tag;          // sweep index and stream tag
    int update;               // 0: bond energies only, no move
    int energy;               // accumulate bond energies into eacc
};

}  // namespace mpr
