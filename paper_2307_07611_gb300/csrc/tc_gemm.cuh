// tc_gemm.cuh -- interface of the tcgen05 split-BF16 product kernel (tc_gemm.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <vector>

#include "internal.cuh"

namespace triinv {
namespace tc {

constexpr int BM = 128;   // rows of an output tile (UMMA M)
constexpr int BN = 256;   // columns of an output tile (UMMA N)
constexpr int BK = 64;    // k-block staged per pipeline slot (one 128-byte swizzle row)

// One output tile: operand A rows [am, am+128) and columns ak + [kb0*64, kb1*64);
// operand B rows bk + [kb0*64, kb1*64) and columns [bn, bn+256); output origin (om, on);
// b: matrix of a batch (planes and outputs offset by b times their batch strides).
// MODE_LVL only: kind 0 = a W tile, 1 = an X21 tile; before loading its operands the tile
// waits until counter wait0 (wait1) of Epi::cnt reaches need0 (need1) (-1: no wait), and
// after storing it adds one per epilogue warp to counter pub (-1: none).
struct Tile {
    int am, ak, bk, bn, kb0, kb1, om, on;
    int b = 0;
    int kind = 0;
    int wait0 = -1, need0 = 0, wait1 = -1, need1 = 0;
    int pub = -1;
};

// Products summed into one FP32 accumulator: sum_t A_{a[t]} * B_{b[t]}.
struct Terms {
    int n;
    int a[6];
    int b[6];
};

// Epilogue targets (see the modes in tc_gemm.cu).
struct Epi {
    float *x;          // FP32 matrix (lower view through TRANS), leading dimension ldx
    int64_t ldx;
    __nv_bfloat16 *o0, *o1, *o2;   // BF16 output planes, column-major, leading dim ldo
    int64_t ldo;
    int64_t mlim, nlim;            // output rows / columns that exist
    float alpha = 1.f, beta = 0.f; // MODE_GEN: x <- alpha * acc + beta * x
    int cmask = 0;                 // MODE_GEN: part of x written: 0 full, 1 lower, 2 upper,
                                   // 3 / 4 strict lower / upper with a zero diagonal
    float dadd = 0.f;              // MODE_GEN (cmask 0..2): added to diagonal entries
    int64_t xs = 0, os = 0;        // batch strides (elements) of x and of the output planes
    const int *skip = nullptr;     // MODE_RES: skip_n flags per matrix of the batch; a matrix
    int skip_n = 0;                // with a flag set gets R = 0 (its Newton-Schulz step is a no-op)
    int *cnt = nullptr;            // MODE_LVL: the dependency counters the tiles wait on / add to
};

enum Mode {
    MODE_W = 0,      // o0/o1 <- hi/lo BF16 split of acc                    (W = B X_A)
    MODE_X21 = 1,    // x <- -acc; o0/o1/o2 <- hi/mid/lo split of -acc      (X21 = -X_C W)
    MODE_RES = 2,    // o0 (o1) <- hi (lo) split of I - acc (lower), 0 above (R = I - T X)
    MODE_UPD = 3,    // x += acc on the lower triangle                       (X += X R)
    MODE_F32 = 4,    // x <- acc (plain column-major store, no view)        (verification)
    MODE_GEN = 5,    // x <- alpha acc + beta x, column-major, masked        (general products)
    MODE_GENP = 6,   // MODE_GEN with fused stages and FP32 promotion of the partial sums
                     // every 64 k (the six-term products that must reach ~2^-24)
    MODE_W6 = 7,     // MODE_W with six promoted terms; o0/o1/o2 <- hi/mid/lo  (direct recipe)
    MODE_X216 = 8,   // MODE_X21 with six promoted terms                       (direct recipe)
    MODE_LVL = 9,    // W tiles (kind 0, as MODE_W, epilogue targets of the first Epi) and
                     // X21 tiles (kind 1, as MODE_X21, second Epi) of several split levels in
                     // one launch, ordered by their data dependencies (see Tile); A maps
                     // T0 T1 X0 X1, B maps X0 X1 W0 W1, the X21 terms offset by two planes
};

// A column-major BF16 plane usable as a TMA source: rows x cols, leading dimension ld
// (elements, multiple of 8), device pointer 16-byte aligned.
// batch > 1: `batch` such planes, bstride elements apart (multiple of 8).
struct Plane {
    const __nv_bfloat16 *p;
    int64_t rows, cols, ld;
    int64_t batch = 1, bstride = 0;
};

// Encodes a TMA map over a column-major BF16 plane (inner dimension = rows, 128-byte or
// 64-byte swizzle, zero fill outside the plane) with box box_rows x box_cols: 2-D, or
// 3-D with the batch as the outer dimension (box depth 1) when p.batch > 1.  False if the
// driver entry point is missing or the plane violates the TMA alignment rules.
bool encode_plane(CUtensorMap *m, const Plane &p, int box_rows, int box_cols, bool swizzle64 = false);

// Greedy longest-processing-time assignment of tiles to `ctas` persistent CTAs: tiles are
// reordered so that CTA b owns [offsets[b], offsets[b+1]), each list longest first.  The
// cost of a tile is its number of pipeline slots (k-blocks x terms) plus a fixed
// epilogue cost.  Returns the number of CTAs that received work.
int schedule_lpt(std::vector<Tile> &tiles, int terms, int ctas, std::vector<int> &offsets);

// Encodes the tensor maps, then launches `ctas` persistent CTAs; CTA b processes the
// tiles d_tiles[d_off[b] .. d_off[b+1]).  aplanes/bplanes: up to 3 planes each, indexed
// by `terms`.
// bn: columns of the output tiles the list was built with: BN, or 128 / 64 for the level
// products (MODE_W, MODE_X21, MODE_W6, MODE_X216).
// pair: the list holds 256-row tiles (BN wide; MODE_W, MODE_X21, MODE_RES, MODE_UPD), each
// computed by a cluster of two CTAs; `ctas` is twice the number of lists.
// MODE_LVL: na = nb = 4, bn = 128, epi2 = the X21 tiles' epilogue targets; every CTA of the
// launch must be resident at once (ctas <= SMs; one CTA per SM), since tiles wait on tiles
// of other CTAs (waits are bounded: TRI_ERR_TIMEOUT otherwise).
cudaError_t launch_tc(const Ctx &c, int mode, bool trans, bool unit, const Plane *aplanes,
                      int na, const Plane *bplanes, int nb, const Terms &terms,
                      const Tile *d_tiles, const int *d_off, int ctas, const Epi &epi,
                      double flops, const char *trace_name, int bn = BN, bool pair = false,
                      const Epi *epi2 = nullptr);

// Longest-first assignment like schedule_lpt, for tiles in dependency groups: group g's
// tiles (group[i] = g of tiles[i], groups numbered in dependency order) come after every
// tile of groups < g in each CTA's list; loads carry over from group to group.
int schedule_lpt_groups(std::vector<Tile> &tiles, const std::vector<int> &group, int terms, int ctas,
                        std::vector<int> &offsets);

// Rows of the output tiles of a CTA-pair launch.
constexpr int PAIR_BM = 2 * BM;

// Number of CTA pairs of the product kernel that can run at once on this device (at least
// 1; cached per device).
int pair_lists(const Ctx &c);

}  // namespace tc
}  // namespace triinv
