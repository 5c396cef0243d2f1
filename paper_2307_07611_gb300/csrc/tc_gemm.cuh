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
struct Tile {
    int am, ak, bk, bn, kb0, kb1, om, on;
    int b = 0;
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
cudaError_t launch_tc(const Ctx &c, int mode, bool trans, bool unit, const Plane *aplanes,
                      int na, const Plane *bplanes, int nb, const Terms &terms,
                      const Tile *d_tiles, const int *d_off, int ctas, const Epi &epi,
                      double flops, const char *trace_name, int bn = BN, bool pair = false);

// Rows of the output tiles of a CTA-pair launch.
constexpr int PAIR_BM = 2 * BM;

// Number of CTA pairs of the product kernel that can run at once on this device (at least
// 1; cached per device).
int pair_lists(const Ctx &c);

}  // namespace tc
}  // namespace triinv
