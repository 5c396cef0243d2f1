// trmm_simt.cu -- K2: the two dense products of one split level on CUDA cores
// (FP32 FFMA or FP64 DFMA), used by the plain TRI_F32 / TRI_F64 paths.
//
// For T = [A 0; B C] with X_A = A^-1 and X_C = C^-1 already in place, the block inverse
// of the proof of the main Theorem (Section 3) and of BRSI (Section 5.2) gives
//     X_21 = -X_C B X_A,
// evaluated as two products (each "triangular times full", Eq. "ptfm": m^3 flops):
//     mode 0:  W   = B * X_A     (X_A lower: column block n0 only needs k >= n0)
//     mode 1:  B  <- -X_C * W    (X_C lower: row block m0 only needs k < m0 + BM)
// Every pair of a level (and every matrix of a strided batch) is one more product of the
// same shape, so a level is one launch of the generic triangular-aware product
// (gemm_simt.cu) over all full pairs, plus one for a ragged last pair.  For an upper
// matrix (the transposed lower view) mode 0 reads transposed operands and mode 1
// computes the transposed product, so that every store stays column-major.
#include <algorithm>

#include "gemm.cuh"

namespace triinv {

cudaError_t launch_trmm_level(const Ctx &c, tri_dtype dt, bool trans, bool unit, int mode,
                              int64_t n, void *a, int64_t lda, int64_t h, void *w,
                              int64_t batch, int64_t bstride) {
    const int64_t pairs = level_pairs(n, h);
    if (pairs <= 0 || batch <= 0) return cudaSuccess;
    const size_t es = dt == TRI_F64 ? 8 : 4;
    const int64_t hc_last = std::min<int64_t>(h, n - (pairs - 1) * 2 * h - h);
    const int64_t full = hc_last == h ? pairs : pairs - 1;
    const int low = unit ? OP_LOWER_UNIT : OP_LOWER;
    const int up = unit ? OP_UPPER_UNIT : OP_UPPER;
    const char *name = dt == TRI_F64 ? (mode == 0 ? "trmm_f64_right" : "trmm_f64_left")
                                     : (mode == 0 ? "trmm_f32_right" : "trmm_f32_left");
    auto at = [&](int64_t i, int64_t j) { return (void *)((uint8_t *)a + vidx<false>(i, j, lda) * es); };
    auto wq = [&](int64_t q) { return (void *)((uint8_t *)w + q * h * h * es); };
    const int64_t pstride = 2 * h + 2 * h * lda;      // one pair further along the diagonal
    for (int part = 0; part < 2; ++part) {
        const int64_t q0 = part == 0 ? 0 : full;
        const int64_t np = part == 0 ? full : pairs - full;
        if (np <= 0) continue;
        const int64_t hc = part == 0 ? h : hc_last;
        const int64_t a0 = q0 * 2 * h, c0 = a0 + h;
        GemmArgs g{};
        if (mode == 0) {
            // W = B X_A: B = view(c0 + m, a0 + k), X_A = view(a0 + k, a0 + n), lower.
            g = GemmArgs{hc, h, h, 1.0, trans ? at(a0, c0) : at(c0, a0), lda, OP_FULL,
                         at(a0, a0), lda, low, 0.0, wq(q0), h, OP_FULL};
            g.ta = trans;
            g.tb = trans;
        } else if (!trans) {
            // B <- -X_C W: X_C = view(c0 + m, c0 + k), lower; C column-major at (c0, a0).
            g = GemmArgs{hc, h, hc, -1.0, at(c0, c0), lda, low, wq(q0), h, OP_FULL, 0.0, at(c0, a0), lda,
                         OP_FULL};
        } else {
            // Transposed: (X21)^T = -W^T X_C^T, stored column-major at a + a0 + c0 * lda.
            g = GemmArgs{h, hc, hc, -1.0, wq(q0), h, OP_FULL, at(c0, c0), lda, up, 0.0, at(a0, c0), lda,
                         OP_FULL};
            g.ta = true;
        }
        g.batch = np;
        g.sa = mode == 0 ? pstride : (trans ? h * h : pstride);
        g.sb = mode == 0 ? pstride : (trans ? pstride : h * h);
        g.sc = mode == 0 ? h * h : pstride;
        g.batch2 = batch;
        const int64_t wstride = pairs * h * h;
        g.sa2 = mode == 0 ? bstride : (trans ? wstride : bstride);
        g.sb2 = mode == 0 ? bstride : (trans ? bstride : wstride);
        g.sc2 = mode == 0 ? wstride : bstride;
        cudaError_t e = gemm_simt(c, dt, g, name);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace triinv
