// combrit.cu -- Algorithm COMBRIT (Section 4.1) with beta blocks per level (beta = 2, 4, 8, 16),
// on CUDA cores (FP32 FFMA / FP64 DFMA).
//
// A lower triangular T of order n is walked bottom-up: the leaves (64, or 16 in FP64) are
// inverted by the CRIT recurrence (leaf.cu), then level by level groups of beta diagonal
// blocks of size b, whose inverses X_ii are already in place, become one block of size
// beta * b:
//   1. scale each block row to unit form:  B_ij = X_ii T_ij          (i > j; the unit
//      block matrix T* of Section 4.1)
//   2. invert the unit block matrix (block version of the main Theorem, Section 3, summed
//      by distance from the diagonal, which groups the Hopscotch paths by their first
//      step):  W_ij = -B_ij - sum_{k=j+1}^{i-1} B_ik W_kj
//   3. undo the scaling from the right:     X_ij = W_ij X_jj
// since T = D B with D = diag(T_ii), so T^-1 = B^-1 D^-1.  For beta = 2 this is the split
// of the main path.  Every product of one (i, j) is one launch of the generic product over
// all full groups of the level, plus one for a ragged last group.  An upper matrix runs
// the transposed formulas on its stored blocks, so every store stays column-major.
#include <algorithm>
#include <vector>

#include "gemm.cuh"

namespace triinv {

namespace {

// dst <- dst - src for rows x cols blocks (column-major, leading dims ldd / lds), `count`
// blocks sd / ss elements apart.
template <typename T>
__global__ void sub_block_kernel(T *dst, int64_t ldd, int64_t sd, const T *src, int64_t lds, int64_t ss,
                                 int64_t rows, int64_t cols) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = blockIdx.y;
    if (i >= rows) return;
    const int64_t z = blockIdx.z;
    dst[z * sd + i + j * ldd] -= src[z * ss + i + j * lds];
}

cudaError_t sub_blocks(const Ctx &c, tri_dtype dt, void *dst, int64_t ldd, int64_t sd, const void *src, int64_t lds,
                       int64_t ss, int64_t rows, int64_t cols, int64_t count) {
    if (rows <= 0 || cols <= 0 || count <= 0) return cudaSuccess;
    if (cols > 65535 || count > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((rows + 255) / 256), (unsigned)cols, (unsigned)count);
    if (dt == TRI_F64)
        sub_block_kernel<double><<<grid, 256, 0, c.stream>>>((double *)dst, ldd, sd, (const double *)src, lds, ss,
                                                            rows, cols);
    else
        sub_block_kernel<float><<<grid, 256, 0, c.stream>>>((float *)dst, ldd, sd, (const float *)src, lds, ss,
                                                           rows, cols);
    return cudaGetLastError();
}

int leaf_size(tri_dtype dt) { return dt == TRI_F64 ? 16 : 64; }

}  // namespace

// Scratch: the B and W blocks of every group of the widest level.
size_t combrit_ws_bytes(int64_t n, tri_dtype dt, int beta) {
    const size_t es = dt == TRI_F64 ? 8 : 4;
    const int64_t nblk = (int64_t)beta * (beta - 1) / 2;
    size_t best = 0;
    for (int64_t b = leaf_size(dt); b < n; b *= beta) {
        const int64_t groups = (n + beta * b - 1) / (beta * b);
        best = std::max(best, (size_t)(2 * groups * nblk) * (size_t)(b * b) * es);
    }
    return best;
}

cudaError_t launch_leaf(const Ctx &c, tri_dtype dt, bool trans, bool unit, int64_t n, void *a, int64_t lda, int leaf,
                        int64_t batch, int64_t bstride);

tri_status run_combrit(const Ctx &c, tri_dtype dt, bool trans, bool unit, int64_t n, void *a, int64_t lda, int beta,
                       void *ws) {
    const size_t es = dt == TRI_F64 ? 8 : 4;
    if (launch_leaf(c, dt, trans, unit, n, a, lda, leaf_size(dt), 1, 0) != cudaSuccess) return TRI_ERR_CUDA;
    const int low = unit ? OP_LOWER_UNIT : OP_LOWER, up = unit ? OP_UPPER_UNIT : OP_UPPER;
    const int64_t nblk = (int64_t)beta * (beta - 1) / 2;
    auto bidx = [](int i, int j) { return (int64_t)i * (i - 1) / 2 + j; };   // i > j
    const char *name = dt == TRI_F64 ? "combrit_f64" : "combrit_f32";
    for (int64_t b = leaf_size(dt); b < n; b *= beta) {
        const int64_t gs = beta * b;                     // order of a group
        const int64_t groups = (n + gs - 1) / gs, full = n / gs;
        const int64_t wgrp = nblk * b * b;               // scratch elements of one group
        uint8_t *Bw = (uint8_t *)ws, *Ww = (uint8_t *)ws + (size_t)groups * wgrp * es;
        // storage block (r, c) of the lower view (the stored block (c, r) when trans)
        auto blk = [&](int64_t g, int r, int cc) -> void * {
            const int64_t o = g * gs, i0 = o + (int64_t)r * b, j0 = o + (int64_t)cc * b;
            return (uint8_t *)a + (trans ? (j0 + i0 * lda) : (i0 + j0 * lda)) * es;
        };
        auto bw = [&](uint8_t *base, int64_t g, int i, int j) -> void * {
            return base + (size_t)(g * wgrp + bidx(i, j) * b * b) * es;
        };
        const int64_t gstride = gs + gs * lda;           // one group along the diagonal
        for (int part = 0; part < 2; ++part) {
            const int64_t g0 = part == 0 ? 0 : full, count = part == 0 ? full : groups - full;
            if (count <= 0) continue;
            auto sz = [&](int i) { return std::max<int64_t>(0, std::min<int64_t>(b, n - g0 * gs - (int64_t)i * b)); };
            auto gemm = [&](int64_t m, int64_t nn, int64_t k, double alpha, const void *A, int64_t lda_, int ak,
                            int64_t sa, const void *B, int64_t ldb_, int bk, int64_t sb, double beta_, void *C,
                            int64_t ldc_, int64_t sc) {
                if (m <= 0 || nn <= 0 || k <= 0) return cudaSuccess;
                GemmArgs g{m, nn, k, alpha, A, lda_, ak, B, ldb_, bk, beta_, C, ldc_, OP_FULL};
                g.batch = count;
                g.sa = sa;
                g.sb = sb;
                g.sc = sc;
                return gemm_simt(c, dt, g, name);
            };
            cudaError_t e = cudaSuccess;
            // 1. B_ij = X_ii T_ij   (trans: Bt_ij = T_stored(j,i) XU_ii)
            for (int i = 1; i < beta && e == cudaSuccess; ++i)
                for (int j = 0; j < i && e == cudaSuccess; ++j) {
                    const int64_t si = sz(i), sj = sz(j);
                    if (!trans)
                        e = gemm(si, sj, si, 1.0, blk(g0, i, i), lda, low, gstride, blk(g0, i, j), lda, OP_FULL, gstride,
                                 0.0, bw(Bw, g0, i, j), b, wgrp);
                    else
                        e = gemm(sj, si, si, 1.0, blk(g0, i, j), lda, OP_FULL, gstride, blk(g0, i, i), lda, up, gstride,
                                 0.0, bw(Bw, g0, i, j), b, wgrp);
                }
            // 2. W_ij = -B_ij - sum_k B_ik W_kj, by distance d = i - j >= 2 (d = 1: W = -B,
            //    folded into step 3).  trans: Wt_ij = -Bt_ij - sum_k Wt_kj Bt_ik.
            for (int d = 2; d < beta && e == cudaSuccess; ++d)
                for (int j = 0; j + d < beta && e == cudaSuccess; ++j) {
                    const int i = j + d;
                    const int64_t si = sz(i), sj = sz(j);
                    const int64_t rows = trans ? sj : si, cols = trans ? si : sj;
                    for (int k = j + 1; k < i && e == cudaSuccess; ++k) {
                        const int64_t sk = sz(k);
                        // W_kj with d' = k - j: stored in W if d' >= 2, else -B_kj
                        const bool wk = k - j >= 2;
                        const void *Wkj = wk ? bw(Ww, g0, k, j) : bw(Bw, g0, k, j);
                        const double al = wk ? -1.0 : 1.0;      // -B_ik W_kj, W_kj = -B_kj when d' = 1
                        const double be = k == j + 1 ? 0.0 : 1.0;
                        if (!trans)
                            e = gemm(si, sj, sk, al, bw(Bw, g0, i, k), b, OP_FULL, wgrp, Wkj, b, OP_FULL, wgrp, be,
                                     bw(Ww, g0, i, j), b, wgrp);
                        else
                            e = gemm(sj, si, sk, al, Wkj, b, OP_FULL, wgrp, bw(Bw, g0, i, k), b, OP_FULL, wgrp, be,
                                     bw(Ww, g0, i, j), b, wgrp);
                    }
                    if (e == cudaSuccess)
                        e = sub_blocks(c, dt, bw(Ww, g0, i, j), b, wgrp, bw(Bw, g0, i, j), b, wgrp, rows, cols, count);
                }
            // 3. X_ij = W_ij X_jj  (trans: Xt_ij = XU_jj Wt_ij), over T_ij in place.
            for (int i = 1; i < beta && e == cudaSuccess; ++i)
                for (int j = 0; j < i && e == cudaSuccess; ++j) {
                    const int64_t si = sz(i), sj = sz(j);
                    const bool d1 = i - j == 1;
                    const void *Wij = d1 ? bw(Bw, g0, i, j) : bw(Ww, g0, i, j);
                    const double al = d1 ? -1.0 : 1.0;
                    if (!trans)
                        e = gemm(si, sj, sj, al, Wij, b, OP_FULL, wgrp, blk(g0, j, j), lda, low, gstride, 0.0,
                                 blk(g0, i, j), lda, gstride);
                    else
                        e = gemm(sj, si, sj, al, blk(g0, j, j), lda, up, gstride, Wij, b, OP_FULL, wgrp, 0.0,
                                 blk(g0, i, j), lda, gstride);
                }
            if (e != cudaSuccess) return TRI_ERR_CUDA;
        }
    }
    return TRI_OK;
}

}  // namespace triinv
