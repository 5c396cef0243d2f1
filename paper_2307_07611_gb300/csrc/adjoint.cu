// adjoint.cu -- a7: the adjoint of X = T^-1 and the strided-batched forward.
//
// For a loss with cotangent G = dL/dX, d(T^-1) = -T^-1 dT T^-1 gives
//     dL/dT = -P(X^T G X^T),
// P keeping the free entries of T (its triangle; the diagonal is cleared when it is unit).
// For lower T only tril(G) contributes: (X^T G X^T)_ij with i >= j sums X_ki G_kl X_jl
// over k >= i >= j >= l, i.e. k >= l.  So the kernel evaluates
//     M  = X^T tril(G)          (upper x lower: 2n^3/3 flops)
//     dT = -tril(M X^T)         (full x upper, lower half of the output: n^3/3)
// and symmetrically triu for upper T.  Both products go through the generic
// triangular-aware product (CUDA cores for TRI_F32 / TRI_F64, split-BF16 tensor cores
// with six promoted terms for TRI_F32_MIXED, FP32-class).
#include <algorithm>

#include "gemm.cuh"

namespace triinv {

tri_status run_plain_levels(const Ctx &c, tri_dtype dt, bool trans, bool unit, int64_t n, void *a,
                            int64_t lda, void *ws, int64_t hmax);
tri_status run_mixed_batched(const Ctx &c, bool trans, bool unit, int64_t n, float *a, int64_t lda, int64_t stride,
                             int64_t batch, void *ws);
size_t mixed_batched_ws_bytes(int64_t n, int64_t batch);

namespace {

size_t esz(tri_dtype dt) { return dt == TRI_F64 ? 8 : 4; }
size_t al(size_t x) { return (x + 255) / 256 * 256; }

size_t plain_level_ws(int64_t n, tri_dtype dt) {
    size_t best = 0;
    for (int64_t h = 64; h < n; h *= 2) best = std::max(best, (size_t)(level_pairs(n, h) * h * h) * esz(dt));
    return best;
}

bool bad_enums(tri_uplo u, tri_diag d, tri_dtype t) {
    return !((u == TRI_LOWER || u == TRI_UPPER) && (d == TRI_NONUNIT || d == TRI_UNIT) &&
             (t == TRI_F64 || t == TRI_F32 || t == TRI_F32_MIXED));
}

// Leaf inverses and all split levels for `batch` matrices at once (grid dimension).
tri_status run_plain_batched(const Ctx &c, tri_dtype dt, bool trans, bool unit, int64_t n, void *a,
                             int64_t lda, int64_t stride, int64_t batch, void *ws) {
    if (launch_leaf(c, dt, trans, unit, n, a, lda, 64, batch, stride) != cudaSuccess) return TRI_ERR_CUDA;
    for (int64_t h = 64; h < n; h *= 2) {
        if (launch_trmm_level(c, dt, trans, unit, 0, n, a, lda, h, ws, batch, stride) != cudaSuccess)
            return TRI_ERR_CUDA;
        if (launch_trmm_level(c, dt, trans, unit, 1, n, a, lda, h, ws, batch, stride) != cudaSuccess)
            return TRI_ERR_CUDA;
    }
    return TRI_OK;
}

size_t backward_ws(int64_t n, int64_t batch, tri_dtype dt) {
    size_t m = al((size_t)n * n * esz(dt) * (size_t)batch);
    if (dt == TRI_F32_MIXED) m += al(gemm_tc_ws_bytes(n, n, n, batch));
    return m;
}

tri_status run_backward(const Ctx &c, tri_uplo uplo, tri_diag diag, int64_t n, const void *x, int64_t ldx,
                        int64_t sx, const void *g, int64_t ldg, int64_t sg, void *dt_, int64_t ldd, int64_t sd,
                        int64_t batch, tri_dtype dtype, void *ws) {
    const bool lower = uplo == TRI_LOWER, unit = diag == TRI_UNIT;
    uint8_t *M = (uint8_t *)ws;
    const int64_t ldm = n, sm = n * n;
    void *planes = (uint8_t *)ws + al((size_t)n * n * esz(dtype) * (size_t)batch);
    // op(X) = X^T: upper for lower X, lower for upper X (unit diagonal when T is unit).
    const int xt_kind = lower ? (unit ? OP_UPPER_UNIT : OP_UPPER) : (unit ? OP_LOWER_UNIT : OP_LOWER);
    GemmArgs p1{n, n, n, 1.0, x, ldx, xt_kind, g, ldg, lower ? OP_LOWER : OP_UPPER, 0.0, M, ldm, OP_FULL};
    p1.ta = true;
    p1.batch = batch;
    p1.sa = sx;
    p1.sb = sg;
    p1.sc = sm;
    const int omask = lower ? (unit ? OP_LOWER_UNIT : OP_LOWER) : (unit ? OP_UPPER_UNIT : OP_UPPER);
    GemmArgs p2{n, n, n, -1.0, M, ldm, OP_FULL, x, ldx, xt_kind, 0.0, dt_, ldd, omask};
    p2.tb = true;
    p2.batch = batch;
    p2.sa = sm;
    p2.sb = sx;
    p2.sc = sd;
    cudaError_t e;
    if (dtype == TRI_F32_MIXED && n >= 256) {
        // six promoted terms: the gradient matches the FP32 path's accuracy
        e = gemm_tc(c, p1, 6, planes, "adj:xtg");
        if (e == cudaSuccess) e = gemm_tc(c, p2, 6, planes, "adj:mxt");
    } else {
        const tri_dtype d = dtype == TRI_F64 ? TRI_F64 : TRI_F32;
        e = gemm_simt(c, d, p1, "adj:xtg");
        if (e == cudaSuccess) e = gemm_simt(c, d, p2, "adj:mxt");
    }
    return e == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
}

}  // namespace
}  // namespace triinv

using namespace triinv;

extern "C" {

size_t tri_inv_strided_batched_workspace_size(int64_t n, int64_t batch, tri_dtype dtype) {
    if (n <= 0 || batch <= 0 || bad_enums(TRI_LOWER, TRI_NONUNIT, dtype)) return 0;
    if (dtype == TRI_F32_MIXED && n > 256) return mixed_batched_ws_bytes(n, batch);
    return plain_level_ws(n, dtype == TRI_F64 ? TRI_F64 : TRI_F32) * (size_t)batch;
}

tri_status tri_inv_strided_batched_ex(tri_uplo uplo, tri_diag diag, int64_t n, void *a, int64_t lda,
                                      int64_t stride, int64_t batch, tri_dtype dtype, void *workspace,
                                      size_t ws_bytes, int64_t *d_info, void *stream) {
    if (bad_enums(uplo, diag, dtype) || n < 0 || batch < 0) return TRI_ERR_ARG;
    if (n == 0 || batch == 0) return TRI_OK;
    if (!a || lda < std::max<int64_t>(1, n) || stride < lda * n) return TRI_ERR_ARG;
    if (batch > 65535) return TRI_ERR_UNSUPPORTED;
    const size_t need = tri_inv_strided_batched_workspace_size(n, batch, dtype);
    if (need > 0 && (ws_bytes < need || !workspace || ((uintptr_t)workspace & 255))) return TRI_ERR_NOMEM;
    Ctx c;
    tri_status st = device_ctx_public((cudaStream_t)stream, &c);
    if (st != TRI_OK) return st;
    const bool trans = uplo == TRI_UPPER, unit = diag == TRI_UNIT;
    if ((st = info_begin(c, d_info)) != TRI_OK) return st;
    // Mixed: one launch per product for a whole chunk of matrices (the FP32 levels below
    // the tensor-core size).
    if (dtype == TRI_F32_MIXED && n > 256)
        st = run_mixed_batched(c, trans, unit, n, (float *)a, lda, stride, batch, workspace);
    else
        st = run_plain_batched(c, dtype == TRI_F64 ? TRI_F64 : TRI_F32, trans, unit, n, a, lda, stride, batch,
                               workspace);
    return info_end(c, d_info, st);
}

tri_status tri_inv_strided_batched(tri_uplo uplo, tri_diag diag, int64_t n, void *a, int64_t lda, int64_t stride,
                                   int64_t batch, tri_dtype dtype, void *stream) {
    if (bad_enums(uplo, diag, dtype) || n < 0 || batch < 0) return TRI_ERR_ARG;
    if (n == 0 || batch == 0) return TRI_OK;
    const size_t need = tri_inv_strided_batched_workspace_size(n, batch, dtype);
    cudaStream_t s = (cudaStream_t)stream;
    Ctx c;
    tri_status st = device_ctx_public(s, &c);
    if (st != TRI_OK) return st;
    void *ws = nullptr;
    if (need > 0 && lib_malloc_async(&ws, need, s) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_NOMEM;
    }
    st = tri_inv_strided_batched_ex(uplo, diag, n, a, lda, stride, batch, dtype, ws, need, nullptr, stream);
    if (ws && cudaFreeAsync(ws, s) != cudaSuccess && st == TRI_OK) st = TRI_ERR_CUDA;
    return st;
}

size_t tri_inv_backward_workspace_size(int64_t n, int64_t batch, tri_dtype dtype) {
    if (n <= 0 || batch <= 0 || bad_enums(TRI_LOWER, TRI_NONUNIT, dtype)) return 0;
    return backward_ws(n, batch, dtype);
}

tri_status tri_inv_backward_strided_batched_ex(tri_uplo uplo, tri_diag diag, int64_t n, const void *x, int64_t ldx,
                                               int64_t stride_x, const void *g, int64_t ldg, int64_t stride_g,
                                               void *dt, int64_t lddt, int64_t stride_dt, int64_t batch,
                                               tri_dtype dtype, void *workspace, size_t ws_bytes, void *stream) {
    if (bad_enums(uplo, diag, dtype) || n < 0 || batch < 0) return TRI_ERR_ARG;
    if (n == 0 || batch == 0) return TRI_OK;
    const int64_t mn = std::max<int64_t>(1, n);
    if (!x || !g || !dt || ldx < mn || ldg < mn || lddt < mn) return TRI_ERR_ARG;
    if (batch > 1 && (stride_x < ldx * n || stride_g < ldg * n || stride_dt < lddt * n)) return TRI_ERR_ARG;
    if (batch > 65535) return TRI_ERR_UNSUPPORTED;
    if (ws_bytes < backward_ws(n, batch, dtype) || !workspace || ((uintptr_t)workspace & 255)) return TRI_ERR_NOMEM;
    Ctx c;
    tri_status st = device_ctx_public((cudaStream_t)stream, &c);
    if (st != TRI_OK) return st;
    return run_backward(c, uplo, diag, n, x, ldx, stride_x, g, ldg, stride_g, dt, lddt, stride_dt, batch, dtype,
                        workspace);
}

tri_status tri_inv_backward_strided_batched(tri_uplo uplo, tri_diag diag, int64_t n, const void *x, int64_t ldx,
                                            int64_t stride_x, const void *g, int64_t ldg, int64_t stride_g,
                                            void *dt, int64_t lddt, int64_t stride_dt, int64_t batch,
                                            tri_dtype dtype, void *stream) {
    if (bad_enums(uplo, diag, dtype) || n < 0 || batch < 0) return TRI_ERR_ARG;
    if (n == 0 || batch == 0) return TRI_OK;
    cudaStream_t s = (cudaStream_t)stream;
    Ctx c;
    tri_status st = device_ctx_public(s, &c);
    if (st != TRI_OK) return st;
    const size_t need = backward_ws(n, batch, dtype);
    void *ws = nullptr;
    if (lib_malloc_async(&ws, need, s) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_NOMEM;
    }
    st = tri_inv_backward_strided_batched_ex(uplo, diag, n, x, ldx, stride_x, g, ldg, stride_g, dt, lddt, stride_dt,
                                             batch, dtype, ws, need, stream);
    if (cudaFreeAsync(ws, s) != cudaSuccess && st == TRI_OK) st = TRI_ERR_CUDA;
    return st;
}

tri_status tri_inv_backward(tri_uplo uplo, tri_diag diag, int64_t n, const void *x, int64_t ldx, const void *g,
                            int64_t ldg, void *dt, int64_t lddt, tri_dtype dtype, void *stream) {
    return tri_inv_backward_strided_batched(uplo, diag, n, x, ldx, 0, g, ldg, 0, dt, lddt, 0, 1, dtype, stream);
}

}  // extern "C"
