// brsi.cu -- general inverse by BRSI with gamma blocks (Section 5.2, "Steps of
// BRSI(gamma)"), the block UL-like recursion of the paper, with the column permutation
// P_0 of Step 1.
//
// With the matrix split into nb = gamma blocks (q = ceil(n / gamma) rows, the last one
// ragged), Step 1 sets A_0 = A P_0 and Steps 2-5 repeat, for l = 0 .. nb - 2,
//     A_l = M_l + N_l        M_l: the block upper part of A_l (diagonal blocks included),
//                            N_l: its strictly block lower part,
//     A_{l+1} = I + M_l^-1 N_l.
// N_l has a zero last block column, so each step turns one more trailing block column
// of A_{l+1} into identity columns (above and on the diagonal): only the leading
// "active" part of act_l = b[nb - l] rows and columns changes, and M_l is the identity
// outside it.  After the loop L = A_{nb-1} is block lower triangular with the identity
// on every diagonal block but the first, A P_0 = M_0 ... M_{nb-2} L and
//     A^-1 = P_0 L^-1 M_{nb-2}^-1 ... M_0^-1.
// Per step, on the active part only:
//   M_l^-1   diagonal blocks inverted by gen_inv (the two-block BRSI / block LU route:
//            the "double recursion" of Step 4), off-diagonal blocks by block back
//            substitution, one block row at a time from the bottom:
//                T = M[i, i+1:] Minv[i+1:, i+1:],   Minv[i, i+1:] = -Minv[i, i] T
//   A_{l+1} = I + Minv N     (N: the strictly block lower part of the active square)
//   Y <- Minv Y              (Y accumulates M_l^-1 ... M_0^-1; only the active rows change)
// and at the end Z = L^-1 Y by block forward substitution (L_00 = B inverted by gen_inv,
// L_ii = I for i > 0), then A^-1 = P_0 Z (row j of Z is row perm[j] of A^-1).
// The work grows with gamma (the paper finds gamma = 2 cheapest); all products go
// through the generic product (CUDA cores, or split-BF16 tensor cores for
// TRI_F32_MIXED, which then ends with one Newton-Schulz step against A).
#include <algorithm>
#include <vector>

#include "gemm.cuh"

namespace triinv {

size_t gen_inv_ws_bytes(int64_t n, tri_dtype dt);
tri_status run_gen_inv(const Ctx &c, tri_dtype dt, int64_t n, void *a, int64_t lda, void *ws, int64_t info_base);
tri_status dense_newton_schulz(const Ctx &c, int64_t n, const float *a, int64_t lda, float *x, int64_t ldx,
                               float *r, int64_t ldr, void *planes);

namespace {

size_t al(size_t x) { return (x + 255) / 256 * 256; }
size_t esz(tri_dtype dt) { return dt == TRI_F64 ? 8 : 4; }
constexpr int64_t kTcMin = 512;   // smaller products stay on CUDA cores

std::vector<int64_t> bounds(int64_t n, int gamma) {
    const int64_t q = (n + gamma - 1) / gamma;
    std::vector<int64_t> b;
    for (int i = 0; i <= gamma; ++i) {
        const int64_t v = std::min<int64_t>((int64_t)i * q, n);
        if (b.empty() || v != b.back()) b.push_back(v);
    }
    return b;
}

struct BrsiLayout {
    size_t al_, y, mi, tm, perm, gws, planes, total;
};

BrsiLayout brsi_layout(int64_t n, int gamma, tri_dtype dt) {
    BrsiLayout L{};
    const size_t mat = al((size_t)n * n * esz(dt));
    L.al_ = 0;
    L.y = mat;
    L.mi = 2 * mat;
    L.tm = 3 * mat;
    L.perm = 4 * mat;
    L.gws = L.perm + al((size_t)n * sizeof(int64_t));
    const std::vector<int64_t> b = bounds(n, gamma);
    size_t g = 0;
    for (size_t i = 0; i + 1 < b.size(); ++i) g = std::max(g, gen_inv_ws_bytes(b[i + 1] - b[i], dt));
    L.planes = L.gws + al(g);
    L.total = L.planes + (dt == TRI_F32_MIXED ? al(gemm_tc_ws_bytes(n, n, n)) : 0);
    return L;
}

// dst[:, j] = src[:, perm[j]] (dst leading dimension n)
template <typename T>
__global__ void gather_cols_kernel(T *__restrict__ dst, const T *__restrict__ src, int64_t lds, const int64_t *perm,
                                   int64_t n) {
    const int64_t j = blockIdx.y;
    const int64_t pj = perm ? perm[j] : j;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i + j * n] = src[i + pj * lds];
}

// dst[perm[i], :] = src[i, :] (src leading dimension n)
template <typename T>
__global__ void scatter_rows_kernel(T *__restrict__ dst, int64_t ldd, const T *__restrict__ src, const int64_t *perm,
                                    int64_t n) {
    const int64_t j = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[(perm ? perm[i] : i) + j * ldd] = src[i + j * n];
}

// Block index of row / column i for boundaries of q rows per block.
__device__ __forceinline__ int64_t blk(int64_t i, int64_t q) { return i / q; }

// tm[i, j] = al[i, j] where block(i) > block(j), else 0, on the act x act square.
template <typename T>
__global__ void block_lower_kernel(T *__restrict__ tm, const T *__restrict__ al, int64_t n, int64_t act, int64_t q) {
    const int64_t j = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < act; i += (int64_t)gridDim.x * blockDim.x)
        tm[i + j * n] = blk(i, q) > blk(j, q) ? al[i + j * n] : T(0);
}

// x[i, i] += 1 for i < m (x leading dimension ld)
template <typename T>
__global__ void add_identity_kernel(T *x, int64_t ld, int64_t m) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) x[i + i * ld] += T(1);
}

// x = I on the m x m square (leading dimension ld)
template <typename T>
__global__ void set_identity_kernel(T *x, int64_t ld, int64_t m) {
    const int64_t j = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        x[i + j * ld] = i == j ? T(1) : T(0);
}

struct BrsiCtx {
    const Ctx *c;
    tri_dtype dt;
    void *planes;
};

cudaError_t product(const BrsiCtx &g, const GemmArgs &a, const char *name) {
    if (a.m <= 0 || a.n <= 0) return cudaSuccess;
    if (g.dt == TRI_F32_MIXED && a.m >= kTcMin && a.n >= kTcMin && a.k >= kTcMin)
        return gemm_tc(*g.c, a, 3, g.planes, name);
    return gemm_simt(*g.c, g.dt == TRI_F64 ? TRI_F64 : TRI_F32, a, name);
}

template <typename T>
cudaError_t run_t(const Ctx &c, tri_dtype dt, int64_t n, T *a, int64_t lda, int gamma, const int64_t *dperm,
                  uint8_t *ws) {
    const BrsiLayout L = brsi_layout(n, gamma, dt);
    T *Al = (T *)(ws + L.al_), *Y = (T *)(ws + L.y), *Mi = (T *)(ws + L.mi), *Tm = (T *)(ws + L.tm);
    void *gws = ws + L.gws;
    BrsiCtx g{&c, dt, ws + L.planes};
    const std::vector<int64_t> b = bounds(n, gamma);
    const int nb = (int)b.size() - 1;
    const int64_t q = b[1] - b[0];
    const size_t es = sizeof(T);
    const unsigned gx = (unsigned)std::min<int64_t>((n + 255) / 256, 64);
    auto at = [&](T *m, int64_t i, int64_t j) { return m + i + j * n; };
    TraceScope ts(c.stream, "brsi:setup", 0.0, 0.0);
    // Step 1: A_0 = A P_0;  Y = I
    gather_cols_kernel<T><<<dim3(gx, (unsigned)n), 256, 0, c.stream>>>(Al, a, lda, dperm, n);
    set_identity_kernel<T><<<dim3(gx, (unsigned)n), 256, 0, c.stream>>>(Y, n, n);
    cudaError_t e = cudaGetLastError();
    // Steps 2-5
    for (int l = 0; l + 1 < nb && e == cudaSuccess; ++l) {
        const int na = nb - l;           // active blocks
        const int64_t act = b[na];
        // M_l^-1 on the active square: zero it, diagonal blocks by gen_inv, then back
        // substitution from the last block row up
        e = cudaMemset2DAsync(Mi, n * es, 0, act * es, act, c.stream);
        for (int i = 0; i < na && e == cudaSuccess; ++i) {
            const int64_t r0 = b[i], m = b[i + 1] - b[i];
            e = cudaMemcpy2DAsync(at(Mi, r0, r0), n * es, at(Al, r0, r0), n * es, m * es, m, cudaMemcpyDeviceToDevice,
                                  c.stream);
            if (e == cudaSuccess && run_gen_inv(c, dt, m, at(Mi, r0, r0), n, gws, r0) != TRI_OK) e = cudaErrorUnknown;
        }
        for (int i = na - 2; i >= 0 && e == cudaSuccess; --i) {
            const int64_t r0 = b[i], m = b[i + 1] - b[i], c0 = b[i + 1], w = act - c0;
            // T = M[i, i+1:] Minv[i+1:, i+1:]   (Minv block upper on the rest)
            e = product(g, GemmArgs{m, w, w, 1.0, at(Al, r0, c0), n, OP_FULL, at(Mi, c0, c0), n, OP_FULL, 0.0,
                                    at(Tm, r0, c0), n, OP_FULL}, "brsi:backsub_a");
            // Minv[i, i+1:] = -Minv[i, i] T
            if (e == cudaSuccess)
                e = product(g, GemmArgs{m, w, m, -1.0, at(Mi, r0, r0), n, OP_FULL, at(Tm, r0, c0), n, OP_FULL, 0.0,
                                        at(Mi, r0, c0), n, OP_FULL}, "brsi:backsub_b");
        }
        if (e != cudaSuccess) break;
        // N: strictly block lower part of the active square of A_l
        block_lower_kernel<T><<<dim3(gx, (unsigned)act), 256, 0, c.stream>>>(Tm, Al, n, act, q);
        // A_{l+1} = I + Minv N on the active square (rows and columns beyond it unchanged)
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = product(g, GemmArgs{act, act, act, 1.0, Mi, n, OP_FULL, Tm, n, OP_FULL, 0.0, Al, n, OP_FULL},
                        "brsi:update");
        if (e == cudaSuccess) {
            add_identity_kernel<T><<<(unsigned)((act + 255) / 256), 256, 0, c.stream>>>(Al, n, act);
            e = cudaGetLastError();
        }
        // Y[:act, :] = Minv Y[:act, :]
        if (e == cudaSuccess)
            e = product(g, GemmArgs{act, n, act, 1.0, Mi, n, OP_FULL, Y, n, OP_FULL, 0.0, Tm, n, OP_FULL},
                        "brsi:accumulate");
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(Y, n * es, Tm, n * es, act * es, n, cudaMemcpyDeviceToDevice, c.stream);
    }
    if (e != cudaSuccess) return e;
    // Z = L^-1 Y by block forward substitution, into Tm:  Z_0 = B^-1 Y_0,
    // Z_i = Y_i - L[i, :b_i] Z[:b_i, :] for i > 0
    {
        const int64_t m0 = b[1];
        e = cudaMemcpy2DAsync(Mi, n * es, Al, n * es, m0 * es, m0, cudaMemcpyDeviceToDevice, c.stream);
        if (e == cudaSuccess && run_gen_inv(c, dt, m0, Mi, n, gws, 0) != TRI_OK) e = cudaErrorUnknown;
        if (e == cudaSuccess)
            e = product(g, GemmArgs{m0, n, m0, 1.0, Mi, n, OP_FULL, Y, n, OP_FULL, 0.0, Tm, n, OP_FULL},
                        "brsi:solve0");
        for (int i = 1; i < nb && e == cudaSuccess; ++i) {
            const int64_t r0 = b[i], m = b[i + 1] - b[i];
            e = cudaMemcpy2DAsync(at(Tm, r0, 0), n * es, at(Y, r0, 0), n * es, m * es, n, cudaMemcpyDeviceToDevice,
                                  c.stream);
            if (e == cudaSuccess)
                e = product(g, GemmArgs{m, n, r0, -1.0, at(Al, r0, 0), n, OP_FULL, Tm, n, OP_FULL, 1.0,
                                        at(Tm, r0, 0), n, OP_FULL}, "brsi:solve");
        }
    }
    if (e != cudaSuccess) return e;
    // A^-1 = P_0 Z
    if (dt == TRI_F32_MIXED && n >= kTcMin) {
        // rows into Mi, one Newton-Schulz step against A (still intact), then back over A
        scatter_rows_kernel<T><<<dim3(gx, (unsigned)n), 256, 0, c.stream>>>(Mi, n, Tm, dperm, n);
        e = cudaGetLastError();
        if (e == cudaSuccess &&
            dense_newton_schulz(c, n, (const float *)a, lda, (float *)Mi, n, (float *)Y, n, g.planes) != TRI_OK)
            e = cudaErrorUnknown;
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(a, lda * es, Mi, n * es, n * es, n, cudaMemcpyDeviceToDevice, c.stream);
        return e;
    }
    scatter_rows_kernel<T><<<dim3(gx, (unsigned)n), 256, 0, c.stream>>>(a, lda, Tm, dperm, n);
    return cudaGetLastError();
}

}  // namespace

size_t brsi_ws_bytes(int64_t n, int gamma, tri_dtype dt) { return brsi_layout(n, gamma, dt).total; }

// perm: HOST array or null; uploaded into the workspace (a pageable copy: not inside
// stream capture).
tri_status run_brsi(const Ctx &c, tri_dtype dt, int64_t n, void *a, int64_t lda, int gamma, const int64_t *perm,
                    void *ws) {
    const BrsiLayout L = brsi_layout(n, gamma, dt);
    int64_t *dperm = nullptr;
    if (perm) {
        dperm = (int64_t *)((uint8_t *)ws + L.perm);
        if (cudaMemcpyAsync(dperm, perm, (size_t)n * sizeof(int64_t), cudaMemcpyHostToDevice, c.stream) !=
            cudaSuccess)
            return TRI_ERR_CUDA;
    }
    cudaError_t e = dt == TRI_F64 ? run_t<double>(c, dt, n, (double *)a, lda, gamma, dperm, (uint8_t *)ws)
                                  : run_t<float>(c, dt, n, (float *)a, lda, gamma, dperm, (uint8_t *)ws);
    return e == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
}

}  // namespace triinv
