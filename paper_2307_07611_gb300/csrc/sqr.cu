// sqr.cu -- Algorithm SQR (Section 5.1): A = Q R with the inverse factor S = R^-1 formed
// alongside R, so that A^-1 = S Q^T.
//
// The printed algorithm is modified Gram-Schmidt, one column at a time, each column of S
// computed as soon as the column of R is known.  One column at a time is a chain of
// global reductions on a GPU, so the same factors are built over blocks of columns:
// a recursive column split A = [A1 A2]
//     (Q1, R11, S11) = rec(A1)
//     R12 = Q1^T A2,   A2 <- A2 - Q1 R12         block Gram-Schmidt, run twice (the
//                                                second pass re-orthogonalises and adds
//                                                its coefficients to R12)
//     (Q2, R22, S22) = rec(A2)
//     S12 = -(S11 R12) S22                       the two-block inverse (Section 3 / 4.1)
// so a block column of S is formed as soon as the block column of R is complete, as in
// SQR.  A leaf (at most W columns, all n rows) is orthonormalised by Cholesky QR run
// twice: G = P^T P = R1^T R1,  P <- P R1^-1, and again with R2; its R = R2 R1 and
// S = R1^-1 R2^-1, the triangular inverses by the tiled split of tile_inverse.cuh.  The QR
// with a positive diagonal is unique, so Q, R and S are those of the printed algorithm
// up to rounding.  Cholesky QR needs the leaf panel's condition number below about
// u^-1/2 (Cholesky of the Gram matrix breaks down otherwise); a breakdown (a pivot that is
// not positive and finite) is reported like a zero pivot: the first such column, through
// tri_get_info.
#include <algorithm>
#include <climits>

#include "gemm.cuh"
#include "tile_inverse.cuh"

namespace triinv {
namespace {

constexpr int kPanelThreads = 256;
constexpr int kChunk = 64;          // rows of the panel staged in shared memory at a time
constexpr int kMaxPanelCtas = 64;   // partial Gram matrices reduced by the Cholesky kernel

// One pass over the rows of a leaf panel P (rows x m, m <= W), CTA b taking rows
// [b * rows_per, (b + 1) * rows_per):
//   sapply != null:   P <- P S  (S upper, W x W, leading dimension W)
//   partials != null: the CTA's partial Gram matrix of the (updated) rows, W x W, into
//                     partials + b * W * W
template <typename T, int W>
__global__ void __launch_bounds__(kPanelThreads) qr_panel_kernel(T *p, int64_t ldp, int64_t rows, int m,
                                                                 const T *__restrict__ sapply,
                                                                 T *__restrict__ partials, int64_t rows_per) {
    constexpr int NT = kPanelThreads, CH = kChunk;
    constexpr int AJ = NT / CH;          // column groups of the apply step
    constexpr int AQ = W / AJ;           // outputs per thread per chunk (apply)
    constexpr int GJ = NT / W;           // column groups of the Gram step
    constexpr int GQ = W / GJ;           // Gram entries per thread
    __shared__ T s_s[W][W + 1];
    __shared__ T s_p[CH][W + 1];
    const int tid = threadIdx.x;
    if (sapply)
        for (int idx = tid; idx < W * W; idx += NT) {
            const int i = idx % W, j = idx / W;
            s_s[i][j] = (i <= j && j < m) ? sapply[i + j * W] : T(0);
        }
    T g[GQ];
#pragma unroll
    for (int q = 0; q < GQ; ++q) g[q] = T(0);
    const int gi = tid % W, gj = tid / W;
    const int ar = tid % CH, aj = tid / CH;
    const int64_t r_begin = (int64_t)blockIdx.x * rows_per;
    const int64_t r_end = min(rows, r_begin + rows_per);
    for (int64_t r0 = r_begin; r0 < r_end; r0 += CH) {
        for (int idx = tid; idx < CH * W; idx += NT) {
            const int r = idx % CH, c = idx / CH;
            const int64_t gr = r0 + r;
            s_p[r][c] = (gr < r_end && c < m) ? p[gr + (int64_t)c * ldp] : T(0);
        }
        __syncthreads();
        if (sapply) {
            T acc[AQ];
#pragma unroll
            for (int q = 0; q < AQ; ++q) acc[q] = T(0);
#pragma unroll 8
            for (int k = 0; k < W; ++k) {
                const T v = s_p[ar][k];
#pragma unroll
                for (int q = 0; q < AQ; ++q) acc[q] = fma(v, s_s[k][aj + AJ * q], acc[q]);
            }
            __syncthreads();
            const int64_t gr = r0 + ar;
#pragma unroll
            for (int q = 0; q < AQ; ++q) {
                const int j = aj + AJ * q;
                s_p[ar][j] = acc[q];
                if (gr < r_end && j < m) p[gr + (int64_t)j * ldp] = acc[q];
            }
            __syncthreads();
        }
        if (partials) {
#pragma unroll 4
            for (int r = 0; r < CH; ++r) {
                const T v = s_p[r][gi];
#pragma unroll
                for (int q = 0; q < GQ; ++q) g[q] = fma(v, s_p[r][gj + GJ * q], g[q]);
            }
        }
        __syncthreads();
    }
    if (partials) {
        T *out = partials + (size_t)blockIdx.x * W * W;
#pragma unroll
        for (int q = 0; q < GQ; ++q) out[gi + (gj + GJ * q) * W] = g[q];
    }
}

template <typename T, int W>
constexpr size_t chol_smem() {
    constexpr int nt = W / 32;
    constexpr int tiles = nt * (nt + 1) / 2;
    constexpr int wtiles = (nt / 2) * (nt / 2) > 0 ? (nt / 2) * (nt / 2) : 1;
    return sizeof(T) * (4 * (size_t)W * (W + 1) + 2 * W + (size_t)(tiles + wtiles) * TE);
}

// The Cholesky step of one Cholesky QR pass, one CTA:
//   G = sum of the partial Gram matrices (m x m, identity beyond m),
//   G = R^T R (R upper, positive diagonal), S = R^-1.
// pass 0: S -> sapply, R -> keep.
// pass 1: with S1 = sapply and R1 = keep from pass 0: S2 -> sapply, R2 R1 -> rblk and
//         S1 S2 -> sblk (their m x m upper triangles).
template <typename T, int W>
__global__ void __launch_bounds__(kPanelThreads) qr_chol_kernel(const T *__restrict__ partials, int np, int m,
                                                                int pass, T *sapply, T *keep, T *rblk,
                                                                int64_t ldr, T *sblk, int64_t lds,
                                                                long long *info, int64_t col0) {
    constexpr int NT = kPanelThreads;
    constexpr int EQ = W * W / NT;       // entries per thread
    constexpr int nt = W / 32;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    T (*g)[W + 1] = reinterpret_cast<T (*)[W + 1]>(smem_raw);        // G, then R
    T (*sm)[W + 1] = g + W;                                          // S
    T (*x1)[W + 1] = g + 2 * W;                                      // R1 (pass 1)
    T (*x2)[W + 1] = g + 3 * W;                                      // S1 (pass 1)
    T *rowk = reinterpret_cast<T *>(g + 4 * W);                      // 2 x W
    T *tiles = rowk + 2 * W;
    T *wt = tiles + (size_t)(nt * (nt + 1) / 2) * TE;
    const int tid = threadIdx.x;

    // entries e = tid + NT q:  i = e % W, j = e / W
    T v[EQ];
#pragma unroll
    for (int q = 0; q < EQ; ++q) {
        const int e = tid + NT * q, i = e % W, j = e / W;
        T acc = T(0);
        if (i <= j && j < m)
            for (int b = 0; b < np; ++b) acc += partials[(size_t)b * W * W + e];
        else if (i == j)
            acc = T(1);
        v[q] = acc;
    }
    // Cholesky, right-looking, one barrier per step: the owners of row k publish it,
    // every thread then scales (row k) or updates (rows below) its own entries.
    for (int k = 0; k < m; ++k) {
        T *rk = rowk + (k & 1) * W;
#pragma unroll
        for (int q = 0; q < EQ; ++q) {
            const int e = tid + NT * q, i = e % W, j = e / W;
            if (i == k && j >= k) rk[j] = v[q];
        }
        __syncthreads();
        const T d = rk[k];
        if (tid == 0 && !(d > T(0) && isfinite(d))) atomicMin(info, (long long)(col0 + k));
        const T piv = sqrt(d), rd = T(1) / d;
#pragma unroll
        for (int q = 0; q < EQ; ++q) {
            const int e = tid + NT * q, i = e % W, j = e / W;
            if (i == k && j >= k) v[q] = v[q] / piv;
            else if (i > k && j >= i) v[q] = fma(-rk[i] * rd, rk[j], v[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < EQ; ++q) {
        const int e = tid + NT * q, i = e % W, j = e / W;
        g[i][j] = (i <= j) ? v[q] : T(0);
    }
    __syncthreads();
    // S = R^-1: invert the lower R^T in 32 x 32 tiles, S = ((R^T)^-1)^T.
    for (int idx = tid; idx < (nt * (nt + 1) / 2) * 32 * 32; idx += NT) {
        const int tl = idx / 1024, rc = idx % 1024, r = rc / 32, c = rc % 32;
        int I = 0;
        while ((I + 1) * (I + 2) / 2 <= tl) ++I;
        const int J = tl - I * (I + 1) / 2;
        tile_ptr(tiles, I, J)[r * TP + c] = g[J * 32 + c][I * 32 + r];   // (R^T)(I*32+r, J*32+c)
    }
    __syncthreads();
    invert_tiles<T, NT>(tiles, wt, nt, W);
    for (int idx = tid; idx < W * W; idx += NT) {
        const int i = idx % W, j = idx / W;
        T val = T(0);
        if (i <= j) val = tile_ptr(tiles, j / 32, i / 32)[(j % 32) * TP + (i % 32)];
        sm[i][j] = val;
    }
    __syncthreads();
    if (pass == 0) {
        for (int idx = tid; idx < W * W; idx += NT) {
            const int i = idx % W, j = idx / W;
            sapply[idx] = sm[i][j];
            keep[idx] = g[i][j];
        }
        return;
    }
    for (int idx = tid; idx < W * W; idx += NT) {
        const int i = idx % W, j = idx / W;
        x1[i][j] = keep[idx];
        x2[i][j] = sapply[idx];
    }
    __syncthreads();
    for (int idx = tid; idx < W * W; idx += NT) {
        const int i = idx % W, j = idx / W;
        sapply[idx] = sm[i][j];
        if (i > j || j >= m) continue;
        T r = T(0), s = T(0);
        for (int k = i; k <= j; ++k) {
            r = fma(g[i][k], x1[k][j], r);    // (R2 R1)_ij
            s = fma(x2[i][k], sm[k][j], s);   // (S1 S2)_ij
        }
        rblk[i + j * ldr] = r;
        sblk[i + j * lds] = s;
    }
}

template <typename T>
__global__ void add_block_kernel(T *dst, int64_t ldd, const T *src, int64_t lds, int64_t rows) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = blockIdx.y;
    if (i < rows) dst[i + j * ldd] += src[i + j * lds];
}

size_t esz(tri_dtype dt) { return dt == TRI_F64 ? 8 : 4; }
size_t al(size_t x) { return (x + 255) / 256 * 256; }
int leaf_w(tri_dtype dt) { return dt == TRI_F64 ? 32 : 64; }

int64_t split_point(int64_t m, int w) {
    const int64_t blocks = (m + w - 1) / w;
    return (int64_t)w * ((blocks + 1) / 2);
}

struct QrLayout {
    size_t partials, sapply, keep, tmp, planes, total;
};

QrLayout qr_layout(int64_t n, tri_dtype dt) {
    QrLayout l{};
    const size_t es = esz(dt);
    const int w = leaf_w(dt);
    size_t o = 0;
    l.partials = o;
    o += al((size_t)kMaxPanelCtas * w * w * es);
    l.sapply = o;
    o += al((size_t)w * w * es);
    l.keep = o;
    o += al((size_t)w * w * es);
    l.tmp = o;
    const int64_t h = split_point(n, w);
    o += n > w ? al((size_t)h * (n - h) * es) : 0;
    l.planes = o;
    if (dt == TRI_F32_MIXED && n > w) o += al(gemm_tc_ws_bytes(n, n, n));
    l.total = o;
    return l;
}

struct QrCtx {
    const Ctx *c;
    tri_dtype dt;
    int64_t n;
    uint8_t *a, *r, *s;
    int64_t lda, ldr, lds;
    uint8_t *ws;
    QrLayout lay;
    int np;
    int64_t rows_per;
};

constexpr int64_t kTcMin = 512;

// Tensor cores (mixed) for products that are large and give the grid enough tiles; the
// rest on CUDA cores, with the long-k products split over CTAs.
cudaError_t product(const QrCtx &q, GemmArgs g, const char *name) {
    if (q.dt == TRI_F32_MIXED && g.m >= kTcMin && g.n >= kTcMin && g.k >= kTcMin &&
        ((g.m + 127) / 128) * ((g.n + 255) / 256) >= q.c->sm_count / 2)
        return gemm_tc(*q.c, g, 3, q.ws + q.lay.planes, name);
    g.split_k = true;
    return gemm_simt(*q.c, q.dt == TRI_F64 ? TRI_F64 : TRI_F32, g, name);
}

template <typename T, int W>
cudaError_t leaf_t(const QrCtx &q, int64_t c0, int m) {
    const size_t es = sizeof(T);
    T *p = (T *)(q.a + (size_t)(c0 * q.lda) * es);
    T *partials = (T *)(q.ws + q.lay.partials), *sapply = (T *)(q.ws + q.lay.sapply), *keep = (T *)(q.ws + q.lay.keep);
    T *rblk = (T *)(q.r + (size_t)(c0 + c0 * q.ldr) * es), *sblk = (T *)(q.s + (size_t)(c0 + c0 * q.lds) * es);
    constexpr size_t sm = chol_smem<T, W>();
    cudaError_t e = cudaFuncSetAttribute(qr_chol_kernel<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const cudaStream_t st = q.c->stream;
    TraceScope ts(st, es == 8 ? "sqr_leaf_f64" : "sqr_leaf_f32", 8.0 * (double)q.n * m * m, 0.0);
    qr_panel_kernel<T, W><<<q.np, kPanelThreads, 0, st>>>(p, q.lda, q.n, m, nullptr, partials, q.rows_per);
    qr_chol_kernel<T, W><<<1, kPanelThreads, sm, st>>>(partials, q.np, m, 0, sapply, keep, rblk, q.ldr, sblk, q.lds,
                                                       q.c->info, c0);
    qr_panel_kernel<T, W><<<q.np, kPanelThreads, 0, st>>>(p, q.lda, q.n, m, sapply, partials, q.rows_per);
    qr_chol_kernel<T, W><<<1, kPanelThreads, sm, st>>>(partials, q.np, m, 1, sapply, keep, rblk, q.ldr, sblk, q.lds,
                                                       q.c->info, c0);
    qr_panel_kernel<T, W><<<q.np, kPanelThreads, 0, st>>>(p, q.lda, q.n, m, sapply, nullptr, q.rows_per);
    return cudaGetLastError();
}

cudaError_t leaf(const QrCtx &q, int64_t c0, int m) {
    return q.dt == TRI_F64 ? leaf_t<double, 32>(q, c0, m) : leaf_t<float, 64>(q, c0, m);
}

cudaError_t rec(const QrCtx &q, int64_t c0, int64_t m) {
    const int w = leaf_w(q.dt);
    if (m <= w) return leaf(q, c0, (int)m);
    const size_t es = esz(q.dt);
    const int64_t m1 = split_point(m, w), m2 = m - m1;
    cudaError_t e = rec(q, c0, m1);
    if (e != cudaSuccess) return e;
    auto A = [&](int64_t j) { return (void *)(q.a + (size_t)(j * q.lda) * es); };
    auto R = [&](int64_t i, int64_t j) { return (void *)(q.r + (size_t)(i + j * q.ldr) * es); };
    auto S = [&](int64_t i, int64_t j) { return (void *)(q.s + (size_t)(i + j * q.lds) * es); };
    void *tmp = q.ws + q.lay.tmp;
    const int64_t n = q.n;
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
        // C = Q1^T A2 (R12 on the first pass, its correction on the second)
        void *C = pass == 0 ? R(c0, c0 + m1) : tmp;
        const int64_t ldc = pass == 0 ? q.ldr : m1;
        GemmArgs g1{m1, m2, n, 1.0, A(c0), q.lda, OP_FULL, A(c0 + m1), q.lda, OP_FULL, 0.0, C, ldc, OP_FULL};
        g1.ta = true;
        e = product(q, g1, "sqr:qta");
        // A2 <- A2 - Q1 C
        if (e == cudaSuccess)
            e = product(q, GemmArgs{n, m2, m1, -1.0, A(c0), q.lda, OP_FULL, C, ldc, OP_FULL, 1.0, A(c0 + m1), q.lda,
                                    OP_FULL}, "sqr:update");
    }
    if (e != cudaSuccess) return e;
    if (m2 > 65535) return cudaErrorInvalidValue;
    {
        dim3 grid((unsigned)((m1 + 255) / 256), (unsigned)m2);
        if (q.dt == TRI_F64)
            add_block_kernel<double><<<grid, 256, 0, q.c->stream>>>((double *)R(c0, c0 + m1), q.ldr,
                                                                   (const double *)tmp, m1, m1);
        else
            add_block_kernel<float><<<grid, 256, 0, q.c->stream>>>((float *)R(c0, c0 + m1), q.ldr,
                                                                  (const float *)tmp, m1, m1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    e = rec(q, c0 + m1, m2);
    if (e != cudaSuccess) return e;
    // S12 = -(S11 R12) S22
    e = product(q, GemmArgs{m1, m2, m1, 1.0, S(c0, c0), q.lds, OP_UPPER, R(c0, c0 + m1), q.ldr, OP_FULL, 0.0, tmp, m1,
                            OP_FULL}, "sqr:s12a");
    if (e != cudaSuccess) return e;
    return product(q, GemmArgs{m1, m2, m2, -1.0, tmp, m1, OP_FULL, S(c0 + m1, c0 + m1), q.lds, OP_UPPER, 0.0,
                               S(c0, c0 + m1), q.lds, OP_FULL}, "sqr:s12b");
}

QrCtx make_ctx(const Ctx &c, tri_dtype dt, int64_t n, void *a, int64_t lda, void *r, int64_t ldr, void *s,
               int64_t lds, void *ws) {
    QrCtx q{&c, dt, n, (uint8_t *)a, (uint8_t *)r, (uint8_t *)s, lda, ldr, lds, (uint8_t *)ws, qr_layout(n, dt), 1, 0};
    int64_t np = std::min<int64_t>(kMaxPanelCtas, (n + kChunk - 1) / kChunk);
    int64_t per = (n + np - 1) / np;
    per = (per + kChunk - 1) / kChunk * kChunk;
    q.np = (int)((n + per - 1) / per);
    q.rows_per = per;
    return q;
}

}  // namespace

size_t sqr_ws_bytes(int64_t n, tri_dtype dt) {
    if (n <= 0) return 0;
    return qr_layout(n, dt).total;
}

// A <- Q, r <- R, s <- S = R^-1 (strict lower parts of r and s set to zero).
tri_status run_sqr(const Ctx &c, tri_dtype dt, int64_t n, void *a, int64_t lda, void *r, int64_t ldr, void *s,
                   int64_t lds, void *ws) {
    const size_t es = esz(dt);
    if (cudaMemset2DAsync(r, ldr * es, 0, n * es, n, c.stream) != cudaSuccess ||
        cudaMemset2DAsync(s, lds * es, 0, n * es, n, c.stream) != cudaSuccess)
        return TRI_ERR_CUDA;
    QrCtx q = make_ctx(c, dt, n, a, lda, r, ldr, s, lds, ws);
    return rec(q, 0, n) == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
}

// Scratch of sqr_inv: R and S (n x n each) and the scratch of run_sqr.
size_t sqr_inv_ws_bytes(int64_t n, tri_dtype dt) {
    if (n <= 0) return 0;
    return 2 * al((size_t)n * n * esz(dt)) + sqr_ws_bytes(n, dt);
}

// A <- A^-1 = S Q^T.
tri_status run_sqr_inv(const Ctx &c, tri_dtype dt, int64_t n, void *a, int64_t lda, void *ws) {
    const size_t es = esz(dt), mat = al((size_t)n * n * es);
    uint8_t *r = (uint8_t *)ws, *s = r + mat, *rest = s + mat;
    tri_status st = run_sqr(c, dt, n, a, lda, r, n, s, n, rest);
    if (st != TRI_OK) return st;
    QrCtx q = make_ctx(c, dt, n, a, lda, r, n, s, n, rest);
    GemmArgs g{n, n, n, 1.0, s, n, OP_UPPER, a, lda, OP_FULL, 0.0, r, n, OP_FULL};
    g.tb = true;
    cudaError_t e = product(q, g, "sqr:sqt");
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(a, lda * es, r, n * es, n * es, n, cudaMemcpyDeviceToDevice, c.stream);
    return e == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
}

}  // namespace triinv
