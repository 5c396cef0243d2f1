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
constexpr int kMaxPanelCtas = 128;

// 16-byte shared-memory vector load / store of 16 / sizeof(T) elements.
template <typename T>
__device__ __forceinline__ void ld16(T (&v)[16 / sizeof(T)], const T *p) {
    *reinterpret_cast<uint4 *>(v) = *reinterpret_cast<const uint4 *>(p);
}
template <typename T>
__device__ __forceinline__ void st16(T *p, const T (&v)[16 / sizeof(T)]) {
    *reinterpret_cast<uint4 *>(p) = *reinterpret_cast<const uint4 *>(v);
}

// One pass over the rows of a leaf panel P (rows x m, m <= W), CTA b taking rows
// [b * rows_per, (b + 1) * rows_per) in chunks of kChunk rows, staged transposed
// (s_pt[c][r] = P(r0 + r, c), a column per shared-memory row):
//   sapply != null: P <- P S  (S upper, W x W, leading dimension W)
//   gram != null:   G += P^T P of the (updated) rows, upper triangle, atomically
//                   (G is W x W, zero on entry to the first pass of a leaf)
template <typename T, int W>
__global__ void __launch_bounds__(kPanelThreads) qr_panel_kernel(T *p, int64_t ldp, int64_t rows, int m,
                                                                 const T *__restrict__ sapply, T *gram,
                                                                 int64_t rows_per) {
    constexpr int NT = kPanelThreads, CH = kChunk;
    constexpr int V = 16 / sizeof(T);    // elements per 16-byte vector
    constexpr int PT = CH + V;           // row pitch: an odd number of 16-byte vectors
    constexpr int PS = W + V;
    constexpr int CB = W / 16;           // columns per thread
    constexpr int RB = CH / 16;          // rows per thread (apply)
    static_assert((PT / V) % 2 == 1 && CB % V == 0 && RB % V == 0, "panel layout");
    __shared__ __align__(16) T s_s[W][PS];
    __shared__ __align__(16) T s_pt[W][PT];
    const int tid = threadIdx.x;
    static_assert((W * W) % NT == 0 && (CH * W) % NT == 0, "panel loops");
    if (sapply) {
#pragma unroll
        for (int it = 0; it < W * W / NT; ++it) {
            const int idx = tid + it * NT, k = idx % W, j = idx / W;
            s_s[k][j] = (k <= j && j < m) ? sapply[k + j * W] : T(0);
        }
    }
    const int ti = tid % 16, tj = tid / 16;   // Gram entries (ti + 16 ii, tj + 16 jj)
    const int tr = tid % 16, tc = tid / 16;   // apply outputs rows tr*RB.., columns tc*CB..
    T g[CB][CB];
#pragma unroll
    for (int a = 0; a < CB; ++a)
#pragma unroll
        for (int b = 0; b < CB; ++b) g[a][b] = T(0);
    const int64_t r_begin = (int64_t)blockIdx.x * rows_per;
    const int64_t r_end = min(rows, r_begin + rows_per);
    for (int64_t r0 = r_begin; r0 < r_end; r0 += CH) {
#pragma unroll
        for (int it = 0; it < CH * W / NT; ++it) {
            const int idx = tid + it * NT, r = idx % CH, c = idx / CH;
            const int64_t gr = r0 + r;
            s_pt[c][r] = (gr < r_end && c < m) ? p[gr + (int64_t)c * ldp] : T(0);
        }
        __syncthreads();
        if (sapply) {
            T acc[RB][CB];
#pragma unroll
            for (int a = 0; a < RB; ++a)
#pragma unroll
                for (int b = 0; b < CB; ++b) acc[a][b] = T(0);
#pragma unroll 4
            for (int k = 0; k < W; ++k) {
                T av[RB], bv[CB];
#pragma unroll
                for (int u = 0; u < RB / V; ++u) ld16<T>(*reinterpret_cast<T (*)[V]>(av + u * V), &s_pt[k][tr * RB + u * V]);
#pragma unroll
                for (int u = 0; u < CB / V; ++u) ld16<T>(*reinterpret_cast<T (*)[V]>(bv + u * V), &s_s[k][tc * CB + u * V]);
#pragma unroll
                for (int a = 0; a < RB; ++a)
#pragma unroll
                    for (int b = 0; b < CB; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
            }
            __syncthreads();
#pragma unroll
            for (int b = 0; b < CB; ++b)
#pragma unroll
                for (int u = 0; u < RB / V; ++u) {
                    T w[V];
#pragma unroll
                    for (int x = 0; x < V; ++x) w[x] = acc[u * V + x][b];
                    st16<T>(&s_pt[tc * CB + b][tr * RB + u * V], w);
                }
            __syncthreads();
#pragma unroll
            for (int it = 0; it < CH * W / NT; ++it) {
                const int idx = tid + it * NT, r = idx % CH, c = idx / CH;
                const int64_t gr = r0 + r;
                if (gr < r_end && c < m) p[gr + (int64_t)c * ldp] = s_pt[c][r];
            }
        }
        if (gram) {
#pragma unroll 2
            for (int r = 0; r < CH; r += V) {
                T av[CB][V], bv[CB][V];
#pragma unroll
                for (int a = 0; a < CB; ++a) ld16<T>(av[a], &s_pt[ti + 16 * a][r]);
#pragma unroll
                for (int b = 0; b < CB; ++b) ld16<T>(bv[b], &s_pt[tj + 16 * b][r]);
#pragma unroll
                for (int a = 0; a < CB; ++a)
#pragma unroll
                    for (int b = 0; b < CB; ++b)
#pragma unroll
                        for (int x = 0; x < V; ++x) g[a][b] = fma(av[a][x], bv[b][x], g[a][b]);
            }
        }
        __syncthreads();
    }
    if (gram)
#pragma unroll
        for (int a = 0; a < CB; ++a)
#pragma unroll
            for (int b = 0; b < CB; ++b) {
                const int i = ti + 16 * a, j = tj + 16 * b;
                if (i <= j && j < m) atomicAdd(gram + i + j * W, g[a][b]);
            }
}

template <typename T, int W>
constexpr size_t chol_smem() {
    constexpr int nt = W / 32;
    constexpr int tiles = nt * (nt + 1) / 2;
    constexpr int wtiles = (nt / 2) * (nt / 2) > 0 ? (nt / 2) * (nt / 2) : 1;
    return sizeof(T) * (4 * (size_t)W * (W + 1) + 5 * W + 2 + (size_t)(tiles + wtiles) * TE);
}

// The Cholesky step of one Cholesky QR pass, one CTA:
//   G = the accumulated Gram matrix (m x m, identity beyond m; its buffer is cleared),
//   G = R^T R (R upper, positive diagonal), S = R^-1.
// pass 0: S -> sapply, R -> keep.
// pass 1: with S1 = sapply and R1 = keep from pass 0: S2 -> sapply, R2 R1 -> rblk and
//         S1 S2 -> sblk (their m x m upper triangles).
template <typename T, int W>
__global__ void __launch_bounds__(kPanelThreads) qr_chol_kernel(T *gram, int m, int pass, T *sapply, T *keep,
                                                                T *rblk, int64_t ldr, T *sblk, int64_t lds,
                                                                long long *info, int64_t col0) {
    constexpr int NT = kPanelThreads;
    constexpr int EQ = W * W / NT;       // entries per thread
    constexpr int nt = W / 32;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    T (*g)[W + 1] = reinterpret_cast<T (*)[W + 1]>(smem_raw);        // G, then R
    T (*sm)[W + 1] = g + W;                                          // S
    T (*x1)[W + 1] = g + 2 * W;                                      // R1 (pass 1)
    T (*x2)[W + 1] = g + 3 * W;                                      // S1 (pass 1)
    T *rowk = reinterpret_cast<T *>(g + 4 * W);                      // 2 x 2W: row k, padded
    T *rsb = rowk + 4 * W;                                           // 2: 1 / sqrt(G_kk)
    T *pvt = rsb + 2;                                                // W: the pivots G_kk
    T *tiles = pvt + W;
    T *wt = tiles + (size_t)(nt * (nt + 1) / 2) * TE;
    const int tid = threadIdx.x;

    // Cholesky, right-looking, one barrier per step.  Thread (ci, cg) = (tid % W, tid / W)
    // holds the entries (ci, ci + cg + G q) of the upper triangle (G = NT / W; columns
    // beyond W are padding), so its diagonal entry, when cg = 0, is always v[0].  Step k:
    // the threads of row k publish it (unscaled) and its pivot's 1/sqrt, computed at the end
    // of the previous step; one barrier; the rows below update, row k scales.  The Gram
    // matrix is read and its buffer cleared for the next pass; pivots are checked after.
    constexpr int G = NT / W;
    const int ci = tid % W, cg = tid / W;
    for (int x = tid; x < W * (W + 1); x += NT) (&g[0][0])[x] = T(0);
    for (int x = tid; x < 4 * W; x += NT) rowk[x] = T(0);     // the padding columns stay zero
    T v[EQ];
#pragma unroll
    for (int q = 0; q < EQ; ++q) {
        const int j = ci + cg + G * q;
        T val = T(0);
        if (j < m) {
            val = gram[ci + j * W];
            gram[ci + j * W] = T(0);
        } else if (j < W && j == ci) {
            val = T(1);
        }
        v[q] = val;
    }
    T rs_next = T(1) / sqrt(v[0]);            // 1/sqrt(pivot) for the thread holding (0, 0)
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        T *rk = rowk + (k & 1) * 2 * W;
        if (ci == k) {
#pragma unroll
            for (int q = 0; q < EQ; ++q) {
                const int j = ci + cg + G * q;
                if (j < W) rk[j] = v[q];
            }
            if (cg == 0) {
                pvt[k] = v[0];
                rsb[k & 1] = rs_next;
            }
        }
        __syncthreads();
        const T rs = rsb[k & 1];              // R_kj = G_kj / sqrt(G_kk)
        if (ci > k) {
            const T li = rk[ci] * rs;         // R_k,ci
#pragma unroll
            for (int q = 0; q < EQ; ++q) v[q] = fma(-li, rk[ci + cg + G * q] * rs, v[q]);
            if (cg == 0 && ci == k + 1) rs_next = T(1) / sqrt(v[0]);   // the next pivot's owner
        } else if (ci == k) {
#pragma unroll
            for (int q = 0; q < EQ; ++q) v[q] *= rs;
        }
    }
    if (tid < m && !(pvt[tid] > T(0) && isfinite(pvt[tid]))) atomicMin(info, (long long)(col0 + tid));
    __syncthreads();
#pragma unroll
    for (int q = 0; q < EQ; ++q) {
        const int j = ci + cg + G * q;
        if (j < W) g[ci][j] = v[q];
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
    // (R2 R1)_ij and (S1 S2)_ij over all k: the triangles' stored zeros drop the terms
    // outside i <= k <= j, so every lane runs the same loop.  Entries (i0, j0 + G q).
    const int i0 = tid % W, j0 = tid / W;
    T racc[EQ], sacc[EQ];
#pragma unroll
    for (int q = 0; q < EQ; ++q) racc[q] = sacc[q] = T(0);
#pragma unroll 4
    for (int k = 0; k < W; ++k) {
        const T a = g[i0][k], b = x2[i0][k];
#pragma unroll
        for (int q = 0; q < EQ; ++q) {
            const int j = j0 + G * q;
            racc[q] = fma(a, x1[k][j], racc[q]);
            sacc[q] = fma(b, sm[k][j], sacc[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < EQ; ++q) {
        const int j = j0 + G * q;
        sapply[i0 + j * W] = sm[i0][j];
        if (i0 <= j && j < m) {
            rblk[i0 + j * ldr] = racc[q];
            sblk[i0 + j * lds] = sacc[q];
        }
    }
}

// C = alpha * sum_b P_b (+ beta C): the slices of a split-k product, summed in order.
__global__ void sum_slices_kernel(float *c, int64_t ldc, const float *__restrict__ parts, int64_t m, int64_t n,
                                  int slices, float alpha, float beta) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = blockIdx.y;
    if (i >= m) return;
    const float *pp = parts + i + j * m;
    float acc = 0.f;
    for (int b = 0; b < slices; ++b) acc += pp[(size_t)b * m * n];
    float *pc = c + i + j * ldc;
    *pc = beta == 0.f ? alpha * acc : fmaf(alpha, acc, beta * *pc);
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
    size_t gram, sapply, keep, tmp, parts, planes, total;
};

// Split-k tensor-core products (mixed): slices s with s * tiles <= 2 * kMaxSm, so the
// partial outputs hold at most 2 * kMaxSm tensor-core tiles of 128 x 256.
constexpr int64_t kMaxSm = 160;
constexpr size_t kPartsElems = (size_t)2 * kMaxSm * 128 * 256;

QrLayout qr_layout(int64_t n, tri_dtype dt) {
    QrLayout l{};
    const size_t es = esz(dt);
    const int w = leaf_w(dt);
    size_t o = 0;
    l.gram = o;
    o += al((size_t)w * w * es);
    l.sapply = o;
    o += al((size_t)w * w * es);
    l.keep = o;
    o += al((size_t)w * w * es);
    l.tmp = o;
    const int64_t h = split_point(n, w);
    o += n > w ? al((size_t)h * (n - h) * es) : 0;
    l.parts = o;
    if (dt == TRI_F32_MIXED && n > w) o += al(kPartsElems * 4);
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

// Tensor cores (mixed) for the products with at least 128 rows and columns and k >= 128
// that fill the grid: directly when they have enough 128 x 256 output tiles, else (long
// k) as `s` k-slices run as one batched product into separate partial outputs, summed in
// a fixed order afterwards.  The rest on CUDA cores, with long-k products split over CTAs.
cudaError_t product(const QrCtx &q, GemmArgs g, const char *name) {
    if (q.dt == TRI_F32_MIXED && g.m >= 128 && g.n >= 128 && g.k >= 128 && g.batch == 1) {
        const int64_t tiles = ((g.m + 127) / 128) * ((g.n + 255) / 256);
        const int64_t sm = std::min<int64_t>(q.c->sm_count, kMaxSm);
        if (tiles >= sm / 2 && g.m * g.n * g.k >= (int64_t)1 << 27)
            return gemm_tc(*q.c, g, 3, q.ws + q.lay.planes, name);
        int64_t sl = 1;
        while (sl * 2 * tiles <= 2 * sm && g.k % (sl * 2) == 0 && g.k / (sl * 2) >= 1024) sl *= 2;
        if (sl > 1 && g.akind == OP_FULL && g.bkind == OP_FULL && g.cmask == OP_FULL &&
            (size_t)(sl * g.m * g.n) <= kPartsElems) {
            const int64_t ks = g.k / sl;
            float *parts = (float *)(q.ws + q.lay.parts);
            GemmArgs gb = g;
            gb.k = ks;
            gb.batch = sl;
            gb.sa = g.ta ? ks : ks * g.lda;    // slice b of op(A) = columns [b ks, (b+1) ks) of op(A)
            gb.sb = g.tb ? ks * g.ldb : ks;    // and rows [b ks, (b+1) ks) of op(B)
            gb.alpha = 1.0;
            gb.beta = 0.0;
            gb.c = parts;
            gb.ldc = g.m;
            gb.sc = g.m * g.n;
            cudaError_t e = gemm_tc(*q.c, gb, 3, q.ws + q.lay.planes, name);
            if (e != cudaSuccess) return e;
            if (g.n > 65535) return cudaErrorInvalidValue;
            dim3 grid((unsigned)((g.m + 255) / 256), (unsigned)g.n);
            sum_slices_kernel<<<grid, 256, 0, q.c->stream>>>((float *)g.c, g.ldc, parts, g.m, g.n, (int)sl,
                                                             (float)g.alpha, (float)g.beta);
            return cudaGetLastError();
        }
        if (g.m >= 512 && g.k <= 1024 && tiles >= sm / 2)   // tall, short-k products
            return gemm_tc(*q.c, g, 3, q.ws + q.lay.planes, name);
    }
    g.split_k = true;
    return gemm_simt(*q.c, q.dt == TRI_F64 ? TRI_F64 : TRI_F32, g, name);
}

template <typename T, int W>
cudaError_t leaf_t(const QrCtx &q, int64_t c0, int m) {
    const size_t es = sizeof(T);
    T *p = (T *)(q.a + (size_t)(c0 * q.lda) * es);
    T *gram = (T *)(q.ws + q.lay.gram), *sapply = (T *)(q.ws + q.lay.sapply), *keep = (T *)(q.ws + q.lay.keep);
    T *rblk = (T *)(q.r + (size_t)(c0 + c0 * q.ldr) * es), *sblk = (T *)(q.s + (size_t)(c0 + c0 * q.lds) * es);
    constexpr size_t sm = chol_smem<T, W>();
    cudaError_t e = cudaFuncSetAttribute(qr_chol_kernel<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const cudaStream_t st = q.c->stream;
    TraceScope ts(st, es == 8 ? "sqr_leaf_f64" : "sqr_leaf_f32", 8.0 * (double)q.n * m * m, 0.0);
    qr_panel_kernel<T, W><<<q.np, kPanelThreads, 0, st>>>(p, q.lda, q.n, m, nullptr, gram, q.rows_per);
    qr_chol_kernel<T, W><<<1, kPanelThreads, sm, st>>>(gram, m, 0, sapply, keep, rblk, q.ldr, sblk, q.lds,
                                                       q.c->info, c0);
    qr_panel_kernel<T, W><<<q.np, kPanelThreads, 0, st>>>(p, q.lda, q.n, m, sapply, gram, q.rows_per);
    qr_chol_kernel<T, W><<<1, kPanelThreads, sm, st>>>(gram, m, 1, sapply, keep, rblk, q.ldr, sblk, q.lds,
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
    QrCtx q = make_ctx(c, dt, n, a, lda, r, ldr, s, lds, ws);
    if (cudaMemset2DAsync(r, ldr * es, 0, n * es, n, c.stream) != cudaSuccess ||
        cudaMemset2DAsync(s, lds * es, 0, n * es, n, c.stream) != cudaSuccess ||
        cudaMemsetAsync(q.ws + q.lay.gram, 0, (size_t)leaf_w(dt) * leaf_w(dt) * es, c.stream) != cudaSuccess)
        return TRI_ERR_CUDA;
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
