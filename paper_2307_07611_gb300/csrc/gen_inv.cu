// gen_inv.cu -- a5: general inverse A^-1 = U^-1 L^-1 from an unpivoted block LU.
//
// The factorisation and the inverse factors are built together, block-recursively, in
// the spirit of SKUL (Section 5.1: "S K = A^-1", the inverse factors S = U^-1 and
// K = L^-1 formed alongside L and U) and of the 2-block split of BRSI (Section 5.2, the
// Schur-complement form).  For A = [A11 A12; A21 A22] (Doolittle: L unit lower):
//     (K11, S11) = rec(A11)
//     U12 = K11 A12,   L21 = A21 S11,   A22 <- A22 - L21 U12     (Schur complement)
//     (K22, S22) = rec(A22)
//     K21 = -K22 (L21 K11),   S12 = -(S11 U12) S22               (block inverses, Section 3)
// and finally A^-1 = S K (upper times unit lower).  Leaves (128 x 128 in FP32, 64 x 64 in
// FP64) are factored by one CTA in shared memory, and their L and U are inverted there by
// the tiled split of tile_inverse.cuh.  Flops: LU 2n^3/3, inverse
// factors 2n^3/3, product 2n^3/3.
//
// K (strict lower, unit diagonal implied) and S (upper with diagonal) share one n x n
// workspace buffer.  No pivoting: a zero or non-finite pivot is recorded and reported by
// tri_get_info.
#include <algorithm>
#include <climits>
#include <vector>

#include "gemm.cuh"
#include "tile_inverse.cuh"

namespace triinv {
namespace {

// One leaf block [off, off + nb) of A (nb <= L): unpivoted Doolittle LU, then K = L^-1
// (strict lower part of ks) and S = U^-1 (upper part of ks, with diagonal).
//
// LU: the block sits in registers, warp w owning the BR x BC sub-block (w % WR, w / WR) of
// it and lane (lr, lc) = (lane % 4, lane / 4) RPL rows x CPL columns of that.  Step k:
// the owners of row k publish u_kj (j > k), the owners of column k publish a_ik (i > k)
// and the owner of the pivot publishes 1/u_kk (buffers double-buffered by the parity of
// k; the pivots are checked after the loop); one barrier; then every warp whose sub-block
// has rows below k and columns from k on
// sets l_ik = a_ik / u_kk and a_ij -= l_ik u_kj, the multipliers masked to zero outside the
// trailing block so that every entry takes the same FMA; finished sub-blocks skip the step.
// Column k of L is final at step k and goes straight to shared memory.
// The inverses: L (unit diagonal) and U^T are copied into two sets of 32 x 32 tiles and
// inverted together by the tiled split of tile_inverse.cuh.
// lu_out (may be null, else the same matrix as a): the packed Doolittle factors of the
// block are written back over it (L strictly below the diagonal, U on and above it).
template <typename T, int L, int NT>
__global__ void __launch_bounds__(NT) lu_leaf_kernel(const T *a, int64_t lda, T *__restrict__ ks, int64_t ldk,
                                                     int64_t off, int nb, long long *info, T *lu_out,
                                                     long long info_base) {
    constexpr int NW = NT / 32;
    constexpr int WC = 4, WR = NW / WC;          // grid of warp sub-blocks
    constexpr int BR = L / WR, BC = L / WC;      // sub-block of a warp
    constexpr int RPL = BR / 4, CPL = BC / 8;    // rows / columns of a lane
    static_assert(WR * WC == NW && RPL * 4 == BR && CPL * 8 == BC, "LU register layout");
    constexpr int NTL = L / 32;                  // tile rows
    constexpr int KT = NTL * (NTL + 1) / 2;      // lower tiles
    constexpr int WT = (NTL / 2) * (NTL / 2) > 0 ? (NTL / 2) * (NTL / 2) : 1;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    T (*s)[L + 1] = reinterpret_cast<T (*)[L + 1]>(smem_raw);
    T *tl_ = reinterpret_cast<T *>(smem_raw + sizeof(T) * L * (L + 1));
    T *tu_ = tl_ + (size_t)KT * TE;
    T *wl_ = tu_ + (size_t)KT * TE;
    T *wu_ = wl_ + (size_t)WT * TE;
    T *rkb = wu_ + (size_t)WT * TE;              // 2 x L: row k
    T *ckb = rkb + 2 * L;                        // 2 x L: column k
    T *rpb = ckb + 2 * L;                        // 2: 1 / u_kk
    T *pv = rpb + 2;                             // L: the pivots u_kk
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = NW;
    for (int idx = tid; idx < L * L; idx += NT) {
        const int i = idx % L, j = idx / L;
        T v = (i == j) ? T(1) : T(0);
        if (i < nb && j < nb) v = a[(off + i) + (off + j) * lda];
        s[i][j] = v;
    }
    __syncthreads();
    {
        const int wr = warp % WR, wc = warp / WR, lr = lane % 4, lc = lane / 4;
        const int i0 = wr * BR + lr * RPL, j0 = wc * BC + lc * CPL;
        T v[RPL][CPL];
#pragma unroll
        for (int r = 0; r < RPL; ++r)
#pragma unroll
            for (int c = 0; c < CPL; ++c) v[r][c] = s[i0 + r][j0 + c];
        // k = kb + kr with the inner step unrolled, so that row kr of a lane's block and
        // its column kr % CPL are compile-time register indices (kb is a multiple of RPL,
        // which CPL divides).
        static_assert(RPL % CPL == 0, "step unrolling");
        // 1 / (this lane's candidate for the next pivot): computed at the end of the previous
        // step's update, where it overlaps the remaining FMAs; only the pivot's owner stores it
        T rcp_next = T(1) / v[0][0];
        for (int kb = 0; kb < nb; kb += RPL) {
#pragma unroll
            for (int kr = 0; kr < RPL; ++kr) {
                const int k = kb + kr;
                if (k >= nb) break;
                T *rk = rkb + (k & 1) * L, *ck = ckb + (k & 1) * L;
                const bool own_col = j0 == kb + (kr / CPL) * CPL;
                if (i0 == kb) {            // this lane holds row k: u_kj (j >= k)
#pragma unroll
                    for (int c = 0; c < CPL; ++c) {
                        const T val = v[kr][c];
                        if (j0 + c > k) rk[j0 + c] = val;
                        if (j0 + c == k) {
                            pv[k] = val;
                            rpb[k & 1] = rcp_next;
                        }
                    }
                }
                if (own_col)               // this lane holds column k: a_ik (i > k)
#pragma unroll
                    for (int r = 0; r < RPL; ++r)
                        if (i0 + r > k) ck[i0 + r] = v[r][kr % CPL];
                __syncthreads();
                if ((wr + 1) * BR - 1 > k && (wc + 1) * BC - 1 >= k) {
                    // multipliers masked to the trailing block: rows i > k, columns j > k
                    const T rp = rpb[k & 1];
                    T li[RPL], uj[CPL];
#pragma unroll
                    for (int r = 0; r < RPL; ++r) {
                        const T l = ck[i0 + r] * rp;
                        li[r] = (i0 + r > k) ? l : T(0);
                    }
#pragma unroll
                    for (int c = 0; c < CPL; ++c) uj[c] = (j0 + c > k) ? rk[j0 + c] : T(0);
                    if (own_col)           // column k of L is final: straight to shared memory
#pragma unroll
                        for (int r = 0; r < RPL; ++r)
                            if (i0 + r > k) s[i0 + r][k] = li[r];
#pragma unroll
                    for (int r = 0; r < RPL; ++r)
#pragma unroll
                        for (int c = 0; c < CPL; ++c) v[r][c] = fma(-li[r], uj[c], v[r][c]);
                    rcp_next = T(1) / v[(kr + 1) % RPL][(kr + 1) % CPL];
                }
            }
        }
        // U (on and above the diagonal) from the registers; L is already in place
#pragma unroll
        for (int r = 0; r < RPL; ++r)
#pragma unroll
            for (int c = 0; c < CPL; ++c)
                if (j0 + c >= i0 + r) s[i0 + r][j0 + c] = v[r][c];
        __syncthreads();
    }
    for (int k = tid; k < nb; k += NT)
        if (pv[k] == T(0) || !isfinite(pv[k])) atomicMin(info, info_base + (long long)(off + k));
    if (lu_out)
        for (int idx = tid; idx < nb * nb; idx += NT) {
            const int i = idx % nb, j = idx / nb;
            lu_out[(off + i) + (off + j) * lda] = s[i][j];
        }
    const int nt = (nb + 31) / 32;
    const int ntiles = nt * (nt + 1) / 2;
    // tiles of the lower view: set 0 = L (unit diagonal), set 1 = U^T
    for (int x = warp; x < 2 * ntiles; x += nwarps) {
        const int set = x / ntiles, tl = x % ntiles;
        int I = 0;
        while ((I + 1) * (I + 2) / 2 <= tl) ++I;
        const int J = tl - I * (I + 1) / 2;
        T *tp = tile_ptr(set == 0 ? tl_ : tu_, I, J);
        for (int c = 0; c < 32; ++c) {
            const int i = I * 32 + lane, j = J * 32 + c;
            T v;
            if (i >= nb || j >= nb) v = (i == j) ? T(1) : T(0);
            else if (j > i) v = T(0);
            else if (j == i) v = set == 0 ? T(1) : s[i][i];
            else v = set == 0 ? s[i][j] : s[j][i];
            tp[lane * TP + c] = v;
        }
    }
    __syncthreads();
    {
        T *const tls[2] = {tl_, tu_};
        T *const wts[2] = {wl_, wu_};
        invert_tiles_multi<T, NT, 2>(tls, wts, nt, nb);
    }
    for (int x = warp; x < 2 * ntiles; x += nwarps) {
        const int set = x / ntiles, tl = x % ntiles;
        int I = 0;
        while ((I + 1) * (I + 2) / 2 <= tl) ++I;
        const int J = tl - I * (I + 1) / 2;
        const T *tp = tile_ptr(set == 0 ? tl_ : tu_, I, J);
        for (int c = 0; c < 32; ++c) {
            const int i = I * 32 + lane, j = J * 32 + c;
            if (i >= nb || j >= nb || j > i) continue;
            if (set == 0) {
                if (j < i) ks[(off + i) + (off + j) * ldk] = tp[lane * TP + c];   // K, strict lower
            } else {
                ks[(off + j) + (off + i) * ldk] = tp[lane * TP + c];              // S = (U^T)^-1 ^T
            }
        }
    }
}

template <typename T, int L>
constexpr size_t lu_leaf_smem() {
    constexpr int NTL = L / 32;
    constexpr int KT = NTL * (NTL + 1) / 2;
    constexpr int WT = (NTL / 2) * (NTL / 2) > 0 ? (NTL / 2) * (NTL / 2) : 1;
    return sizeof(T) * ((size_t)L * (L + 1) + 2 * (size_t)(KT + WT) * TE + 5 * L + 2);
}

struct Node {
    int64_t off, m1, m2;
};

int leaf_size(tri_dtype dt) { return dt == TRI_F64 ? 64 : 128; }
size_t esz(tri_dtype dt) { return dt == TRI_F64 ? 8 : 4; }

int64_t split_point(int64_t m, int L) {
    const int64_t blocks = (m + L - 1) / L;
    return (int64_t)L * ((blocks + 1) / 2);
}

// Temp sizes per recursion depth (elements): three buffers of m1 * m2 each.
void depth_sizes(int64_t n, int L, std::vector<int64_t> &sz) {
    sz.clear();
    std::vector<int64_t> level{n};
    while (true) {
        int64_t best = 0;
        std::vector<int64_t> next;
        for (int64_t m : level) {
            if (m <= L) continue;
            const int64_t m1 = split_point(m, L), m2 = m - m1;
            best = std::max(best, m1 * m2);
            next.push_back(m1);
            next.push_back(m2);
        }
        if (next.empty()) break;
        sz.push_back(best);
        level.swap(next);
    }
}

size_t al(size_t x) { return (x + 255) / 256 * 256; }

struct GenLayout {
    size_t ks, temps, planes, a0, total;
    std::vector<size_t> depth_off;
};

constexpr int64_t kTcMin = 512;   // smaller products stay on CUDA cores

// with_ks: the K\S buffer lives in the scratch (gen_inv); SKUL writes it to the caller's.
GenLayout gen_layout(int64_t n, tri_dtype dt, bool with_ks = true) {
    GenLayout g{};
    const int L = leaf_size(dt);
    std::vector<int64_t> sz;
    depth_sizes(n, L, sz);
    g.ks = with_ks ? al((size_t)n * n * esz(dt)) : 0;
    size_t o = g.ks;
    for (int64_t s : sz) {
        g.depth_off.push_back(o);
        o += 3 * al((size_t)s * esz(dt));
    }
    g.temps = o - g.ks;
    g.planes = 0;
    g.a0 = 0;
    if (dt == TRI_F32_MIXED) {
        g.planes = al(gemm_tc_ws_bytes(n, n, n));
        // gen_inv's Newton-Schulz step needs the original A (FP32, leading dimension n)
        if (with_ks && n >= kTcMin) g.a0 = al((size_t)n * n * 4);
    }
    g.total = o + g.planes + g.a0;
    return g;
}

struct GenCtx {
    const Ctx *c;
    tri_dtype dt;
    uint8_t *ws;
    GenLayout lay;
    int L;
    bool keep = false;   // write L21, U12 and the leaf factors back over A (SKUL)
    long long info_base = 0;   // added to the reported pivot index (a block of a larger matrix)
};

// Mixed products: three terms (about 2^-16 relative) in gen_inv, whose Newton-Schulz step
// then restores FP32 accuracy against A; six promoted terms (about 2^-24) in SKUL, whose
// factors are the result and get no refinement, and in gen_inv under the direct recipe
// (tri_set_mixed_recipe), which then skips the Newton-Schulz step.
cudaError_t product(const GenCtx &g, const GemmArgs &a, const char *name) {
    if (g.dt == TRI_F32_MIXED && a.m >= kTcMin && a.n >= kTcMin && a.k >= kTcMin)
        return gemm_tc(*g.c, a, (g.keep || g.c->recipe == TRI_RECIPE_DIRECT) ? 6 : 3,
                       g.ws + g.lay.ks + g.lay.temps, name);
    return gemm_simt(*g.c, g.dt == TRI_F64 ? TRI_F64 : TRI_F32, a, name);
}

cudaError_t launch_leaf_lu(const GenCtx &g, void *a, int64_t lda, void *ks, int64_t ldk, int64_t off, int nb) {
    TraceScope ts(g.c->stream, g.dt == TRI_F64 ? "lu_leaf_f64" : "lu_leaf_f32",
                  (double)nb * nb * nb * 4.0 / 3.0, 0.0);
    if (g.dt == TRI_F64) {
        constexpr int L = 64, NT = 256;
        constexpr size_t sm = lu_leaf_smem<double, L>();
        cudaError_t e = cudaFuncSetAttribute(lu_leaf_kernel<double, L, NT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        lu_leaf_kernel<double, L, NT><<<1, NT, sm, g.c->stream>>>((const double *)a, lda, (double *)ks, ldk,
                                                                  off, nb, g.c->info,
                                                                  g.keep ? (double *)a : nullptr, g.info_base);
    } else {
        constexpr int L = 128, NT = 512;
        constexpr size_t sm = lu_leaf_smem<float, L>();
        cudaError_t e = cudaFuncSetAttribute(lu_leaf_kernel<float, L, NT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        lu_leaf_kernel<float, L, NT><<<1, NT, sm, g.c->stream>>>((const float *)a, lda, (float *)ks, ldk, off,
                                                                 nb, g.c->info, g.keep ? (float *)a : nullptr,
                                                                 g.info_base);
    }
    return cudaGetLastError();
}

cudaError_t rec(const GenCtx &g, uint8_t *a, int64_t lda, uint8_t *ks, int64_t ldk, int64_t off, int64_t m,
                int depth) {
    const size_t es = esz(g.dt);
    if (m <= g.L) return launch_leaf_lu(g, a, lda, ks, ldk, off, (int)m);
    const int64_t m1 = split_point(m, g.L), m2 = m - m1;
    cudaError_t e = rec(g, a, lda, ks, ldk, off, m1, depth + 1);
    if (e != cudaSuccess) return e;
    auto A = [&](int64_t i, int64_t j) { return (void *)(a + ((off + i) + (off + j) * lda) * es); };
    auto KS = [&](int64_t i, int64_t j) { return (void *)(ks + ((off + i) + (off + j) * ldk) * es); };
    uint8_t *tb = g.ws + g.lay.depth_off[depth];
    const size_t tsz = al((size_t)m1 * m2 * es);
    void *T1 = tb, *T2 = tb + tsz, *T3 = tb + 2 * tsz;
    // U12 = K11 A12  (m1 x m2)
    e = product(g, GemmArgs{m1, m2, m1, 1.0, KS(0, 0), ldk, OP_LOWER_UNIT, A(0, m1), lda, OP_FULL, 0.0, T1, m1,
                            OP_FULL}, "gen:u12");
    if (e != cudaSuccess) return e;
    // L21 = A21 S11  (m2 x m1)
    e = product(g, GemmArgs{m2, m1, m1, 1.0, A(m1, 0), lda, OP_FULL, KS(0, 0), ldk, OP_UPPER, 0.0, T2, m2,
                            OP_FULL}, "gen:l21");
    if (e != cudaSuccess) return e;
    // A22 <- A22 - L21 U12
    e = product(g, GemmArgs{m2, m2, m1, -1.0, T2, m2, OP_FULL, T1, m1, OP_FULL, 1.0, A(m1, m1), lda, OP_FULL},
                "gen:schur");
    if (e != cudaSuccess) return e;
    if (g.keep) {   // A12 <- U12, A21 <- L21 (the originals are no longer needed)
        e = cudaMemcpy2DAsync(A(0, m1), lda * es, T1, m1 * es, m1 * es, m2, cudaMemcpyDeviceToDevice, g.c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(A(m1, 0), lda * es, T2, m2 * es, m2 * es, m1, cudaMemcpyDeviceToDevice,
                                  g.c->stream);
        if (e != cudaSuccess) return e;
    }
    e = rec(g, a, lda, ks, ldk, off + m1, m2, depth + 1);
    if (e != cudaSuccess) return e;
    // K21 = -K22 (L21 K11)
    e = product(g, GemmArgs{m2, m1, m1, 1.0, T2, m2, OP_FULL, KS(0, 0), ldk, OP_LOWER_UNIT, 0.0, T3, m2,
                            OP_FULL}, "gen:k21a");
    if (e != cudaSuccess) return e;
    e = product(g, GemmArgs{m2, m1, m2, -1.0, KS(m1, m1), ldk, OP_LOWER_UNIT, T3, m2, OP_FULL, 0.0, KS(m1, 0),
                            ldk, OP_FULL}, "gen:k21b");
    if (e != cudaSuccess) return e;
    // S12 = -(S11 U12) S22
    e = product(g, GemmArgs{m1, m2, m1, 1.0, KS(0, 0), ldk, OP_UPPER, T1, m1, OP_FULL, 0.0, T3, m1, OP_FULL},
                "gen:s12a");
    if (e != cudaSuccess) return e;
    return product(g, GemmArgs{m1, m2, m2, -1.0, T3, m1, OP_FULL, KS(m1, m1), ldk, OP_UPPER, 0.0, KS(0, m1), ldk,
                               OP_FULL}, "gen:s12b");
}

template <typename T>
__global__ void take_diag_kernel(const T *__restrict__ a, int64_t lda, T *__restrict__ d, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = a[i + i * lda];
}

// Doolittle -> Crout with D = diag(U_d):  L = L_d D,  U = D^-1 U_d,  K = L^-1 = D^-1 K_d,
// S = U^-1 = S_d D.  The diagonals stay: L_ii = d_i in a, and K_ii = 1/d_i = (S_d)_ii in sk.
template <typename T>
__global__ void crout_form_kernel(T *__restrict__ a, int64_t lda, T *__restrict__ sk, int64_t ldsk,
                                  const T *__restrict__ d, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = blockIdx.y;
    if (i >= n || i == j) return;
    T *pa = a + i + j * lda, *ps = sk + i + j * ldsk;
    if (i > j) {
        *pa = *pa * d[j];
        *ps = *ps / d[i];
    } else {
        *pa = *pa / d[i];
        *ps = *ps * d[j];
    }
}

}  // namespace

size_t gen_inv_ws_bytes(int64_t n, tri_dtype dt) {
    if (n <= 0) return 0;
    return gen_layout(n, dt).total;
}

tri_status dense_newton_schulz(const Ctx &c, int64_t n, const float *a, int64_t lda, float *x, int64_t ldx,
                               float *r, int64_t ldr, void *planes);

// TRI_F32_MIXED with n >= kTcMin ends with one Newton-Schulz step on the dense inverse,
//     R = I - A X     six promoted terms (FP32 class; R is a difference of nearly equal
//                     quantities, so it needs the full 24 bits of A and X)
//     X <- X + X R    one term: R is as small as the three-term inverse's residual, so the
//                     BF16 error of this product is far below FP32 rounding of X
// which brings the normwise residual from the three-term products' level to FP32 level.
// R is written over the K\S buffer, which the final product has consumed.
tri_status run_gen_inv(const Ctx &c, tri_dtype dt, int64_t n, void *a, int64_t lda, void *ws, int64_t info_base) {
    GenCtx g{&c, dt, (uint8_t *)ws, gen_layout(n, dt), leaf_size(dt)};
    g.info_base = info_base;
    uint8_t *ks = (uint8_t *)ws;
    const int64_t ldk = n;
    const bool ns = g.lay.a0 > 0 && c.recipe != TRI_RECIPE_DIRECT;
    float *a0 = ns ? (float *)(g.ws + g.lay.ks + g.lay.temps + g.lay.planes) : nullptr;
    cudaError_t e = cudaSuccess;
    if (ns) e = cudaMemcpy2DAsync(a0, n * 4, a, lda * 4, n * 4, n, cudaMemcpyDeviceToDevice, c.stream);
    if (e != cudaSuccess) return TRI_ERR_CUDA;
    e = rec(g, (uint8_t *)a, lda, ks, ldk, 0, n, 0);
    if (e != cudaSuccess) return TRI_ERR_CUDA;
    // A^-1 = S K
    e = product(g, GemmArgs{n, n, n, 1.0, ks, ldk, OP_UPPER, ks, ldk, OP_LOWER_UNIT, 0.0, a, lda, OP_FULL},
                "gen:sk");
    if (e != cudaSuccess || !ns) return e == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
    return dense_newton_schulz(c, n, a0, n, (float *)a, lda, (float *)ks, ldk, g.ws + g.lay.ks + g.lay.temps);
}

// One Newton-Schulz step on a dense FP32 inverse X of A: R = I - A X (six promoted
// split-BF16 terms) into r, then X += X R (one term).  planes: gemm_tc_ws_bytes(n, n, n).
tri_status dense_newton_schulz(const Ctx &c, int64_t n, const float *a, int64_t lda, float *x, int64_t ldx,
                               float *r, int64_t ldr, void *planes) {
    GemmArgs g{n, n, n, -1.0, a, lda, OP_FULL, x, ldx, OP_FULL, 0.0, r, ldr, OP_FULL};
    g.dadd = 1.0;
    cudaError_t e = gemm_tc(c, g, 6, planes, "gen:ns_res");
    if (e != cudaSuccess) return TRI_ERR_CUDA;
    e = gemm_tc(c, GemmArgs{n, n, n, 1.0, x, ldx, OP_FULL, r, ldr, OP_FULL, 1.0, x, ldx, OP_FULL}, 1, planes,
                "gen:ns_upd");
    return e == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
}

size_t skul_ws_bytes(int64_t n, tri_dtype dt) {
    if (n <= 0) return 0;
    return gen_layout(n, dt, false).total + al((size_t)n * esz(dt));
}

// SKUL (Algorithm SKUL, Section 5.1): the recursion above with the factors kept, then the
// Crout scaling, so that a = L\U (U unit upper) and sk = K\S (S unit upper).
tri_status run_skul(const Ctx &c, tri_dtype dt, int64_t n, void *a, int64_t lda, void *sk, int64_t ldsk, void *ws) {
    if (n > 65535) return TRI_ERR_UNSUPPORTED;   // one grid row per column in crout_form_kernel
    GenCtx g{&c, dt, (uint8_t *)ws, gen_layout(n, dt, false), leaf_size(dt), true};
    cudaError_t e = rec(g, (uint8_t *)a, lda, (uint8_t *)sk, ldsk, 0, n, 0);
    if (e != cudaSuccess) return TRI_ERR_CUDA;
    void *d = g.ws + g.lay.total;
    const unsigned rb = (unsigned)((n + 255) / 256);
    TraceScope ts(c.stream, "skul:crout_form", 0.0, 6.0 * (double)n * n * esz(dt));
    if (dt == TRI_F64) {
        take_diag_kernel<double><<<rb, 256, 0, c.stream>>>((const double *)a, lda, (double *)d, n);
        crout_form_kernel<double><<<dim3(rb, (unsigned)n), 256, 0, c.stream>>>((double *)a, lda, (double *)sk, ldsk,
                                                                             (const double *)d, n);
    } else {
        take_diag_kernel<float><<<rb, 256, 0, c.stream>>>((const float *)a, lda, (float *)d, n);
        crout_form_kernel<float><<<dim3(rb, (unsigned)n), 256, 0, c.stream>>>((float *)a, lda, (float *)sk, ldsk,
                                                                            (const float *)d, n);
    }
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
}

}  // namespace triinv
