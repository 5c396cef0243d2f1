// trmm_simt.cu -- K2: the two dense products of one split level on CUDA cores
// (FP32 FFMA or FP64 DFMA), used by the plain TRI_F32 / TRI_F64 paths.
//
// For T = [A 0; B C] with X_A = A^-1 and X_C = C^-1 already in place, the block inverse
// of the proof of the main Theorem (Section 3) and of BRSI (Section 5.2) gives
//     X_21 = -X_C B X_A,
// evaluated as two products (each "triangular times full", Eq. "ptfm": m^3 flops):
//     mode 0:  W   = B * X_A     (X_A lower: column block n0 only needs k >= n0)
//     mode 1:  B  <- -X_C * W    (X_C lower: row block m0 only needs k < m0 + BM)
// Every pair of one level is independent: grid.z runs over them.
//
// Tiling: BM x BN output tile per CTA, BK-deep k-slices staged through double-buffered
// shared memory (registers prefetch slice k+1 while slice k is multiplied); each thread
// owns TM x TN outputs.  With TM = TN = 8 a thread's rows are {4*ty..4*ty+3} and
// {BM/2+4*ty..}, which keeps the vectorised shared-memory reads conflict-free.
// Zero tiles of the triangular operand are skipped through the k range; entries of the
// unreferenced triangle are never loaded (they are replaced by 0, or 1 on a unit
// diagonal).
#include <algorithm>

#include "internal.cuh"

namespace triinv {
namespace {

template <typename T, int BM, int BN, int BK, int TM, int TN>
struct Cfg {
    static constexpr int NT = (BM / TM) * (BN / TN);
    static constexpr int PAD = 4;
    static constexpr int A_PER = BM * BK / NT;
    static constexpr int B_PER = BN * BK / NT;
    static_assert((BM * BK) % NT == 0 && (BN * BK) % NT == 0, "load split");
    static_assert(TM == 4 || TM == 8, "TM");
    static_assert(TN == 4 || TN == 8, "TN");
};

// Row (or column) owned by a thread for its r-th micro-tile element.
template <int BX, int TX>
__device__ __forceinline__ int micro_index(int t, int r) {
    if (TX == 8) return (r < 4) ? (t * 4 + r) : (BX / 2 + t * 4 + (r - 4));
    return t * TX + r;
}

template <typename T, int BM, int BN, int BK, int TM, int TN, bool TRANS, bool UNIT, int MODE>
__global__ void __launch_bounds__(Cfg<T, BM, BN, BK, TM, TN>::NT)
trmm_level_kernel(T *__restrict__ a, int64_t lda, int64_t n, int64_t h, T *__restrict__ w,
                  int64_t pairs, int64_t bstride) {
    using C = Cfg<T, BM, BN, BK, TM, TN>;
    constexpr int NT = C::NT;
    __shared__ __align__(16) T As[2][BK][BM + C::PAD];
    __shared__ __align__(16) T Bs[2][BK][BN + C::PAD];

    const int tid = threadIdx.x;
    const int64_t bz = blockIdx.z / pairs;       // matrix of a strided batch
    const int64_t q = blockIdx.z % pairs;
    a += bz * bstride;
    w += bz * pairs * h * h;
    const int64_t a0 = q * 2 * h;             // first row/col of the A block
    const int64_t c0 = a0 + h;                // first row/col of the C block
    const int64_t hc = min(h, n - c0);        // rows of C (ragged on the last pair)
    const int64_t m0 = (int64_t)blockIdx.y * BM;
    const int64_t n0 = (int64_t)blockIdx.x * BN;
    if (m0 >= hc || n0 >= h) return;
    T *wq = w + q * h * h;

    // k range with the zero tiles of the triangular operand removed.
    int64_t kbeg, kend;
    if (MODE == 0) { kbeg = (n0 / BK) * BK; kend = h; }
    else { kbeg = 0; kend = min(m0 + BM, hc); }

    // Element fetchers.  A is (m, k), B is (k, nn) in tile-local coordinates.
    auto fetchA = [&](int64_t m, int64_t k) -> T {
        const int64_t gm = m0 + m;
        if (gm >= hc || k >= kend) return T(0);
        if (MODE == 0) return a[vidx<TRANS>(c0 + gm, a0 + k, lda)];        // B block
        if (k > gm) return T(0);                                            // X_C lower
        if (UNIT && k == gm) return T(1);
        return a[vidx<TRANS>(c0 + gm, c0 + k, lda)];
    };
    auto fetchB = [&](int64_t k, int64_t nn) -> T {
        const int64_t gn = n0 + nn;
        if (gn >= h || k >= kend) return T(0);
        if (MODE == 0) {                                                     // X_A lower
            if (k < gn) return T(0);
            if (UNIT && k == gn) return T(1);
            return a[vidx<TRANS>(a0 + k, a0 + gn, lda)];
        }
        return wq[k + gn * h];                                               // W col-major
    };
    // Which index is contiguous in memory decides the thread->element map of the loads.
    constexpr bool A_CONTIG_M = !TRANS;                 // A: (m,k) contiguous along m?
    constexpr bool B_CONTIG_K = (MODE == 1) || !TRANS;  // B: (k,nn) contiguous along k?

    T ra[C::A_PER], rb[C::B_PER];
    auto gload = [&](int64_t kt) {
#pragma unroll
        for (int r = 0; r < C::A_PER; ++r) {
            const int idx = tid + r * NT;
            int m, k;
            if (A_CONTIG_M) { m = idx % BM; k = idx / BM; }
            else { k = idx % BK; m = idx / BK; }
            ra[r] = fetchA(m, kt + k);
        }
#pragma unroll
        for (int r = 0; r < C::B_PER; ++r) {
            const int idx = tid + r * NT;
            int k, nn;
            if (B_CONTIG_K) { k = idx % BK; nn = idx / BK; }
            else { nn = idx % BN; k = idx / BN; }
            rb[r] = fetchB(kt + k, nn);
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int r = 0; r < C::A_PER; ++r) {
            const int idx = tid + r * NT;
            int m, k;
            if (A_CONTIG_M) { m = idx % BM; k = idx / BM; }
            else { k = idx % BK; m = idx / BK; }
            As[buf][k][m] = ra[r];
        }
#pragma unroll
        for (int r = 0; r < C::B_PER; ++r) {
            const int idx = tid + r * NT;
            int k, nn;
            if (B_CONTIG_K) { k = idx % BK; nn = idx / BK; }
            else { nn = idx % BN; k = idx / BN; }
            Bs[buf][k][nn] = rb[r];
        }
    };

    const int tx = tid % (BN / TN);
    const int ty = tid / (BN / TN);
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    int buf = 0;
    if (kbeg < kend) {
        gload(kbeg);
        sstore(0);
        __syncthreads();
    }
    for (int64_t kt = kbeg; kt < kend; kt += BK) {
        const bool more = kt + BK < kend;
        if (more) gload(kt + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T fa[TM], fb[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) fa[i] = As[buf][kk][micro_index<BM, TM>(ty, i)];
#pragma unroll
            for (int j = 0; j < TN; ++j) fb[j] = Bs[buf][kk][micro_index<BN, TN>(tx, j)];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(fa[i], fb[j], acc[i][j]);
        }
        if (more) {
            sstore(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }

    // Epilogue.
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t gm = m0 + micro_index<BM, TM>(ty, i);
        if (gm >= hc) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int64_t gn = n0 + micro_index<BN, TN>(tx, j);
            if (gn >= h) continue;
            if (MODE == 0) wq[gm + gn * h] = acc[i][j];
            else a[vidx<TRANS>(c0 + gm, a0 + gn, lda)] = -acc[i][j];
        }
    }
}

template <typename T, int BM, int BN, int BK, int TM, int TN, int MODE>
cudaError_t launch_cfg(const Ctx &c, bool trans, bool unit, int64_t n, T *a, int64_t lda,
                       int64_t h, T *w, int64_t batch, int64_t bstride) {
    using C = Cfg<T, BM, BN, BK, TM, TN>;
    const int64_t pairs = level_pairs(n, h);
    if (pairs <= 0 || batch <= 0) return cudaSuccess;
    if (pairs * batch > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((h + BN - 1) / BN), (unsigned)((h + BM - 1) / BM), (unsigned)(pairs * batch));
    if (trans) {
        if (unit) trmm_level_kernel<T, BM, BN, BK, TM, TN, true, true, MODE><<<grid, C::NT, 0, c.stream>>>(a, lda, n, h, w, pairs, bstride);
        else trmm_level_kernel<T, BM, BN, BK, TM, TN, true, false, MODE><<<grid, C::NT, 0, c.stream>>>(a, lda, n, h, w, pairs, bstride);
    } else {
        if (unit) trmm_level_kernel<T, BM, BN, BK, TM, TN, false, true, MODE><<<grid, C::NT, 0, c.stream>>>(a, lda, n, h, w, pairs, bstride);
        else trmm_level_kernel<T, BM, BN, BK, TM, TN, false, false, MODE><<<grid, C::NT, 0, c.stream>>>(a, lda, n, h, w, pairs, bstride);
    }
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t launch_mode(const Ctx &c, bool trans, bool unit, int64_t n, T *a, int64_t lda,
                        int64_t h, T *w, int64_t batch, int64_t bstride) {
    if (sizeof(T) == 4 && h >= 128)
        return launch_cfg<T, 128, 128, 8, 8, 8, MODE>(c, trans, unit, n, a, lda, h, w, batch, bstride);
    return launch_cfg<T, 64, 64, 16, 4, 4, MODE>(c, trans, unit, n, a, lda, h, w, batch, bstride);
}

}  // namespace

cudaError_t launch_trmm_level(const Ctx &c, tri_dtype dt, bool trans, bool unit, int mode,
                              int64_t n, void *a, int64_t lda, int64_t h, void *w,
                              int64_t batch, int64_t bstride) {
    const int64_t pairs = level_pairs(n, h);
    if (pairs <= 0) return cudaSuccess;
    // Algorithmic flops: mode 0 is hc x h times an h x h lower operand, 2*hc*sum(h-j);
    // mode 1 is an hc x hc lower operand times hc x h.  Only the last pair may be ragged.
    const int64_t hc_last = std::min<int64_t>(h, n - (pairs - 1) * 2 * h - h);
    const double es = dt == TRI_F64 ? 8.0 : 4.0;
    double flops = 0.0, bytes = 0.0;
    for (int k = 0; k < 2; ++k) {
        const double cnt = k == 0 ? (double)(pairs - 1) : 1.0;
        const double hc = k == 0 ? (double)h : (double)hc_last;
        const double hd = (double)h;
        flops += cnt * (mode == 0 ? hc * hd * (hd + 1.0) : hd * hc * (hc + 1.0));
        bytes += cnt * es * (mode == 0 ? (hc * hd + hd * (hd + 1) / 2 + hc * hd)
                                       : (hc * (hc + 1) / 2 + hc * hd + hc * hd));
    }
    const char *name = dt == TRI_F64 ? (mode == 0 ? "trmm_f64_right" : "trmm_f64_left")
                                     : (mode == 0 ? "trmm_f32_right" : "trmm_f32_left");
    TraceScope ts(c.stream, name, flops * (double)batch, bytes * (double)batch);
    if (dt == TRI_F64) {
        if (mode == 0) return launch_mode<double, 0>(c, trans, unit, n, (double *)a, lda, h, (double *)w, batch, bstride);
        return launch_mode<double, 1>(c, trans, unit, n, (double *)a, lda, h, (double *)w, batch, bstride);
    }
    if (mode == 0) return launch_mode<float, 0>(c, trans, unit, n, (float *)a, lda, h, (float *)w, batch, bstride);
    return launch_mode<float, 1>(c, trans, unit, n, (float *)a, lda, h, (float *)w, batch, bstride);
}

}  // namespace triinv
