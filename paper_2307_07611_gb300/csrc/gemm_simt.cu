// gemm_simt.cu -- generic triangular-aware product on CUDA cores (FP32 FFMA / FP64 DFMA):
//     C = alpha * A * B + beta * C
// with A (M x K), B (K x N), C (M x N) column-major and each operand full, lower or upper
// triangular (optionally with an implicit unit diagonal).  The zero part of a triangular
// operand is skipped through the k range of each tile and never loaded.  Used by the
// general inverse (block LU with inverse factors, then U^-1 L^-1) and by the adjoint.
#include <algorithm>

#include "gemm.cuh"

namespace triinv {
namespace {

template <typename T, int BM, int BN, int BK, int TM, int TN>
struct GCfg {
    static constexpr int NT = (BM / TM) * (BN / TN);
    static constexpr int PAD = 4;
    static constexpr int A_PER = BM * BK / NT;
    static constexpr int B_PER = BN * BK / NT;
};

template <int BX, int TX>
__device__ __forceinline__ int gmicro(int t, int r) {
    if (TX == 8) return (r < 4) ? (t * 4 + r) : (BX / 2 + t * 4 + (r - 4));
    return t * TX + r;
}

// Element (r, c) of op(P) (P or P^T, P column-major) for a triangular-kind operand;
// r, c index op(P).  Entries outside the triangle are never read.
template <typename T>
__device__ __forceinline__ T tri_fetch(const T *p, int64_t ld, bool tr, int kind, int64_t r, int64_t c) {
    const int64_t o = tr ? (c + r * ld) : (r + c * ld);
    switch (kind) {
        case OP_FULL: return p[o];
        case OP_LOWER: return c <= r ? p[o] : T(0);
        case OP_UPPER: return c >= r ? p[o] : T(0);
        case OP_LOWER_UNIT: return c < r ? p[o] : (c == r ? T(1) : T(0));
        case OP_UPPER_UNIT: return c > r ? p[o] : (c == r ? T(1) : T(0));
    }
    return T(0);
}

template <typename T, int BM, int BN, int BK, int TM, int TN, bool TA, bool TB>
__global__ void __launch_bounds__(GCfg<T, BM, BN, BK, TM, TN>::NT)
gemm_simt_kernel(int64_t M, int64_t N, int64_t K, T alpha, const T *__restrict__ A, int64_t lda,
                 int akind, const T *__restrict__ B, int64_t ldb, int bkind, T beta, T *C,
                 int64_t ldc, int cmask, int64_t sa, int64_t sb, int64_t sc, int64_t nb1,
                 int64_t sa2, int64_t sb2, int64_t sc2, int ksplit) {
    using Cf = GCfg<T, BM, BN, BK, TM, TN>;
    constexpr int NT = Cf::NT;
    __shared__ __align__(16) T As[2][BK][BM + Cf::PAD];
    __shared__ __align__(16) T Bs[2][BK][BN + Cf::PAD];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * BM;
    const int n0 = blockIdx.x * BN;
    if (m0 >= M || n0 >= N) return;
    // blockIdx.z = matrix * ksplit + k slice
    const int ks = (int)(blockIdx.z % ksplit);
    {
        const int64_t z = blockIdx.z / ksplit;
        const int64_t inner = z % nb1, outer = z / nb1;
        A += inner * sa + outer * sa2;
        B += inner * sb + outer * sb2;
        C += inner * sc + outer * sc2;
    }
    // Output mask: skip tiles entirely outside the stored triangle.
    const bool c_low = cmask == OP_LOWER || cmask == OP_LOWER_UNIT;
    const bool c_up = cmask == OP_UPPER || cmask == OP_UPPER_UNIT;
    if (c_low && n0 > m0 + BM - 1) return;
    if (c_up && m0 > n0 + BN - 1) return;

    int kbeg = 0, kend = (int)K;
    const bool a_low = (akind == OP_LOWER || akind == OP_LOWER_UNIT);
    const bool a_up = (akind == OP_UPPER || akind == OP_UPPER_UNIT);
    const bool b_low = (bkind == OP_LOWER || bkind == OP_LOWER_UNIT);
    const bool b_up = (bkind == OP_UPPER || bkind == OP_UPPER_UNIT);
    const bool a_unit = akind == OP_LOWER_UNIT || akind == OP_UPPER_UNIT;
    const bool b_unit = bkind == OP_LOWER_UNIT || bkind == OP_UPPER_UNIT;
    if (a_low) kend = min(kend, m0 + BM);          // op(A)(m,k) = 0 for k > m
    if (a_up) kbeg = max(kbeg, (m0 / BK) * BK);    // op(A)(m,k) = 0 for k < m
    if (b_low) kbeg = max(kbeg, (n0 / BK) * BK);   // op(B)(k,n) = 0 for k < n
    if (b_up) kend = min(kend, n0 + BN);           // op(B)(k,n) = 0 for k > n
    if (ksplit > 1) {
        // this CTA's slice of the k range (whole BK steps); the slices add into a C that
        // was zeroed before the launch
        const int len = ((kend - kbeg + ksplit - 1) / ksplit + BK - 1) / BK * BK;
        const int kb = kbeg + ks * len;
        kend = min(kend, kb + len);
        kbeg = kb;
        if (kbeg >= kend) return;
    }

    // Thread -> element maps follow the contiguous index of each operand in memory.
    // Each thread keeps a pointer per loaded element and advances it by one k-slice per
    // step; the masks are 32-bit compares.
    int am[Cf::A_PER], ak[Cf::A_PER], bk[Cf::B_PER], bn[Cf::B_PER];
    const T *pa[Cf::A_PER];
    const T *pb[Cf::B_PER];
    const int64_t a_kstep = TA ? 1 : lda, b_kstep = TB ? ldb : 1;
#pragma unroll
    for (int r = 0; r < Cf::A_PER; ++r) {
        const int idx = tid + r * NT;
        if (TA) { ak[r] = idx % BK; am[r] = idx / BK; }
        else { am[r] = idx % BM; ak[r] = idx / BM; }
        const int64_t gm = m0 + am[r], gk = kbeg + ak[r];
        pa[r] = A + (TA ? (gk + gm * lda) : (gm + gk * lda));
        am[r] += m0;
    }
#pragma unroll
    for (int r = 0; r < Cf::B_PER; ++r) {
        const int idx = tid + r * NT;
        if (TB) { bn[r] = idx % BN; bk[r] = idx / BN; }
        else { bk[r] = idx % BK; bn[r] = idx / BK; }
        const int64_t gk = kbeg + bk[r], gn = n0 + bn[r];
        pb[r] = B + (TB ? (gn + gk * ldb) : (gk + gn * ldb));
        bn[r] += n0;
    }
    const int Mi = (int)M, Ni = (int)N;

    T ra[Cf::A_PER], rb[Cf::B_PER];
    auto gload = [&](int kt) {
#pragma unroll
        for (int r = 0; r < Cf::A_PER; ++r) {
            const int m = am[r], k = kt + ak[r];
            bool ok = m < Mi && k < kend;
            if (a_low) ok = ok && k <= m;
            if (a_up) ok = ok && k >= m;
            T v = ok ? *pa[r] : T(0);
            if (a_unit && k == m) v = T(1);
            ra[r] = v;
            pa[r] += BK * a_kstep;
        }
#pragma unroll
        for (int r = 0; r < Cf::B_PER; ++r) {
            const int k = kt + bk[r], nn = bn[r];
            bool ok = nn < Ni && k < kend;
            if (b_low) ok = ok && k >= nn;
            if (b_up) ok = ok && k <= nn;
            T v = ok ? *pb[r] : T(0);
            if (b_unit && k == nn) v = T(1);
            rb[r] = v;
            pb[r] += BK * b_kstep;
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int r = 0; r < Cf::A_PER; ++r) As[buf][ak[r]][am[r] - m0] = ra[r];
#pragma unroll
        for (int r = 0; r < Cf::B_PER; ++r) Bs[buf][bk[r]][bn[r] - n0] = rb[r];
    };
    const int tx = tid % (BN / TN), ty = tid / (BN / TN);
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
    for (int kt = kbeg; kt < kend; kt += BK) {
        const bool more = kt + BK < kend;
        if (more) gload(kt + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T fa[TM], fb[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) fa[i] = As[buf][kk][gmicro<BM, TM>(ty, i)];
#pragma unroll
            for (int j = 0; j < TN; ++j) fb[j] = Bs[buf][kk][gmicro<BN, TN>(tx, j)];
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
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int gm = m0 + gmicro<BM, TM>(ty, i);
        if (gm >= Mi) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int gn = n0 + gmicro<BN, TN>(tx, j);
            if (gn >= Ni) continue;
            if (c_low && gn > gm) continue;
            if (c_up && gm > gn) continue;
            T *c = C + gm + (int64_t)gn * ldc;
            if ((cmask == OP_LOWER_UNIT || cmask == OP_UPPER_UNIT) && gm == gn) {
                if (ksplit == 1) *c = T(0);
                continue;
            }
            if (ksplit > 1) atomicAdd(c, alpha * acc[i][j]);
            else *c = beta == T(0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *c);
        }
    }
}

// Zeroes the part of C (M x N per matrix) that a product with output mask cmask writes.
template <typename T>
__global__ void zero_masked_kernel(T *C, int64_t M, int64_t N, int64_t ldc, int cmask, int64_t sc, int64_t nb1,
                                   int64_t sc2) {
    const int64_t gm = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gn = blockIdx.y;
    if (gm >= M) return;
    const bool c_low = cmask == OP_LOWER || cmask == OP_LOWER_UNIT;
    const bool c_up = cmask == OP_UPPER || cmask == OP_UPPER_UNIT;
    if ((c_low && gn > gm) || (c_up && gm > gn)) return;
    const int64_t z = blockIdx.z, inner = z % nb1, outer = z / nb1;
    C[inner * sc + outer * sc2 + gm + gn * ldc] = T(0);
}

template <typename T, int BM, int BN, int BK, int TM, int TN, bool TA, bool TB>
cudaError_t launch_g2(const Ctx &c, const GemmArgs &g, int ksplit) {
    using Cf = GCfg<T, BM, BN, BK, TM, TN>;
    const int64_t mats = g.batch * g.batch2;
    if (ksplit > 1) {
        if (g.n > 65535) return cudaErrorInvalidValue;
        dim3 zg((unsigned)((g.m + 255) / 256), (unsigned)g.n, (unsigned)mats);
        zero_masked_kernel<T><<<zg, 256, 0, c.stream>>>((T *)g.c, g.m, g.n, g.ldc, g.cmask, g.sc, g.batch, g.sc2);
    }
    dim3 grid((unsigned)((g.n + BN - 1) / BN), (unsigned)((g.m + BM - 1) / BM), (unsigned)(mats * ksplit));
    gemm_simt_kernel<T, BM, BN, BK, TM, TN, TA, TB><<<grid, Cf::NT, 0, c.stream>>>(
        g.m, g.n, g.k, (T)g.alpha, (const T *)g.a, g.lda, g.akind, (const T *)g.b, g.ldb, g.bkind,
        (T)g.beta, (T *)g.c, g.ldc, g.cmask, g.sa, g.sb, g.sc, g.batch, g.sa2, g.sb2, g.sc2, ksplit);
    return cudaGetLastError();
}

template <typename T, int BM, int BN, int BK, int TM, int TN>
cudaError_t launch_g(const Ctx &c, const GemmArgs &g, int ksplit = 1) {
    if (g.ta) return g.tb ? launch_g2<T, BM, BN, BK, TM, TN, true, true>(c, g, ksplit)
                          : launch_g2<T, BM, BN, BK, TM, TN, true, false>(c, g, ksplit);
    return g.tb ? launch_g2<T, BM, BN, BK, TM, TN, false, true>(c, g, ksplit)
                : launch_g2<T, BM, BN, BK, TM, TN, false, false>(c, g, ksplit);
}

// FP64 products run on a part with little FP64 throughput per SM (2 DFMA per clock):
// 32 x 32 tiles, and the k range split over several CTAs (atomic adds into a zeroed C)
// until the grid covers about four waves of the SMs.  Split only when beta == 0; C never
// overlaps A or B in the callers (level products write the workspace or the B block they
// no longer read).
cudaError_t launch_f64(const Ctx &c, const GemmArgs &g) {
    const int64_t mats = g.batch * g.batch2;
    const int64_t tiles = ((g.m + 31) / 32) * ((g.n + 31) / 32) * mats;
    int ksplit = 1;
    if (g.beta == 0.0 && tiles < 4 * (int64_t)c.sm_count) {
        const int64_t want = (4 * (int64_t)c.sm_count + tiles - 1) / tiles;
        const int64_t most = std::max<int64_t>(1, g.k / 16);   // at least one 16-wide k step per slice
        ksplit = (int)std::min<int64_t>({want, most, 64, 65535 / mats});
        ksplit = std::max(ksplit, 1);
    }
    return launch_g<double, 32, 32, 16, 2, 2>(c, g, ksplit);
}

}  // namespace

double gemm_flops(const GemmArgs &g) {
    // 2 x the multiply-adds that are not structurally zero.
    const double M = (double)g.m, N = (double)g.n, K = (double)g.k;
    const bool a_tri = g.akind != OP_FULL, b_tri = g.bkind != OP_FULL;
    if (!a_tri && !b_tri) return 2.0 * M * N * K;
    if (a_tri && !b_tri) return M * (M + 1) * N;           // square triangular A (M == K)
    if (!a_tri && b_tri) return M * N * (N + 1);           // square triangular B (N == K)
    const bool a_low = g.akind == OP_LOWER || g.akind == OP_LOWER_UNIT;
    const bool b_low = g.bkind == OP_LOWER || g.bkind == OP_LOWER_UNIT;
    if (a_low == b_low) return M * (M + 1) * (M + 2) / 3.0;  // triangular result
    return M * (M + 1) * (2 * M + 1) / 3.0;                 // upper x lower or lower x upper
}

cudaError_t gemm_simt(const Ctx &c, tri_dtype dt, const GemmArgs &g, const char *trace_name) {
    if (g.dadd != 0.0) return cudaErrorInvalidValue;   // diagonal addend: tensor-core path only
    if (g.m <= 0 || g.n <= 0 || g.batch <= 0 || g.batch2 <= 0) return cudaSuccess;
    if (g.batch * g.batch2 > 65535 || g.m >= (1ll << 31) || g.n >= (1ll << 31) || g.k >= (1ll << 31))
        return cudaErrorInvalidValue;
    TraceScope ts(c.stream, trace_name, gemm_flops(g) * (double)(g.batch * g.batch2), 0.0);
    if (dt == TRI_F64) return launch_f64(c, g);
    const bool big = g.m >= 128 && g.n >= 128;
    const int64_t bt = big ? 128 : 64;
    int ksplit = 1;
    const int64_t mats = g.batch * g.batch2;
    const int64_t tiles = ((g.m + bt - 1) / bt) * ((g.n + bt - 1) / bt) * mats;
    if (g.split_k && g.beta == 0.0 && tiles < 2 * (int64_t)c.sm_count) {
        const int64_t want = (2 * (int64_t)c.sm_count + tiles - 1) / tiles;
        const int64_t most = std::max<int64_t>(1, g.k / 128);   // at least 128 of k per slice
        ksplit = (int)std::max<int64_t>(1, std::min<int64_t>({want, most, 64, 65535 / mats}));
    }
    if (big) return launch_g<float, 128, 128, 8, 8, 8>(c, g, ksplit);
    return launch_g<float, 64, 64, 16, 4, 4>(c, g, ksplit);
}

}  // namespace triinv
