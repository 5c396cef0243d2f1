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

// FP32, 128 x 128 output tile, 16-wide k steps, both operands column-major without a
// transpose (the plain path's level products of lower matrices, the general inverse's
// products): 16-byte loads of whole 4-element groups along each operand's contiguous
// index (A along m, B along k).  A k step whose tile lies inside both operands' stored
// triangles and inside the matrix is loaded without masks; the others (diagonal tiles,
// ragged edges) go through per-element masks.  The host picks this kernel only when
// every group is 16-byte aligned (base pointers, leading dimensions and batch strides
// multiples of 4 elements).
constexpr int VBM = 128, VBN = 128, VBK = 16, VNT = 256;

__global__ void __launch_bounds__(VNT, 2)
gemm_simt_vec_kernel(int64_t M, int64_t N, int64_t K, float alpha, const float *__restrict__ A, int64_t lda,
                     int akind, const float *__restrict__ B, int64_t ldb, int bkind, float beta, float *C,
                     int64_t ldc, int cmask, int64_t sa, int64_t sb, int64_t sc, int64_t nb1, int64_t sa2,
                     int64_t sb2, int64_t sc2, int ksplit) {
    __shared__ __align__(16) float As[2][VBK][VBM + 4];
    __shared__ __align__(16) float Bs[2][VBK][VBN + 4];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * VBM;
    const int n0 = blockIdx.x * VBN;
    if (m0 >= M || n0 >= N) return;
    const int ks = (int)(blockIdx.z % ksplit);
    {
        const int64_t z = blockIdx.z / ksplit;
        const int64_t inner = z % nb1, outer = z / nb1;
        A += inner * sa + outer * sa2;
        B += inner * sb + outer * sb2;
        C += inner * sc + outer * sc2;
    }
    const bool c_low = cmask == OP_LOWER || cmask == OP_LOWER_UNIT;
    const bool c_up = cmask == OP_UPPER || cmask == OP_UPPER_UNIT;
    if (c_low && n0 > m0 + VBM - 1) return;
    if (c_up && m0 > n0 + VBN - 1) return;
    const bool a_low = (akind == OP_LOWER || akind == OP_LOWER_UNIT);
    const bool a_up = (akind == OP_UPPER || akind == OP_UPPER_UNIT);
    const bool b_low = (bkind == OP_LOWER || bkind == OP_LOWER_UNIT);
    const bool b_up = (bkind == OP_UPPER || bkind == OP_UPPER_UNIT);
    const bool a_unit = akind == OP_LOWER_UNIT || akind == OP_UPPER_UNIT;
    const bool b_unit = bkind == OP_LOWER_UNIT || bkind == OP_UPPER_UNIT;
    int kbeg = 0, kend = (int)K;
    if (a_low) kend = min(kend, m0 + VBM);
    if (a_up) kbeg = max(kbeg, (m0 / VBK) * VBK);
    if (b_low) kbeg = max(kbeg, (n0 / VBK) * VBK);
    if (b_up) kend = min(kend, n0 + VBN);
    if (ksplit > 1) {
        const int len = ((kend - kbeg + ksplit - 1) / ksplit + VBK - 1) / VBK * VBK;
        const int kb = kbeg + ks * len;
        kend = min(kend, kb + len);
        kbeg = kb;
        if (kbeg >= kend) return;
    }
    const int Mi = (int)M, Ni = (int)N;
    // A: thread -> rows am..am+3 (one 16-byte group), k rows ak and ak + 8 of the step
    const int am = (tid & 31) * 4, ak = tid >> 5;
    // B: thread -> k rows bk..bk+3 (one group), columns bn and bn + 64
    const int bk = (tid & 3) * 4, bn = tid >> 2;
    const bool m_full = m0 + VBM <= Mi, n_full = n0 + VBN <= Ni;
    float4 ra[2], rb[2];
    auto gload = [&](int kt) {
        // whole step inside the stored triangles and the matrix: no masks
        bool fast = kt + VBK <= kend;
        if (a_low) fast = fast && kt + VBK <= m0 + (a_unit ? 0 : 1);      // k <= m (k < m for unit)
        if (a_up) fast = fast && kt >= m0 + VBM - (a_unit ? 0 : 1);
        if (b_low) fast = fast && kt >= n0 + VBN - (b_unit ? 0 : 1);
        if (b_up) fast = fast && kt + VBK <= n0 + (b_unit ? 0 : 1);
        if (fast && m_full) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
                ra[h] = *reinterpret_cast<const float4 *>(A + (m0 + am) + (int64_t)(kt + ak + 8 * h) * lda);
        } else {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float v[4];
                const int k = kt + ak + 8 * h;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int m = m0 + am + i;
                    bool ok = m < Mi && k < kend;
                    if (a_low) ok = ok && k <= m;
                    if (a_up) ok = ok && k >= m;
                    float x = ok ? A[m + (int64_t)k * lda] : 0.f;
                    if (a_unit && k == m) x = 1.f;
                    v[i] = x;
                }
                ra[h] = make_float4(v[0], v[1], v[2], v[3]);
            }
        }
        if (fast && n_full) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
                rb[h] = *reinterpret_cast<const float4 *>(B + (kt + bk) + (int64_t)(n0 + bn + 64 * h) * ldb);
        } else {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float v[4];
                const int nn = n0 + bn + 64 * h;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int k = kt + bk + i;
                    bool ok = nn < Ni && k < kend;
                    if (b_low) ok = ok && k >= nn;
                    if (b_up) ok = ok && k <= nn;
                    float x = ok ? B[k + (int64_t)nn * ldb] : 0.f;
                    if (b_unit && k == nn) x = 1.f;
                    v[i] = x;
                }
                rb[h] = make_float4(v[0], v[1], v[2], v[3]);
            }
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int h = 0; h < 2; ++h) *reinterpret_cast<float4 *>(&As[buf][ak + 8 * h][am]) = ra[h];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            Bs[buf][bk + 0][bn + 64 * h] = rb[h].x;
            Bs[buf][bk + 1][bn + 64 * h] = rb[h].y;
            Bs[buf][bk + 2][bn + 64 * h] = rb[h].z;
            Bs[buf][bk + 3][bn + 64 * h] = rb[h].w;
        }
    };
    // compute: thread (ty, tx) owns rows ty*4 + {0..3} and 64 + ty*4 + {0..3}, likewise columns
    const int tx = tid % 16, ty = tid / 16;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    int buf = 0;
    if (kbeg < kend) {
        gload(kbeg);
        sstore(0);
        __syncthreads();
    }
    for (int kt = kbeg; kt < kend; kt += VBK) {
        const bool more = kt + VBK < kend;
        if (more) gload(kt + VBK);
#pragma unroll
        for (int kk = 0; kk < VBK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + tx * 4]);
            const float fa[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float fb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(fa[i], fb[j], acc[i][j]);
        }
        if (more) {
            sstore(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (gm >= Mi) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int gn = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (gn >= Ni) continue;
            if (c_low && gn > gm) continue;
            if (c_up && gm > gn) continue;
            float *c = C + gm + (int64_t)gn * ldc;
            if ((cmask == OP_LOWER_UNIT || cmask == OP_UPPER_UNIT) && gm == gn) {
                if (ksplit == 1) *c = 0.f;
                continue;
            }
            if (ksplit > 1) atomicAdd(c, alpha * acc[i][j]);
            else *c = beta == 0.f ? alpha * acc[i][j] : fmaf(alpha, acc[i][j], beta * *c);
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

// 16-byte groups of both operands: base pointers, leading dimensions and batch strides
// multiples of 4 FP32 elements.
bool vec_aligned(const GemmArgs &g) {
    auto ok = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    return ok(g.a) && ok(g.b) && g.lda % 4 == 0 && g.ldb % 4 == 0 && g.sa % 4 == 0 && g.sb % 4 == 0 &&
           g.sa2 % 4 == 0 && g.sb2 % 4 == 0;
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
    if (big && !g.ta && !g.tb && vec_aligned(g)) {
        if (ksplit > 1) {
            if (g.n > 65535) return cudaErrorInvalidValue;
            dim3 zg((unsigned)((g.m + 255) / 256), (unsigned)g.n, (unsigned)mats);
            zero_masked_kernel<float><<<zg, 256, 0, c.stream>>>((float *)g.c, g.m, g.n, g.ldc, g.cmask, g.sc, g.batch,
                                                                g.sc2);
        }
        dim3 grid((unsigned)((g.n + VBN - 1) / VBN), (unsigned)((g.m + VBM - 1) / VBM), (unsigned)(mats * ksplit));
        gemm_simt_vec_kernel<<<grid, VNT, 0, c.stream>>>(g.m, g.n, g.k, (float)g.alpha, (const float *)g.a, g.lda,
                                                         g.akind, (const float *)g.b, g.ldb, g.bkind, (float)g.beta,
                                                         (float *)g.c, g.ldc, g.cmask, g.sa, g.sb, g.sc, g.batch,
                                                         g.sa2, g.sb2, g.sc2, ksplit);
        return cudaGetLastError();
    }
    if (big) return launch_g<float, 128, 128, 8, 8, 8>(c, g, ksplit);
    return launch_g<float, 64, 64, 16, 4, 4>(c, g, ksplit);
}

}  // namespace triinv
