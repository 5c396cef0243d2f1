// leaf.cu -- K1: in-place inverse of the diagonal leaf blocks.
//
// Each CTA owns one leaf (an nb x nb diagonal block of the lower view, nb <= LEAF) and
// runs the column recurrence of CRIT (Section 4.2, Algorithm "CRIT", transposed to
// lower form):
//     x_jj = 1/t_jj,    x_ij = -(1/t_ii) * sum_{k=j}^{i-1} t_ik x_kj.
// The sum is evaluated right-looking: after row k of X is final, every pending entry
// (i > k, j <= k) adds t_ik * x_kj.  This is the same sum in the same ascending-k order
// as the recurrence; it just lets all (i, j) pairs advance together, one barrier per k.
// Each thread keeps its entries of X in registers (column j = tid % LEAF, rows
// i = tid / LEAF + r * (NT / LEAF)); T sits in shared memory.
//
// Ill-conditioned leaves (FP32): when max|X| max|T| of the FP32 inverse exceeds the growth
// limit (tri_set_growth_limit), the leaf is inverted again with FP64 arithmetic.
//
// Rounding: 1/t_ii is one IEEE round-to-nearest division, so the diagonal of X is
// exactly RN(1/t_ii); off-diagonal entries use fused multiply-adds and a multiplication
// by that reciprocal (the paper's "appropriate diagonal matrix multiplication", Section
// 2), which differs from a division by t_ii by at most one rounding.
#include <climits>
#include <type_traits>

#include "internal.cuh"

namespace triinv {
namespace {

// Loads the leaf's lower triangle into ts as U (the strict upper part and the padding
// become zero, the padded diagonal one); the contiguous index runs fastest across threads.
// Returns this thread's max |t_ik| over the valid part.
template <typename U, typename T, int LEAF, int NT, bool TRANS, bool UNIT>
__device__ __forceinline__ float load_leaf(const T *__restrict__ a, int64_t lda, int64_t r0, int nb,
                                           U (*ts)[LEAF + 1]) {
    float tmax = 0.f;
    for (int idx = threadIdx.x; idx < LEAF * LEAF; idx += NT) {
        int i, k;
        if (TRANS) { i = idx / LEAF; k = idx % LEAF; }
        else { i = idx % LEAF; k = idx / LEAF; }
        U v = U(0);
        if (i < nb && k < nb) {
            if (k < i) v = (U)a[vidx<TRANS>(r0 + i, r0 + k, lda)];
            else if (k == i) v = UNIT ? U(1) : (U)a[vidx<TRANS>(r0 + i, r0 + i, lda)];
            tmax = fmaxf(tmax, fabsf((float)v));
        } else if (i == k) {
            v = U(1);
        }
        ts[i][k] = v;
    }
    return tmax;
}

// The right-looking column recurrence on the leaf in ts (type U), into acc (this thread's
// column j = tid % LEAF, rows tid / LEAF + r * (NT / LEAF)).  Ends with a barrier.
template <typename U, int LEAF, int NT>
__device__ __forceinline__ void leaf_recurrence(U (*ts)[LEAF + 1], U *dinv, U (*xrow)[LEAF], int nb,
                                                U (&acc)[LEAF * LEAF / NT]) {
    constexpr int G = NT / LEAF;
    constexpr int RPT = LEAF * LEAF / NT;
    const int tid = threadIdx.x;
    if (tid < LEAF) dinv[tid] = U(1) / ts[tid][tid];
    __syncthreads();
    const int j = tid % LEAF;
    const int ig = tid / LEAF;
#pragma unroll
    for (int r = 0; r < RPT; ++r) acc[r] = U(0);
    for (int k = 0; k < nb; ++k) {
        const U dk = dinv[k];
        // Row k becomes final: x_kk = 1/t_kk, x_kj = -acc_kj / t_kk (j < k).
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int i = ig + r * G;
            if (i == k && j <= k) {
                const U x = (j == k) ? dk : -acc[r] * dk;
                acc[r] = x;
                xrow[k & 1][j] = x;
            }
        }
        __syncthreads();
        if (j <= k) {
            const U xkj = xrow[k & 1][j];
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int i = ig + r * G;
                if (i > k) acc[r] = fma(ts[i][k], xkj, acc[r]);
            }
        }
    }
    __syncthreads();
}

// tau > 0 (FP32 leaves only): growth limit.  When the FP32 inverse of the leaf has
// max|X| max|T| > tau, the leaf (still unchanged in memory) is inverted again with FP64
// arithmetic in the same shared memory, and that result is stored rounded to FP32.
template <typename T, int LEAF, int NT, bool TRANS, bool UNIT>
__global__ void __launch_bounds__(NT) leaf_kernel(T *__restrict__ a, int64_t lda, int64_t n,
                                                  long long *__restrict__ info, int64_t bstride, float tau) {
    static_assert(NT % LEAF == 0 && (LEAF * LEAF) % NT == 0, "thread layout");
    constexpr int G = NT / LEAF;          // row groups
    constexpr int RPT = LEAF * LEAF / NT; // rows per thread
    constexpr bool FALLBACK = std::is_same<T, float>::value;
    using W = typename std::conditional<FALLBACK, double, T>::type;   // widest type used
    __shared__ __align__(16) W ts_raw[LEAF][LEAF + 1];
    __shared__ W dinv_raw[LEAF];
    __shared__ W xrow_raw[2][LEAF];
    __shared__ unsigned s_tmax, s_xmax;
    T (*ts)[LEAF + 1] = reinterpret_cast<T (*)[LEAF + 1]>(&ts_raw[0][0]);

    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * LEAF;
    a += (int64_t)blockIdx.y * bstride;          // matrix of a strided batch
    const int nb = (int)((n - r0) < (int64_t)LEAF ? (n - r0) : (int64_t)LEAF);
    if (tid == 0) s_tmax = s_xmax = 0u;

    const float tmax = load_leaf<T, T, LEAF, NT, TRANS, UNIT>(a, lda, r0, nb, ts);
    __syncthreads();
    if (tid < LEAF) {
        T d = ts[tid][tid];
        if (tid < nb && (d == T(0) || !isfinite(d)))
            atomicMin(info, gridDim.y > 1 ? (long long)blockIdx.y : (long long)(r0 + tid));
    }
    T acc[RPT];
    leaf_recurrence<T, LEAF, NT>(ts, reinterpret_cast<T *>(dinv_raw), reinterpret_cast<T (*)[LEAF]>(&xrow_raw[0][0]),
                                 nb, acc);
    const int j = tid % LEAF;
    const int ig = tid / LEAF;
    if constexpr (FALLBACK) {
        if (tau > 0.f) {
            float xmax = 0.f;
#pragma unroll
            for (int r = 0; r < RPT; ++r)
                if (ig + r * G < nb && j < nb) xmax = fmaxf(xmax, fabsf(acc[r]));
            // one shared-memory atomic per warp (non-negative floats order like their bits)
            float v = xmax, w = tmax;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
                w = fmaxf(w, __shfl_xor_sync(0xffffffffu, w, o));
            }
            if ((tid & 31) == 0) {
                atomicMax(&s_xmax, __float_as_uint(v));
                atomicMax(&s_tmax, __float_as_uint(w));
            }
            __syncthreads();
            const float growth = __uint_as_float(s_xmax) * __uint_as_float(s_tmax);
            if (!(growth <= tau)) {   // uniform over the CTA
                load_leaf<double, T, LEAF, NT, TRANS, UNIT>(a, lda, r0, nb, ts_raw);
                __syncthreads();
                double accd[RPT];
                leaf_recurrence<double, LEAF, NT>(ts_raw, dinv_raw, xrow_raw, nb, accd);
#pragma unroll
                for (int r = 0; r < RPT; ++r) acc[r] = (T)accd[r];
            }
        }
    }
    // Stage X through shared memory so the global store is coalesced.
#pragma unroll
    for (int r = 0; r < RPT; ++r) ts[ig + r * G][j] = acc[r];
    __syncthreads();
    for (int idx = tid; idx < LEAF * LEAF; idx += NT) {
        int i, k;
        if (TRANS) { i = idx / LEAF; k = idx % LEAF; }
        else { i = idx % LEAF; k = idx / LEAF; }
        if (i < nb && k < nb && k <= i && !(UNIT && i == k))
            a[vidx<TRANS>(r0 + i, r0 + k, lda)] = ts[i][k];
    }
}

template <typename T, int LEAF>
cudaError_t launch_leaf_t(const Ctx &c, bool trans, bool unit, int64_t n, T *a, int64_t lda,
                          int64_t batch, int64_t bstride) {
    const float tau = std::is_same<T, float>::value ? c.tau : 0.f;
    constexpr int NT = LEAF >= 32 ? 256 : 128;
    const int64_t blocks = (n + LEAF - 1) / LEAF;
    if (blocks <= 0 || batch <= 0) return cudaSuccess;
    dim3 grid((unsigned)blocks, (unsigned)batch);
    if (trans) {
        if (unit) leaf_kernel<T, LEAF, NT, true, true><<<grid, NT, 0, c.stream>>>(a, lda, n, c.info, bstride, tau);
        else leaf_kernel<T, LEAF, NT, true, false><<<grid, NT, 0, c.stream>>>(a, lda, n, c.info, bstride, tau);
    } else {
        if (unit) leaf_kernel<T, LEAF, NT, false, true><<<grid, NT, 0, c.stream>>>(a, lda, n, c.info, bstride, tau);
        else leaf_kernel<T, LEAF, NT, false, false><<<grid, NT, 0, c.stream>>>(a, lda, n, c.info, bstride, tau);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_leaf_dispatch(const Ctx &c, bool trans, bool unit, int64_t n, T *a,
                                 int64_t lda, int leaf, int64_t batch, int64_t bstride) {
    switch (leaf) {
        case 16: return launch_leaf_t<T, 16>(c, trans, unit, n, a, lda, batch, bstride);
        case 32: return launch_leaf_t<T, 32>(c, trans, unit, n, a, lda, batch, bstride);
        case 64: return launch_leaf_t<T, 64>(c, trans, unit, n, a, lda, batch, bstride);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_leaf(const Ctx &c, tri_dtype dt, bool trans, bool unit, int64_t n, void *a,
                        int64_t lda, int leaf, int64_t batch, int64_t bstride) {
    const int64_t nleaves = (n + leaf - 1) / leaf;
    const double nb = (double)leaf;
    TraceScope ts(c.stream, dt == TRI_F64 ? "leaf_f64" : "leaf_f32",
                  (double)batch * nleaves * nb * nb * nb / 3.0,
                  (double)batch * 2.0 * (double)n * nb / 2.0 * (dt == TRI_F64 ? 8.0 : 4.0));
    if (dt == TRI_F64) return launch_leaf_dispatch<double>(c, trans, unit, n, (double *)a, lda, leaf, batch, bstride);
    return launch_leaf_dispatch<float>(c, trans, unit, n, (float *)a, lda, leaf, batch, bstride);
}

}  // namespace triinv
