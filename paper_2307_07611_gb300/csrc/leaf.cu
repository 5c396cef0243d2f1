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
// Rounding: 1/t_ii is one IEEE round-to-nearest division, so the diagonal of X is
// exactly RN(1/t_ii); off-diagonal entries use fused multiply-adds and a multiplication
// by that reciprocal (the paper's "appropriate diagonal matrix multiplication", Section
// 2), which differs from a division by t_ii by at most one rounding.
#include <climits>

#include "internal.cuh"

namespace triinv {
namespace {

template <typename T, int LEAF, int NT, bool TRANS, bool UNIT>
__global__ void __launch_bounds__(NT) leaf_kernel(T *__restrict__ a, int64_t lda, int64_t n,
                                                  long long *__restrict__ info, int64_t bstride) {
    static_assert(NT % LEAF == 0 && (LEAF * LEAF) % NT == 0, "thread layout");
    constexpr int G = NT / LEAF;          // row groups
    constexpr int RPT = LEAF * LEAF / NT; // rows per thread
    __shared__ T ts[LEAF][LEAF + 1];
    __shared__ T dinv[LEAF];
    __shared__ T xrow[2][LEAF];

    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * LEAF;
    a += (int64_t)blockIdx.y * bstride;          // matrix of a strided batch
    const int nb = (int)((n - r0) < (int64_t)LEAF ? (n - r0) : (int64_t)LEAF);

    // Load the lower triangle of the leaf (the strict upper part and the padding become
    // zero, the padded diagonal one).  The contiguous index runs fastest across threads.
    for (int idx = tid; idx < LEAF * LEAF; idx += NT) {
        int i, k;
        if (TRANS) { i = idx / LEAF; k = idx % LEAF; }
        else { i = idx % LEAF; k = idx / LEAF; }
        T v = T(0);
        if (i < nb && k < nb) {
            if (k < i) v = a[vidx<TRANS>(r0 + i, r0 + k, lda)];
            else if (k == i) v = UNIT ? T(1) : a[vidx<TRANS>(r0 + i, r0 + i, lda)];
        } else if (i == k) {
            v = T(1);
        }
        ts[i][k] = v;
    }
    __syncthreads();
    if (tid < LEAF) {
        T d = ts[tid][tid];
        if (tid < nb && (d == T(0) || !isfinite(d)))
            atomicMin(info, gridDim.y > 1 ? (long long)blockIdx.y : (long long)(r0 + tid));
        dinv[tid] = T(1) / d;
    }
    __syncthreads();

    const int j = tid % LEAF;
    const int ig = tid / LEAF;
    T acc[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) acc[r] = T(0);

    for (int k = 0; k < nb; ++k) {
        const T dk = dinv[k];
        // Row k becomes final: x_kk = 1/t_kk, x_kj = -acc_kj / t_kk (j < k).
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int i = ig + r * G;
            if (i == k && j <= k) {
                const T x = (j == k) ? dk : -acc[r] * dk;
                acc[r] = x;
                xrow[k & 1][j] = x;
            }
        }
        __syncthreads();
        if (j <= k) {
            const T xkj = xrow[k & 1][j];
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int i = ig + r * G;
                if (i > k) acc[r] = fma(ts[i][k], xkj, acc[r]);
            }
        }
    }
    __syncthreads();
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
    constexpr int NT = LEAF >= 32 ? 256 : 128;
    const int64_t blocks = (n + LEAF - 1) / LEAF;
    if (blocks <= 0 || batch <= 0) return cudaSuccess;
    dim3 grid((unsigned)blocks, (unsigned)batch);
    if (trans) {
        if (unit) leaf_kernel<T, LEAF, NT, true, true><<<grid, NT, 0, c.stream>>>(a, lda, n, c.info, bstride);
        else leaf_kernel<T, LEAF, NT, true, false><<<grid, NT, 0, c.stream>>>(a, lda, n, c.info, bstride);
    } else {
        if (unit) leaf_kernel<T, LEAF, NT, false, true><<<grid, NT, 0, c.stream>>>(a, lda, n, c.info, bstride);
        else leaf_kernel<T, LEAF, NT, false, false><<<grid, NT, 0, c.stream>>>(a, lda, n, c.info, bstride);
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
