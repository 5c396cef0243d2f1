// split.cu -- K4: FP32 -> BF16 planes for the mixed-precision path.
//
// A value v (FP32) is written as three BF16 pieces v = hi + mid + lo with
//   hi = RN(v), mid = RN(v - hi), lo = RN(v - hi - mid),
// every subtraction exact in FP32, so hi + mid + lo reproduces v for normal values.
// The tensor-core products take 3 (or 6) pairs of these pieces.
//
// Planes are column-major n x n with leading dimension ldp and hold the LOWER view of
// the matrix.  Only blocks that the products read are written: the lower triangle and
// the 256 x 256 diagonal blocks (whose strict upper part is written as zero, since a
// product tile that straddles the diagonal reads it).
#include <cuda_bf16.h>

#include "internal.cuh"

namespace triinv {
namespace {

constexpr int TS = 32;   // transpose tile

__device__ __forceinline__ void split3(float v, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
    h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// One 32x32 tile (ti, tj) per CTA (blockIdx.x = ti, blockIdx.y = tj), 32x8 threads.
// DIAG_ONLY: only tiles inside the diagonal 256-blocks are processed.
template <bool TRANS, bool UNIT, bool DIAG_ONLY>
__global__ void __launch_bounds__(256) split_kernel(const float *__restrict__ a, int64_t lda, int64_t n,
                                                    __nv_bfloat16 *__restrict__ p0,
                                                    __nv_bfloat16 *__restrict__ p1,
                                                    __nv_bfloat16 *__restrict__ p2, int64_t ldp) {
    const int64_t i0 = (int64_t)blockIdx.x * TS;   // rows
    const int64_t j0 = (int64_t)blockIdx.y * TS;   // cols
    if (i0 >= n || j0 >= n) return;
    const bool diag_block = (i0 / 256) == (j0 / 256);
    if (DIAG_ONLY && !diag_block) return;
    if (!diag_block && j0 > i0) return;            // strictly upper block: never read
    __shared__ float tile[TS][TS + 1];             // tile[i - i0][j - j0]
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    // Load (only the referenced triangle; the rest reads as 0, a unit diagonal as 1).
    for (int r = ty; r < TS; r += 8) {
        int64_t i, j;
        if (TRANS) { i = i0 + r; j = j0 + tx; }    // contiguous along j
        else { i = i0 + tx; j = j0 + r; }          // contiguous along i
        float v = 0.f;
        if (i < n && j < n) {
            if (j < i) v = a[vidx<TRANS>(i, j, lda)];
            else if (j == i) v = UNIT ? 1.f : a[vidx<TRANS>(i, i, lda)];
        }
        if (TRANS) tile[r][tx] = v;
        else tile[tx][r] = v;
    }
    __syncthreads();
    for (int r = ty; r < TS; r += 8) {
        const int64_t i = i0 + tx, j = j0 + r;
        if (i >= n || j >= n) continue;
        __nv_bfloat16 h, m, l;
        split3(tile[tx][r], h, m, l);
        const int64_t o = i + j * ldp;
        p0[o] = h;
        p1[o] = m;
        p2[o] = l;
    }
}

}  // namespace

cudaError_t launch_split_planes(const Ctx &c, bool trans, bool unit, bool diag_only, int64_t n,
                                const float *a, int64_t lda, __nv_bfloat16 *p0, __nv_bfloat16 *p1,
                                __nv_bfloat16 *p2, int64_t ldp) {
    const int64_t t = (n + TS - 1) / TS;
    if (t <= 0) return cudaSuccess;
    dim3 grid((unsigned)t, (unsigned)t);
    const double elems = diag_only ? (double)n * 256.0 : (double)n * n / 2.0;
    TraceScope ts(c.stream, diag_only ? "split_diag" : "split_t", 0.0, elems * (4.0 + 6.0));
#define TRI_SPLIT(TR, UN, DO) split_kernel<TR, UN, DO><<<grid, 256, 0, c.stream>>>(a, lda, n, p0, p1, p2, ldp)
    if (diag_only) {
        if (trans) { if (unit) TRI_SPLIT(true, true, true); else TRI_SPLIT(true, false, true); }
        else { if (unit) TRI_SPLIT(false, true, true); else TRI_SPLIT(false, false, true); }
    } else {
        if (trans) { if (unit) TRI_SPLIT(true, true, false); else TRI_SPLIT(true, false, false); }
        else { if (unit) TRI_SPLIT(false, true, false); else TRI_SPLIT(false, false, false); }
    }
#undef TRI_SPLIT
    return cudaGetLastError();
}

}  // namespace triinv
