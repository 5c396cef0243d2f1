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

constexpr int TS = 64;   // tile edge; 256 threads, each thread two rows of a column at a time

__device__ __forceinline__ void split3(float v, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
    h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// One 64 x 64 tile per CTA.  DIAG_ONLY: blockIdx.z is the diagonal 256-block and
// (blockIdx.x, blockIdx.y) the tile inside it; otherwise (blockIdx.x, blockIdx.y) is the
// tile of the whole matrix, blockIdx.z the matrix of a batch (source as_ and planes ps
// elements apart), and tiles that no product reads return at once, as do tiles outside
// the split levels lmin .. lmax: an off-diagonal 256-block (I, J) is the B block of split
// half-size 256 * 2^l with l the highest set bit of I XOR J (diagonal blocks: level 0).
// Thread t owns rows (2*(t%32), 2*(t%32)+1) of the tile and columns t/32 + 8*c, so a warp
// stores 64 consecutive rows (128 bytes per plane) per column.
template <bool TRANS, bool UNIT, bool DIAG_ONLY>
__global__ void __launch_bounds__(256) split_kernel(const float *__restrict__ a, int64_t lda, int64_t n,
                                                    __nv_bfloat16 *__restrict__ p0,
                                                    __nv_bfloat16 *__restrict__ p1,
                                                    __nv_bfloat16 *__restrict__ p2, int64_t ldp,
                                                    bool skip_diag, int64_t as_, int64_t ps, int lmin,
                                                    int lmax) {
    int64_t i0, j0;
    if (!DIAG_ONLY && blockIdx.z) {
        a += (int64_t)blockIdx.z * as_;
        p0 += (int64_t)blockIdx.z * ps;
        p1 += (int64_t)blockIdx.z * ps;
        p2 += (int64_t)blockIdx.z * ps;
    }
    if (DIAG_ONLY) {
        i0 = (int64_t)blockIdx.z * 256 + blockIdx.x * TS;
        j0 = (int64_t)blockIdx.z * 256 + blockIdx.y * TS;
    } else {
        i0 = (int64_t)blockIdx.x * TS;
        j0 = (int64_t)blockIdx.y * TS;
        const bool diag_block = (i0 / 256) == (j0 / 256);
        if (!diag_block && j0 > i0) return;        // strictly upper block: never read
        if (diag_block && skip_diag) return;       // written by the diagonal-block kernel
        const int lv = diag_block ? 0 : 31 - __clz((unsigned)((i0 / 256) ^ (j0 / 256)));
        if (lv < lmin || lv > lmax) return;
    }
    if (i0 >= n || j0 >= n) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // Off-diagonal 64 x 64 tile inside the matrix, column-major source with 16-byte rows:
    // thread t converts rows i0 + 8 (t % 8) .. + 7 of columns j0 + t / 8 and j0 + 32 + t / 8
    // (two float4 loads, one 16-byte store per plane); a warp covers 4 whole columns.
    if (!TRANS && !DIAG_ONLY && (i0 / 256) != (j0 / 256) && i0 + TS <= n && j0 + TS <= n &&
        (((uintptr_t)a & 15) == 0) && (lda % 4) == 0 && (ldp % 8) == 0) {
        const int t = threadIdx.x, r8 = (t & 7) * 8;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int64_t j = j0 + (t >> 3) + 32 * cc, i = i0 + r8;
            const float4 u = *reinterpret_cast<const float4 *>(a + i + j * lda);
            const float4 v = *reinterpret_cast<const float4 *>(a + i + 4 + j * lda);
            const float x[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
            uint32_t hw[4], mw[4], lw[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                __nv_bfloat16 h0, m0, l0, h1, m1, l1;
                split3(x[2 * e], h0, m0, l0);
                split3(x[2 * e + 1], h1, m1, l1);
                const __nv_bfloat162 hp = __halves2bfloat162(h0, h1), mp = __halves2bfloat162(m0, m1),
                                     lp = __halves2bfloat162(l0, l1);
                hw[e] = *reinterpret_cast<const uint32_t *>(&hp);
                mw[e] = *reinterpret_cast<const uint32_t *>(&mp);
                lw[e] = *reinterpret_cast<const uint32_t *>(&lp);
            }
            const int64_t o = i + j * ldp;
            *reinterpret_cast<uint4 *>(p0 + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4 *>(p1 + o) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
            *reinterpret_cast<uint4 *>(p2 + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        return;
    }
    // Referenced triangle only; the rest reads as 0 and a unit diagonal as 1.
    auto fetch = [&](int64_t i, int64_t j) -> float {
        if (i >= n || j >= n || j > i) return 0.f;
        if (j == i) return UNIT ? 1.f : a[vidx<TRANS>(i, i, lda)];
        return a[vidx<TRANS>(i, j, lda)];
    };
    if (TRANS) {
        // The source is contiguous along j: stage the tile through shared memory.
        __shared__ float tile[TS][TS + 1];         // tile[i - i0][j - j0]
        for (int e = threadIdx.x; e < TS * TS; e += 256) {
            const int ii = e / TS, jj = e % TS;
            tile[ii][jj] = fetch(i0 + ii, j0 + jj);
        }
        __syncthreads();
        for (int c = w; c < TS; c += 8) {
            const int64_t j = j0 + c;
            const int64_t i = i0 + 2 * lane;
            if (j >= n || i >= n) continue;
            __nv_bfloat16 h0, m0, l0, h1, m1, l1;
            split3(tile[2 * lane][c], h0, m0, l0);
            split3(tile[2 * lane + 1][c], h1, m1, l1);
            const int64_t o = i + j * ldp;
            if (i + 1 < n && !(o & 1)) {
                *(__nv_bfloat162 *)(p0 + o) = __halves2bfloat162(h0, h1);
                *(__nv_bfloat162 *)(p1 + o) = __halves2bfloat162(m0, m1);
                *(__nv_bfloat162 *)(p2 + o) = __halves2bfloat162(l0, l1);
            } else {
                p0[o] = h0; p1[o] = m0; p2[o] = l0;
                if (i + 1 < n) { p0[o + 1] = h1; p1[o + 1] = m1; p2[o + 1] = l1; }
            }
        }
    } else {
        for (int c = w; c < TS; c += 8) {
            const int64_t j = j0 + c;
            const int64_t i = i0 + 2 * lane;
            if (j >= n || i >= n) continue;
            __nv_bfloat16 h0, m0, l0, h1, m1, l1;
            split3(fetch(i, j), h0, m0, l0);
            split3(fetch(i + 1, j), h1, m1, l1);
            const int64_t o = i + j * ldp;
            if (i + 1 < n && !(o & 1)) {
                *(__nv_bfloat162 *)(p0 + o) = __halves2bfloat162(h0, h1);
                *(__nv_bfloat162 *)(p1 + o) = __halves2bfloat162(m0, m1);
                *(__nv_bfloat162 *)(p2 + o) = __halves2bfloat162(l0, l1);
            } else {
                p0[o] = h0; p1[o] = m0; p2[o] = l0;
                if (i + 1 < n) { p0[o + 1] = h1; p1[o + 1] = m1; p2[o + 1] = l1; }
            }
        }
    }
}

// Rectangle rows x cols (column-major, lds) -> planes, with the triangle kind of the
// operand applied (0 outside the stored triangle, 1 on an implicit unit diagonal).
// Thread t owns rows 2*(t%32), 2*(t%32)+1 of a 64-row strip; blockIdx.y = 8-column group;
// blockIdx.z = matrix of a batch (source as_ and planes ps elements apart).
template <bool TR>
__global__ void __launch_bounds__(256) split_rect_kernel(const float *__restrict__ a, int64_t lds,
                                                         int64_t rows, int64_t cols, int kind,
                                                         __nv_bfloat16 *__restrict__ p0,
                                                         __nv_bfloat16 *__restrict__ p1,
                                                         __nv_bfloat16 *__restrict__ p2, int64_t ldp,
                                                         int64_t as_, int64_t ps) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (blockIdx.z) {
        a += (int64_t)blockIdx.z * as_;
        p0 += (int64_t)blockIdx.z * ps;
        p1 += (int64_t)blockIdx.z * ps;
        if (p2) p2 += (int64_t)blockIdx.z * ps;
    }
    const int64_t i = (int64_t)blockIdx.x * 64 + 2 * lane;
    const int64_t j = (int64_t)blockIdx.y * 8 + w;
    if (i >= rows || j >= cols) return;
    // element (r, j) of op(src): src itself, or its transpose (TR)
    auto at = [&](int64_t r) -> float { return TR ? a[j + r * lds] : a[r + j * lds]; };
    auto fetch = [&](int64_t r) -> float {
        if (r >= rows) return 0.f;
        switch (kind) {
            case 1: return j <= r ? at(r) : 0.f;                        // lower
            case 2: return j >= r ? at(r) : 0.f;                        // upper
            case 3: return j < r ? at(r) : (j == r ? 1.f : 0.f);        // lower, unit
            case 4: return j > r ? at(r) : (j == r ? 1.f : 0.f);        // upper, unit
            default: return at(r);
        }
    };
    __nv_bfloat16 h0, m0, l0, h1, m1, l1;
    split3(fetch(i), h0, m0, l0);
    split3(fetch(i + 1), h1, m1, l1);
    const int64_t o = i + j * ldp;
    if (i + 1 < rows && !(o & 1)) {
        *(__nv_bfloat162 *)(p0 + o) = __halves2bfloat162(h0, h1);
        *(__nv_bfloat162 *)(p1 + o) = __halves2bfloat162(m0, m1);
        if (p2) *(__nv_bfloat162 *)(p2 + o) = __halves2bfloat162(l0, l1);
    } else {
        p0[o] = h0; p1[o] = m0;
        if (p2) p2[o] = l0;
        if (i + 1 < rows) {
            p0[o + 1] = h1; p1[o + 1] = m1;
            if (p2) p2[o + 1] = l1;
        }
    }
}

}  // namespace

cudaError_t launch_split_rect(const Ctx &c, const float *a, int64_t lds, int64_t rows, int64_t cols,
                              int kind, __nv_bfloat16 *p0, __nv_bfloat16 *p1, __nv_bfloat16 *p2,
                              int64_t ldp, bool trans, int64_t batch, int64_t as_, int64_t ps) {
    if (rows <= 0 || cols <= 0 || batch <= 0) return cudaSuccess;
    if (batch > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((rows + 63) / 64), (unsigned)((cols + 7) / 8), (unsigned)batch);
    TraceScope ts(c.stream, "split_rect", 0.0, (double)batch * rows * cols * (4.0 + (p2 ? 6.0 : 4.0)));
    if (trans) split_rect_kernel<true><<<grid, 256, 0, c.stream>>>(a, lds, rows, cols, kind, p0, p1, p2, ldp, as_, ps);
    else split_rect_kernel<false><<<grid, 256, 0, c.stream>>>(a, lds, rows, cols, kind, p0, p1, p2, ldp, as_, ps);
    return cudaGetLastError();
}

cudaError_t launch_split_planes(const Ctx &c, bool trans, bool unit, bool diag_only, int64_t n,
                                const float *a, int64_t lda, __nv_bfloat16 *p0, __nv_bfloat16 *p1,
                                __nv_bfloat16 *p2, int64_t ldp, bool skip_diag, int64_t batch,
                                int64_t as_, int64_t ps, int lmin, int lmax) {
    const int64_t t = (n + TS - 1) / TS;
    if (t <= 0 || batch <= 0) return cudaSuccess;
    if (batch > 65535 || (diag_only && batch > 1)) return cudaErrorInvalidValue;
    dim3 grid = diag_only ? dim3(256 / TS, 256 / TS, (unsigned)((n + 255) / 256))
                          : dim3((unsigned)t, (unsigned)t, (unsigned)batch);
    const double elems = (diag_only ? (double)n * 256.0 : (double)n * n / 2.0) * (double)batch;
    TraceScope ts(c.stream, diag_only ? "split_diag" : "split_t", 0.0, elems * (4.0 + 6.0));
#define TRI_SPLIT(TR, UN, DO) \
    split_kernel<TR, UN, DO><<<grid, 256, 0, c.stream>>>(a, lda, n, p0, p1, p2, ldp, skip_diag, as_, ps, lmin, lmax)
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
