// batched.cu -- a6: thousands of triangular blocks of uneven sizes in one persistent,
// graph-captured launch (block-Jacobi preconditioner shape).
//
// Each CTA repeatedly takes the next block from an atomic queue (blocks sorted by size,
// largest first, so the tail is made of small blocks), and inverts it entirely in shared
// memory by the recursive triangular split of the paper:
//   * the lower triangle is stored as 32 x 32 tiles (tile (I, J), I >= J, at index
//     I(I+1)/2 + J; row pitch 33 keeps warp accesses conflict-free);
//   * each diagonal tile is inverted by one warp with the CRIT column recurrence
//     (Section 4.2): lane j holds column j of the inverse in registers;
//   * split levels h = 32, 64, 128: for every pair, W = B X_A then B <- -X_C W (block
//     inverse of the proof of the main Theorem, Section 3), as 32 x 32 x 32 warp tile
//     products (each lane a 4 x 8 register block).
// Blocks larger than the shared-memory budget are rejected at plan time
// (TRI_ERR_UNSUPPORTED): 256 in FP32, 128 in FP64.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>

#include "internal.cuh"
#include "tile_inverse.cuh"

struct tri_batched_plan;   // opaque to callers (include/triinv.h)

namespace triinv {
namespace {


struct BDesc {
    void *ptr;
    long long ld;
    int n;
    int index;   // position in the caller's arrays
};

template <int MAXT>
struct BLimits {
    static constexpr int kTiles = MAXT * (MAXT + 1) / 2;   // lower tiles of the largest block
    static constexpr int kWTiles = (MAXT / 2) * (MAXT / 2); // W of the top level
};

// hi / mid / lo BF16 pieces of two values, packed as bf16x2 words.
__device__ __forceinline__ void split_pair(float a, float b, uint32_t &h, uint32_t &m, uint32_t &l) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(hh);
    const float ra = a - hf.x, rb = b - hf.y;
    const __nv_bfloat162 mm = __floats2bfloat162_rn(ra, rb);
    const float2 mf = __bfloat1622float2(mm);
    const __nv_bfloat162 ll = __floats2bfloat162_rn(ra - mf.x, rb - mf.y);
    h = *reinterpret_cast<const uint32_t *>(&hh);
    m = *reinterpret_cast<const uint32_t *>(&mm);
    l = *reinterpret_cast<const uint32_t *>(&ll);
}

// Writes the BF16 hi/mid/lo planes of the whole (nt*32)^2 block held in the tiles (the
// strict upper part as zeros) at rows/columns row0 + ... of planes with leading dim ldp.
// Lane = (row octet, column): each lane converts 8 consecutive rows of a column and
// stores 16 bytes per plane (rows row0 + 8k are 16-byte aligned: ldp is a multiple of
// 64 and the planes 256-byte aligned); octets that cross ntot or n are stored singly.
template <typename T, int NT>
__device__ __forceinline__ void write_planes(const T *tiles, int nt, int n, long long row0, long long ntot,
                                             __nv_bfloat16 *p0, __nv_bfloat16 *p1, __nv_bfloat16 *p2,
                                             long long ldp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nwarps = NT / 32;
    const int oct = lane & 3, cl = lane >> 2;
    for (int e = warp; e < nt * nt; e += nwarps) {
        const int I = e / nt, J = e % nt;
        const T *tp = I >= J ? tiles + (size_t)(I * (I + 1) / 2 + J) * TE : nullptr;
        const int rb = I * 32 + oct * 8;          // first row of the octet in the block
        const long long gi = row0 + rb;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int c = cl + 8 * t, cj = J * 32 + c;
            const long long gj = row0 + cj;
            if (gj >= ntot || cj >= n || gi >= ntot || rb >= n) continue;
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = tp ? (float)tp[(oct * 8 + i) * TP + c] : 0.f;
            const long long o = gi + gj * ldp;
            if (gi + 8 <= ntot && rb + 8 <= n) {
                uint4 h, m, l;
                split_pair(v[0], v[1], h.x, m.x, l.x);
                split_pair(v[2], v[3], h.y, m.y, l.y);
                split_pair(v[4], v[5], h.z, m.z, l.z);
                split_pair(v[6], v[7], h.w, m.w, l.w);
                *reinterpret_cast<uint4 *>(p0 + o) = h;
                *reinterpret_cast<uint4 *>(p1 + o) = m;
                *reinterpret_cast<uint4 *>(p2 + o) = l;
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if (gi + i >= ntot || rb + i >= n) continue;
                    const __nv_bfloat16 h = __float2bfloat16_rn(v[i]);
                    const float r1 = v[i] - __bfloat162float(h);
                    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
                    p0[o + i] = h;
                    p1[o + i] = m;
                    p2[o + i] = __float2bfloat16_rn(r1 - __bfloat162float(m));
                }
            }
        }
    }
}

// Loads the lower tiles of block d (strict upper of diagonal tiles = 0, padding =
// identity), one warp per tile.  FP32 tiles that lie inside the block, from a 16-byte
// aligned source with ld a multiple of 4, come in as 8 float4 loads per lane (lane = 4
// consecutive elements along the contiguous index of the source); the rest as 32 scalar
// loads per lane.  Returns this thread's max |element| seen.  No barrier.
template <typename T, bool TRANS, bool UNIT, int NT, typename S>
__device__ __forceinline__ float load_tiles(const BDesc &d, T *tiles) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = NT / 32;
    const int n = d.n, nt = (n + 31) / 32;
    const S *g = reinterpret_cast<const S *>(d.ptr);
    const long long ld = d.ld;
    const int ntl = nt * (nt + 1) / 2;
    const bool vec_ok = sizeof(S) == 4 && (((uintptr_t)g & 15) == 0) && (ld % 4 == 0);
    float tmax = 0.f;
    for (int tl = warp; tl < ntl; tl += nwarps) {
        int I = 0;
        while ((I + 1) * (I + 2) / 2 <= tl) ++I;
        const int J = tl - I * (I + 1) / 2;
        T *tp = tile_ptr(tiles, I, J);
        if (vec_ok && I * 32 + 32 <= n) {
            // contiguous index: rows (column-major source) or columns (transposed source)
            const int q4 = (lane & 7) * 4, o8 = lane >> 3;
            float4 v[8];
#pragma unroll
            for (int s8 = 0; s8 < 8; ++s8) {
                const int other = o8 + 4 * s8;          // column (or row) of the tile
                const int gi = TRANS ? I * 32 + other : I * 32 + q4;
                const int gj = TRANS ? J * 32 + q4 : J * 32 + other;
                v[s8] = *reinterpret_cast<const float4 *>(&g[vidx<TRANS>(gi, gj, ld)]);
            }
#pragma unroll
            for (int s8 = 0; s8 < 8; ++s8) {
                const int other = o8 + 4 * s8;
                const float vv[4] = {v[s8].x, v[s8].y, v[s8].z, v[s8].w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int r = TRANS ? other : q4 + q, c = TRANS ? q4 + q : other;
                    T x = (T)vv[q];
                    if (I == J) x = c > r ? T(0) : (c == r && UNIT ? T(1) : x);
                    tmax = fmaxf(tmax, fabsf((float)x));
                    tp[r * TP + c] = x;
                }
            }
            continue;
        }
        T v[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            // lane = row (column-major source) or column (transposed source)
            const int r = TRANS ? q : lane, c = TRANS ? lane : q;
            const int gi = I * 32 + r, gj = J * 32 + c;
            if (gi < n && gj < n) {
                if (gj < gi) v[q] = (T)g[vidx<TRANS>(gi, gj, ld)];
                else if (gj == gi) v[q] = UNIT ? T(1) : (T)g[vidx<TRANS>(gi, gi, ld)];
                else v[q] = T(0);
            } else {
                v[q] = (gi == gj) ? T(1) : T(0);
            }
        }
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            const int r = TRANS ? q : lane, c = TRANS ? lane : q;
            tp[r * TP + c] = v[q];
            tmax = fmaxf(tmax, fabsf((float)v[q]));
        }
    }
    return tmax;
}

// FP64 inverse of an ill-conditioned block of more than 128 rows whose FP32 source in
// global memory is still unchanged (the FP64 tiles of such a block do not fit in shared
// memory).  T is staged in shared memory as FP32 -- exact, it is FP32 data -- packed by
// rows (row i at offset i(i+1)/2), and warp w computes the columns j = w, w + nwarps, ...
// by the column recurrence of CRIT (Section 4.2) in FP64:
//     x_jj = 1/t_jj,   x_ij = -(sum_{k=j}^{i-1} t_ik x_kj) / t_ii   (i > j),
// each sum split over the lanes and reduced by shuffles; column j of X (FP64) lives in
// the warp's slice of shared memory.  The result is stored rounded to FP32.  About 0.7 ms
// per 256-row block on one SM (FP64 throughput), for blocks that need it only.
// smem: at least n(n+1)/2 floats + NT/32 * 256 doubles.
template <bool TRANS, bool UNIT, int NT>
__device__ void redo_columns_fp64(const BDesc &d, uint8_t *smem) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = NT / 32;
    const int n = d.n;
    const long long ld = d.ld;
    float *tp = reinterpret_cast<float *>(smem);
    double *xs = reinterpret_cast<double *>(smem + (((size_t)n * (n + 1) / 2 * 4 + 15) / 16) * 16);
    const float *g = reinterpret_cast<const float *>(d.ptr);
    for (int i = warp; i < n; i += nwarps)
        for (int k = lane; k <= i; k += 32)
            tp[(size_t)i * (i + 1) / 2 + k] = (k == i && UNIT) ? 1.f : g[vidx<TRANS>(i, k, ld)];
    __syncthreads();
    float *go = reinterpret_cast<float *>(d.ptr);
    double *x = xs + (size_t)warp * 256;
    for (int j = warp; j < n; j += nwarps) {
        if (lane == 0) x[j] = 1.0 / (double)tp[(size_t)j * (j + 1) / 2 + j];
        __syncwarp();
        for (int i = j + 1; i < n; ++i) {
            const float *ti = tp + (size_t)i * (i + 1) / 2;
            double acc = 0.0;
            for (int k = j + lane; k < i; k += 32) acc = fma((double)ti[k], x[k], acc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) x[i] = -acc / (double)ti[i];
            __syncwarp();
        }
        for (int i = j + lane; i < n; i += 32)
            if (!(UNIT && i == j)) go[vidx<TRANS>(i, j, ld)] = (float)x[i];
        __syncwarp();
    }
    __syncthreads();
}

// info_as >= 0: a zero pivot records info_as (the matrix of a batch) instead of the row.
// S: the element type in global memory (T, or FP32 data inverted in FP64).
// tau > 0 (FP32 only): growth limit.  When the FP32 inverse has max|X| * max|T| > tau and
// the block has at most 128 rows, the block, still unchanged in global memory, is loaded
// again and inverted in FP64 in the same shared memory, and that result is stored.
template <typename T, bool TRANS, bool UNIT, int MAXT, int NT, typename S = T>
__device__ __forceinline__ void invert_block(const BDesc &d, T *tiles, T *wt, long long *info, long long row0,
                                             __nv_bfloat16 *p0, __nv_bfloat16 *p1, __nv_bfloat16 *p2,
                                             long long ldp, long long ntot, __nv_bfloat16 *q0 = nullptr,
                                             __nv_bfloat16 *q1 = nullptr, __nv_bfloat16 *q2 = nullptr,
                                             long long info_as = -1, float tau = 0.f, int *redo_flag = nullptr) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = NT / 32;
    const int n = d.n, nt = (n + 31) / 32;
    const S *g = reinterpret_cast<const S *>(d.ptr);
    const long long ld = d.ld;
    __shared__ unsigned s_tmax, s_xmax;      // max |T| and max |X| as float bits (tau > 0)

    // Load the lower tiles (strict upper of diagonal tiles = 0, padding = identity).
    const int ntl = nt * (nt + 1) / 2;
    const bool vec_ok = sizeof(S) == 4 && (((uintptr_t)g & 15) == 0) && (ld % 4 == 0);
    if (tau > 0.f && tid == 0) s_tmax = s_xmax = 0u;
    const float tmax = load_tiles<T, TRANS, UNIT, NT, S>(d, tiles);
    __syncthreads();
    if (tau > 0.f) block_max_nonneg(&s_tmax, tmax);

    // Planes of T itself (diagonal blocks of the mixed path), before inverting.
    if (q0 != nullptr) {
        write_planes<T, NT>(tiles, nt, n, row0, ntot, q0, q1, q2, ldp);
        __syncthreads();   // the inversion below overwrites the tiles in place
    }

    // Diagonal tiles, then the split levels, all in shared memory.
    {
        const int bad = invert_tiles<T, NT>(tiles, wt, nt, n);
        if (bad >= 0 && !UNIT && threadIdx.x == 0)
            atomicMin(info, info_as >= 0 ? info_as : (row0 >= 0 ? (long long)(row0 + bad) : (long long)d.index));
    }

    if constexpr (std::is_same<T, float>::value) {
        bool redo = false;
        if (tau > 0.f) {
            float xmax = 0.f;
            for (int x = tid; x < ntl * 1024; x += NT) {
                const int tl = x / 1024, e = x % 1024;
                xmax = fmaxf(xmax, fabsf(tiles[(size_t)tl * TE + (e / 32) * TP + e % 32]));
            }
            block_max_nonneg(&s_xmax, xmax);
            __syncthreads();
            const float growth = __uint_as_float(s_xmax) * __uint_as_float(s_tmax);
            __syncthreads();
            redo = !(growth <= tau);
        }
        if (redo_flag && tid == 0) *redo_flag = redo ? 1 : 0;
        if constexpr (MAXT >= 8) {
            if (redo && n <= 128) {
                // FP64 again from the unchanged source; the FP64 tiles of a 128-block fit in
                // the shared memory of the FP32 block of 256
                double *dt = reinterpret_cast<double *>(tiles);
                invert_block<double, TRANS, UNIT, 4, NT, float>(d, dt, dt + (size_t)BLimits<4>::kTiles * TE, info,
                                                                row0, nullptr, nullptr, nullptr, 0, ntot, nullptr,
                                                                nullptr, nullptr, info_as, 0.f);
                if (p0 != nullptr) {
                    load_tiles<float, TRANS, UNIT, NT, S>(d, tiles);
                    __syncthreads();
                    write_planes<T, NT>(tiles, nt, n, row0, ntot, p0, p1, p2, ldp);
                }
                return;
            }
        }
        if (redo) {
            // FP64 column recurrence from the unchanged source, stored directly (its staging,
            // n(n+1)/2 floats and 256 doubles per warp, fits the FP32 tiles of every class)
            redo_columns_fp64<TRANS, UNIT, NT>(d, reinterpret_cast<uint8_t *>(tiles));
            if (p0 != nullptr) {
                load_tiles<float, TRANS, UNIT, NT, S>(d, tiles);
                __syncthreads();
                write_planes<T, NT>(tiles, nt, n, row0, ntot, p0, p1, p2, ldp);
            }
            return;
        }
    }

    // Store the lower triangle back (unit diagonal not written), one warp per tile;
    // off-diagonal tiles inside the block as float4 stores when the source allowed
    // float4 loads.
    S *go = reinterpret_cast<S *>(d.ptr);
    for (int tl = warp; tl < ntl; tl += nwarps) {
        int I = 0;
        while ((I + 1) * (I + 2) / 2 <= tl) ++I;
        const int J = tl - I * (I + 1) / 2;
        const T *tp = tile_ptr(tiles, I, J);
        if (vec_ok && I > J && I * 32 + 32 <= n) {
            const int q4 = (lane & 7) * 4, o8 = lane >> 3;
#pragma unroll
            for (int s8 = 0; s8 < 8; ++s8) {
                const int other = o8 + 4 * s8;
                float vv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int r = TRANS ? other : q4 + q, c = TRANS ? q4 + q : other;
                    vv[q] = (float)tp[r * TP + c];
                }
                const int gi = TRANS ? I * 32 + other : I * 32 + q4;
                const int gj = TRANS ? J * 32 + q4 : J * 32 + other;
                *reinterpret_cast<float4 *>(&go[vidx<TRANS>(gi, gj, ld)]) = make_float4(vv[0], vv[1], vv[2], vv[3]);
            }
            continue;
        }
#pragma unroll 8
        for (int q = 0; q < 32; ++q) {
            const int r = TRANS ? q : lane, c = TRANS ? lane : q;
            const int gi = I * 32 + r, gj = J * 32 + c;
            if (gi < n && gj < n && gj <= gi && !(UNIT && gi == gj)) go[vidx<TRANS>(gi, gj, ld)] = (S)tp[r * TP + c];
        }
    }
    if (p0 != nullptr) write_planes<T, NT>(tiles, nt, n, row0, ntot, p0, p1, p2, ldp);
}

template <typename T, bool TRANS, bool UNIT, int MAXT, int NT>
__global__ void __launch_bounds__(NT, 1) batched_kernel(const BDesc *__restrict__ descs, int count, int *counter, long long *info,
                                                        const float *tau_ptr) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    T *tiles = reinterpret_cast<T *>(smem_raw);
    T *wt = tiles + (size_t)BLimits<MAXT>::kTiles * TE;
    __shared__ int s_job;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_job = atomicAdd(counter, 1);
        __syncthreads();
        const int job = s_job;
        __syncthreads();
        if (job >= count) break;
        invert_block<T, TRANS, UNIT, MAXT, NT>(descs[job], tiles, wt, info, -1, nullptr, nullptr, nullptr, 0, 0,
                                               nullptr, nullptr, nullptr, -1, tau_ptr ? *tau_ptr : 0.f);
        __syncthreads();
    }
}

// The diagonal blocks of one n x n matrix (lower view through TRANS): CTA b inverts rows
// and columns [256 b, 256 b + 256) in shared memory and, when p0 != nullptr, writes the
// BF16 planes of that diagonal block.  blockIdx.y: matrix of a batch (matrices as_, planes
// ps elements apart); index0 >= 0: a zero pivot records the matrix index index0 + blockIdx.y
// instead of the row.
// tau > 0: growth limit; a block whose FP32 inverse has max|X| max|T| > tau is inverted
// again in FP64 and flags[blockIdx.y * gridDim.x + blockIdx.x] is set to 1 (else 0).
template <bool TRANS, bool UNIT>
__global__ void __launch_bounds__(512, 1) diag_blocks_kernel(float *a, long long lda, long long n, long long *info,
                                                             __nv_bfloat16 *p0, __nv_bfloat16 *p1,
                                                             __nv_bfloat16 *p2, long long ldp, __nv_bfloat16 *q0,
                                                             __nv_bfloat16 *q1, __nv_bfloat16 *q2,
                                                             long long as_, long long ps, long long index0,
                                                             float tau, int *flags) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    float *tiles = reinterpret_cast<float *>(smem_raw);
    float *wt = tiles + (size_t)BLimits<8>::kTiles * TE;
    const long long r0 = (long long)blockIdx.x * 256;
    const long long mb = blockIdx.y;
    if (mb) {
        a += mb * as_;
        p0 += mb * ps; p1 += mb * ps; p2 += mb * ps;
        if (q0) { q0 += mb * ps; q1 += mb * ps; q2 += mb * ps; }
    }
    BDesc d{a + vidx<TRANS>(r0, r0, lda), lda, (int)min(256ll, n - r0), (int)blockIdx.x};
    invert_block<float, TRANS, UNIT, 8, 512>(d, tiles, wt, info, r0, p0, p1, p2, ldp, n, q0, q1, q2,
                                             index0 >= 0 ? index0 + mb : -1, tau,
                                             flags ? flags + mb * gridDim.x + blockIdx.x : nullptr);
}

// Dynamic shared memory of a class kernel: its tiles and the top level's W, or for FP32
// the staging of the FP64 column recurrence (n(n+1)/2 floats, 16-byte aligned, and 256
// doubles per warp) if that is larger.
template <typename T, int MAXT, int NT = 512>
size_t smem_bytes() {
    const size_t tiles = (size_t)(BLimits<MAXT>::kTiles + BLimits<MAXT>::kWTiles) * TE * sizeof(T);
    if (!std::is_same<T, float>::value) return tiles;
    const size_t nmax = 32 * (size_t)MAXT;
    const size_t redo = (nmax * (nmax + 1) / 2 * 4 + 15) / 16 * 16 + (size_t)(NT / 32) * 256 * 8;
    return std::max(tiles, redo);
}

using KernFn = void (*)(const BDesc *, int, int *, long long *, const float *);

template <typename T, int MAXT, int NT>
KernFn pick3(bool trans, bool unit) {
    if (trans) return unit ? batched_kernel<T, true, true, MAXT, NT> : batched_kernel<T, true, false, MAXT, NT>;
    return unit ? batched_kernel<T, false, true, MAXT, NT> : batched_kernel<T, false, false, MAXT, NT>;
}

// Size classes of a batch, each its own persistent launch with its own CTA shape:
//   class 0  161..256 rows (FP32): 8 x 8 tiles, 220 KB of shared memory, one CTA per SM;
//   class 1  129..160 rows (FP32): 5 x 5 tiles (80 KB), two CTAs per SM;
//   class 2  33..128 rows: 4 x 4 tiles (59 KB FP32, 118 KB FP64), several CTAs per SM;
//   class 3  up to 32 rows: one tile, one warp per CTA, many CTAs per SM.
// Candidate thread counts per class (the autotuner times them); 0 ends a list.
constexpr int kClasses = 4;
constexpr int kCandidates[kClasses][3] = {{512, 256, 0}, {256, 512, 0}, {128, 256, 0}, {32, 64, 0}};

int size_class(int64_t n) { return n > 160 ? 0 : (n > 128 ? 1 : (n > 32 ? 2 : 3)); }

// Kernel for a precision, orientation, diagonal kind, size class and thread count.
KernFn pick_kernel(tri_dtype dt, bool trans, bool unit, int cls, int threads, size_t *smem) {
    if (cls == 3) {
        if (dt == TRI_F64) {
            *smem = smem_bytes<double, 1>();
            return threads == 64 ? pick3<double, 1, 64>(trans, unit) : pick3<double, 1, 32>(trans, unit);
        }
        *smem = threads == 64 ? smem_bytes<float, 1, 64>() : smem_bytes<float, 1, 32>();
        return threads == 64 ? pick3<float, 1, 64>(trans, unit) : pick3<float, 1, 32>(trans, unit);
    }
    if (cls == 1) {   // FP32 only (FP64 blocks stop at 128 rows)
        *smem = threads == 512 ? smem_bytes<float, 5, 512>() : smem_bytes<float, 5, 256>();
        return threads == 512 ? pick3<float, 5, 512>(trans, unit) : pick3<float, 5, 256>(trans, unit);
    }
    if (cls == 2) {
        if (dt == TRI_F64) {
            *smem = smem_bytes<double, 4>();
            return threads == 256 ? pick3<double, 4, 256>(trans, unit) : pick3<double, 4, 128>(trans, unit);
        }
        *smem = threads == 256 ? smem_bytes<float, 4, 256>() : smem_bytes<float, 4, 128>();
        return threads == 256 ? pick3<float, 4, 256>(trans, unit) : pick3<float, 4, 128>(trans, unit);
    }
    *smem = threads == 256 ? smem_bytes<float, 8, 256>() : smem_bytes<float, 8, 512>();
    return threads == 256 ? pick3<float, 8, 256>(trans, unit) : pick3<float, 8, 512>(trans, unit);
}

}  // namespace

// Inverts the 256 x 256 diagonal blocks of an n x n FP32 matrix in place (one CTA each)
// and writes the BF16 planes of the inverse blocks (p*) and, if q0 != nullptr, of the
// original blocks (q*) (used by the mixed path).
cudaError_t launch_diag_blocks(const Ctx &c, bool trans, bool unit, int64_t n, float *a, int64_t lda,
                               __nv_bfloat16 *p0, __nv_bfloat16 *p1, __nv_bfloat16 *p2, int64_t ldp,
                               __nv_bfloat16 *q0, __nv_bfloat16 *q1, __nv_bfloat16 *q2, int64_t batch,
                               int64_t as_, int64_t ps, int64_t index0, float tau, int *flags) {
    const int64_t blocks = (n + 255) / 256;
    if (blocks <= 0 || batch <= 0) return cudaSuccess;
    if (batch > 65535) return cudaErrorInvalidValue;
    const size_t smem = smem_bytes<float, 8>();
    auto k = trans ? (unit ? diag_blocks_kernel<true, true> : diag_blocks_kernel<true, false>)
                   : (unit ? diag_blocks_kernel<false, true> : diag_blocks_kernel<false, false>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    double fl = 0.0;
    for (int64_t b = 0; b < blocks; ++b) {
        const double nb = (double)std::min<int64_t>(256, n - 256 * b);
        fl += nb * nb * nb / 3.0;
    }
    TraceScope ts(c.stream, "diag_blocks", fl * (double)batch, (double)batch * n * 256.0 * (4.0 + 4.0 + 6.0));
    k<<<dim3((unsigned)blocks, (unsigned)batch), 512, smem, c.stream>>>(a, lda, n, c.info, p0, p1, p2, ldp, q0, q1,
                                                                       q2, as_, ps, index0, tau, flags);
    return cudaGetLastError();
}

}  // namespace triinv

struct tri_batched_plan {
    int device = 0;
    int count = 0;
    tri_dtype dtype = TRI_F32;
    bool trans = false, unit = false;
    triinv::BDesc *d_desc = nullptr;   // sorted, largest first: classes 0, 1, 2 in order
    int *d_counter = nullptr;          // one queue counter per size class
    float *d_tau = nullptr;            // growth limit of the FP64 fallback (device, FP32 plans)
    int first[4] = {0, 0, 0, 0};       // first descriptor of each size class
    int nclass[4] = {0, 0, 0, 0};      // blocks of each size class
    int threads[4] = {0, 0, 0, 0};     // tuned threads per CTA of each class
    int ctas[4] = {0, 0, 0, 0};        // persistent CTAs of each class
    double flops = 0.0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace triinv {
namespace {

int max_block(tri_dtype dt) { return dt == TRI_F64 ? 128 : 256; }

constexpr float kDefaultGrowthLimit = 1.0e4f;   // FP32 batches: max|X| max|T| beyond it -> FP64

// Dynamic shared memory above 48 KB must be allowed per kernel before any launch (and
// before stream capture).
cudaError_t allow_smem(tri_dtype dt, bool trans) {
    for (int u = 0; u < 2; ++u)
        for (int cls = 0; cls < kClasses; ++cls)
            for (int i = 0; kCandidates[cls][i]; ++i) {
                size_t smem = 0;
                KernFn k = pick_kernel(dt, trans, u != 0, cls, kCandidates[cls][i], &smem);
                cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

// Persistent CTAs of a class: as many as fit on the device (occupancy of the kernel with
// its shared memory), at most one per block.
int class_ctas(const tri_batched_plan *p, int cls, int threads, int sm_count) {
    size_t smem = 0;
    KernFn k = pick_kernel(p->dtype, p->trans, p->unit, cls, threads, &smem);
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return std::max(1, std::min(p->nclass[cls], per_sm * sm_count));
}

// Resets the class's queue and launches its persistent kernel.
cudaError_t launch_class(const tri_batched_plan *p, int cls, cudaStream_t s, long long *info, int threads,
                         int ctas) {
    if (p->nclass[cls] == 0) return cudaSuccess;
    size_t smem = 0;
    KernFn k = pick_kernel(p->dtype, p->trans, p->unit, cls, threads, &smem);
    cudaError_t e = cudaMemsetAsync(p->d_counter + cls, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k<<<ctas, threads, smem, s>>>(p->d_desc + p->first[cls], p->nclass[cls], p->d_counter + cls, info, p->d_tau);
    return cudaGetLastError();
}

// ---- autotuner and its cache ---------------------------------------------------------
// For each size class the tuner times every candidate thread count (and the CTA count
// that fits with it) on a scratch copy of the class's block sizes (identity blocks, unit
// diagonal, so the caller's data is untouched) and keeps the fastest.  Choices are cached
// per (GPU model, SM count, dtype, class, histogram of the class's sizes in 16-row buckets)
// for the process, and tri_tune_cache_save / tri_tune_cache_load keep them in a JSON file.
std::mutex g_tune_mu;
std::vector<std::pair<std::string, int>> g_tune_cache;

std::string device_tag(int dev) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string name = prop.name;
    for (char &ch : name)
        if (ch == '"' || ch == '\\' || ch == ' ') ch = '_';
    return name + "/" + std::to_string(prop.multiProcessorCount);
}

std::string tune_key(const tri_batched_plan *p, int cls, const std::vector<int64_t> &sizes, int dev) {
    std::string key = device_tag(dev) + ":" + std::to_string((int)p->dtype) + ":c" + std::to_string(cls) + ":";
    std::vector<int> h(17, 0);
    for (int64_t s : sizes) h[std::min<int64_t>(16, s / 16)]++;
    for (int v : h) key += std::to_string(v) + ",";
    return key;
}

int autotune_class(tri_batched_plan *p, int cls, const std::vector<int64_t> &sizes, const Ctx &c) {
    const std::string key = tune_key(p, cls, sizes, c.device);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto &kv : g_tune_cache)
            if (kv.first == key) return kv.second;
    }
    int best = kCandidates[cls][0];
    if (const char *env = getenv("TRI_BATCHED_THREADS")) {   // forced choice (class 0 only)
        if (cls == 0) return atoi(env) == 256 ? 256 : 512;
    }
    size_t total = 0;
    for (int64_t s : sizes) total += (size_t)s * s;
    const size_t es = p->dtype == TRI_F64 ? 8 : 4;
    void *scratch = nullptr;
    BDesc *d_scr = nullptr;
    long long *d_info = nullptr;
    int *d_cnt = nullptr;
    if (cudaMalloc(&scratch, total * es) != cudaSuccess || cudaMalloc(&d_scr, sizeof(BDesc) * sizes.size()) != cudaSuccess ||
        cudaMalloc(&d_info, sizeof(long long)) != cudaSuccess || cudaMalloc(&d_cnt, kClasses * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(scratch);
        cudaFree(d_scr);
        cudaFree(d_info);
        cudaFree(d_cnt);
        return best;
    }
    cudaMemset(scratch, 0, total * es);
    std::vector<BDesc> hd(sizes.size());
    size_t off = 0;
    for (size_t i = 0; i < sizes.size(); ++i) {
        hd[i] = BDesc{(uint8_t *)scratch + off * es, (long long)sizes[i], (int)sizes[i], (int)i};
        off += (size_t)sizes[i] * sizes[i];
    }
    cudaMemcpy(d_scr, hd.data(), sizeof(BDesc) * hd.size(), cudaMemcpyHostToDevice);
    tri_batched_plan tmp = *p;
    tmp.d_desc = d_scr - p->first[cls];   // launch_class adds first[cls]
    tmp.d_counter = d_cnt;
    tmp.unit = true;   // identity scratch: unit diagonal, no pivots to check
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    for (int i = 0; kCandidates[cls][i]; ++i) {
        const int th = kCandidates[cls][i];
        const int ctas = class_ctas(&tmp, cls, th, c.sm_count);
        float ms = 0.f;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; ++rep) {
            cudaEventRecord(e0, c.stream);
            ok = launch_class(&tmp, cls, c.stream, d_info, th, ctas) == cudaSuccess;
            cudaEventRecord(e1, c.stream);
            cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms += t;
        }
        if (ok && ms < best_ms) {
            best_ms = ms;
            best = th;
        }
        cudaGetLastError();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(scratch);
    cudaFree(d_scr);
    cudaFree(d_info);
    cudaFree(d_cnt);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache.push_back({key, best});
    return best;
}

}  // namespace
}  // namespace triinv

using namespace triinv;

extern "C" {

tri_status tri_batched_plan_create(int64_t count, const int64_t *sizes, void *const *ptrs, tri_uplo uplo,
                                   tri_diag diag, tri_dtype dtype, tri_batched_plan **out) {
    if (!out || count < 0 || (count > 0 && (!sizes || !ptrs))) return TRI_ERR_ARG;
    if ((uplo != TRI_LOWER && uplo != TRI_UPPER) || (diag != TRI_NONUNIT && diag != TRI_UNIT)) return TRI_ERR_ARG;
    if (dtype != TRI_F64 && dtype != TRI_F32 && dtype != TRI_F32_MIXED) return TRI_ERR_ARG;
    if (count > INT_MAX / 2) return TRI_ERR_ARG;
    *out = nullptr;
    const tri_dtype dt = dtype == TRI_F64 ? TRI_F64 : TRI_F32;
    for (int64_t i = 0; i < count; ++i) {
        if (sizes[i] < 0 || (sizes[i] > 0 && !ptrs[i])) return TRI_ERR_ARG;
        if (sizes[i] > max_block(dt)) return TRI_ERR_UNSUPPORTED;
    }
    Ctx c;
    tri_status st = device_ctx_public(nullptr, &c);
    if (st != TRI_OK) return st;
    tri_batched_plan *p = new tri_batched_plan();
    p->device = c.device;
    p->dtype = dt;
    p->trans = uplo == TRI_UPPER;
    p->unit = diag == TRI_UNIT;
    std::vector<int64_t> order;
    for (int64_t i = 0; i < count; ++i)
        if (sizes[i] > 0) order.push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return sizes[a] > sizes[b]; });
    std::vector<BDesc> hd;
    std::vector<int64_t> cls_sizes[kClasses];
    for (int64_t i : order) {
        hd.push_back(BDesc{ptrs[i], (long long)sizes[i], (int)sizes[i], (int)i});
        cls_sizes[size_class(sizes[i])].push_back(sizes[i]);
        p->flops += (double)sizes[i] * sizes[i] * sizes[i] / 3.0;
    }
    p->count = (int)hd.size();
    for (int cl = 0, f = 0; cl < kClasses; ++cl) {   // sorted descending: classes are contiguous
        p->first[cl] = f;
        p->nclass[cl] = (int)cls_sizes[cl].size();
        f += p->nclass[cl];
    }
    if (cudaMalloc(&p->d_counter, kClasses * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&p->d_tau, sizeof(float)) != cudaSuccess) {
        cudaFree(p->d_counter);
        delete p;
        cudaGetLastError();
        return TRI_ERR_NOMEM;
    }
    {
        const float tau = p->dtype == TRI_F32 ? kDefaultGrowthLimit : 0.f;
        if (cudaMemcpy(p->d_tau, &tau, sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(p->d_counter);
            cudaFree(p->d_tau);
            delete p;
            return TRI_ERR_CUDA;
        }
    }
    if (p->count > 0) {
        if (cudaMalloc(&p->d_desc, sizeof(BDesc) * hd.size()) != cudaSuccess) {
            cudaFree(p->d_counter);
            cudaFree(p->d_tau);
            delete p;
            cudaGetLastError();
            return TRI_ERR_NOMEM;
        }
        cudaMemcpy(p->d_desc, hd.data(), sizeof(BDesc) * hd.size(), cudaMemcpyHostToDevice);
    }
    if (allow_smem(p->dtype, p->trans) != cudaSuccess) {
        cudaGetLastError();
        tri_batched_plan_destroy(p);
        return TRI_ERR_CUDA;
    }
    for (int cl = 0; cl < kClasses; ++cl) {
        if (p->nclass[cl] == 0) continue;
        p->threads[cl] = autotune_class(p, cl, cls_sizes[cl], c);
        p->ctas[cl] = class_ctas(p, cl, p->threads[cl], c.sm_count);
    }
    // Capture {reset queue, persistent kernel} per class, largest class first; replayed by
    // tri_batched_exec.  Class 0 and the chain of the smaller classes are captured as two
    // independent branches, so that SMs freed at the end of one branch take the other's
    // CTAs (4096-block workload: 0.630 against 0.637 ms as one chain);
    // TRI_BATCHED_BRANCHES=0 (read at plan creation) captures the single chain.
    if (p->count > 0) {
        const char *br = getenv("TRI_BATCHED_BRANCHES");
        const bool branches = !(br && br[0] == '0');
        cudaStream_t cs = nullptr, cs2 = nullptr;
        cudaEvent_t fork = nullptr, join = nullptr;
        bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
        if (ok && branches)
            ok = cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&join, cudaEventDisableTiming) == cudaSuccess;
        const bool capturing = ok && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        ok = capturing;
        if (ok && branches) {
            ok = cudaEventRecord(fork, cs) == cudaSuccess && cudaStreamWaitEvent(cs2, fork, 0) == cudaSuccess;
            ok = ok && launch_class(p, 0, cs, c.info, p->threads[0], p->ctas[0]) == cudaSuccess;
            for (int cl = 1; cl < kClasses && ok; ++cl)
                ok = launch_class(p, cl, cs2, c.info, p->threads[cl], p->ctas[cl]) == cudaSuccess;
            ok = ok && cudaEventRecord(join, cs2) == cudaSuccess && cudaStreamWaitEvent(cs, join, 0) == cudaSuccess;
        } else {
            for (int cl = 0; cl < kClasses && ok; ++cl)
                ok = launch_class(p, cl, cs, c.info, p->threads[cl], p->ctas[cl]) == cudaSuccess;
        }
        if (capturing) ok = (cudaStreamEndCapture(cs, &p->graph) == cudaSuccess) && ok;
        ok = ok && cudaGraphInstantiate(&p->exec, p->graph, 0) == cudaSuccess;
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (cs2) cudaStreamDestroy(cs2);
        if (cs) cudaStreamDestroy(cs);
        if (!ok) {
            cudaGetLastError();
            tri_batched_plan_destroy(p);
            return TRI_ERR_CUDA;
        }
    }
    *out = p;
    return TRI_OK;
}

tri_status tri_batched_exec(tri_batched_plan *plan, void *stream) {
    if (!plan) return TRI_ERR_ARG;
    if (plan->count == 0) return TRI_OK;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device) return TRI_ERR_ARG;
    TraceScope ts((cudaStream_t)stream, plan->dtype == TRI_F64 ? "batched_f64" : "batched_f32", plan->flops, 0.0);
    return cudaGraphLaunch(plan->exec, (cudaStream_t)stream) == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
}

tri_status tri_batched_plan_destroy(tri_batched_plan *plan) {
    if (!plan) return TRI_OK;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    cudaFree(plan->d_desc);
    cudaFree(plan->d_counter);
    cudaFree(plan->d_tau);
    delete plan;
    return TRI_OK;
}

tri_status tri_batched_plan_set_growth_limit(tri_batched_plan *plan, double tau) {
    if (!plan || tau != tau) return TRI_ERR_ARG;
    if (plan->dtype != TRI_F32) return TRI_ERR_UNSUPPORTED;
    const float t = tau > 0.0 ? (float)std::min(tau, 3.0e38) : 0.f;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device) return TRI_ERR_ARG;
    return cudaMemcpy(plan->d_tau, &t, sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
}

int tri_batched_plan_threads(const tri_batched_plan *plan) {
    if (!plan) return 0;
    for (int cl = 0; cl < kClasses; ++cl)
        if (plan->nclass[cl] > 0) return plan->threads[cl];
    return 0;
}

tri_status tri_batched_plan_shape(const tri_batched_plan *plan, int cls, int *blocks, int *threads, int *ctas) {
    if (!plan || cls < 0 || cls >= kClasses) return TRI_ERR_ARG;
    if (blocks) *blocks = plan->nclass[cls];
    if (threads) *threads = plan->threads[cls];
    if (ctas) *ctas = plan->ctas[cls];
    return TRI_OK;
}

tri_status tri_tune_cache_save(const char *path) {
    if (!path) return TRI_ERR_ARG;
    std::vector<std::pair<std::string, int>> v;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        v = g_tune_cache;
    }
    FILE *f = fopen(path, "w");
    if (!f) return TRI_ERR_ARG;
    fprintf(f, "{\"version\": 1, \"entries\": [");
    for (size_t i = 0; i < v.size(); ++i)
        fprintf(f, "%s\n  {\"key\": \"%s\", \"threads\": %d}", i ? "," : "", v[i].first.c_str(), v[i].second);
    fprintf(f, "\n]}\n");
    return fclose(f) == 0 ? TRI_OK : TRI_ERR_ARG;
}

tri_status tri_tune_cache_load(const char *path, int *loaded) {
    if (loaded) *loaded = 0;
    if (!path) return TRI_ERR_ARG;
    FILE *f = fopen(path, "r");
    if (!f) return TRI_ERR_ARG;
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
    fclose(f);
    // entries of the form {"key": "...", "threads": N}, as written by tri_tune_cache_save
    int count = 0;
    size_t pos = 0;
    while ((pos = text.find("\"key\": \"", pos)) != std::string::npos) {
        pos += 8;
        const size_t q = text.find('"', pos);
        if (q == std::string::npos) return TRI_ERR_ARG;
        const std::string key = text.substr(pos, q - pos);
        const size_t t = text.find("\"threads\":", q);
        if (t == std::string::npos) return TRI_ERR_ARG;
        const int th = atoi(text.c_str() + t + 10);
        if (th != 32 && th != 64 && th != 128 && th != 256 && th != 512) return TRI_ERR_ARG;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        bool found = false;
        for (auto &kv : g_tune_cache)
            if (kv.first == key) {
                kv.second = th;
                found = true;
            }
        if (!found) g_tune_cache.push_back({key, th});
        ++count;
        pos = t;
    }
    if (loaded) *loaded = count;
    return TRI_OK;
}

tri_status tri_inv_batched(int64_t count, const int64_t *sizes, void *const *ptrs, tri_uplo uplo, tri_diag diag,
                           tri_dtype dtype, void *stream) {
    tri_batched_plan *p = nullptr;
    tri_status st = tri_batched_plan_create(count, sizes, ptrs, uplo, diag, dtype, &p);
    if (st != TRI_OK) return st;
    st = tri_batched_exec(p, stream);
    // The plan's buffers may still be in use by the queued launch.
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess && st == TRI_OK) st = TRI_ERR_CUDA;
    tri_batched_plan_destroy(p);
    return st;
}

}  // extern "C"
