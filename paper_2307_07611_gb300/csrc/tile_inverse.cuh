// tile_inverse.cuh -- in-shared-memory inverse of a lower-triangular block stored as
// 32 x 32 tiles (the batched kernel, the diagonal blocks of the mixed path and the LU
// leaves of the general inverse).
//
// Tile (I, J), I >= J, of the lower triangle lives at index I(I+1)/2 + J with row pitch
// TP = 33 (conflict-free warp access).  The inverse follows the paper's recursive split:
//   * each diagonal tile is inverted by one warp with the CRIT column recurrence
//     (Section 4.2): lane j holds column j of the inverse in registers;
//   * split levels h = 32, 64, 128: for every pair, W = B X_A then B <- -X_C W (block
//     inverse of the proof of the main Theorem, Section 3), as 32 x 32 x 32 warp tile
//     products (each lane a 4 x 8 register block).
#pragma once

#include <cuda_runtime.h>

namespace triinv {

constexpr int TP = 33;   // tile row pitch (elements)
constexpr int TE = 32 * TP;

// Maximum of v over the warp's lanes (every lane gets it).
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// *m = max(*m, v) over a CTA for non-negative v (float bits order like the values): one
// shared-memory atomic per warp (all lanes of the warp must take part).
__device__ __forceinline__ void block_max_nonneg(unsigned *m, float v) {
    v = warp_max(v);
    if ((threadIdx.x & 31) == 0) atomicMax(m, __float_as_uint(v));
}

template <typename T>
__device__ __forceinline__ T *tile_ptr(T *tiles, int I, int J) {
    return tiles + (size_t)(I * (I + 1) / 2 + J) * TE;
}

// Warp tile product: acc[4][8] += A (32x32) * B (32x32), lane = (row group, col group).
template <typename T>
__device__ __forceinline__ void warp_mma32(const T *A, const T *B, T (&acc)[4][8], int lane) {
    const int r0 = (lane >> 2) * 4, c0 = (lane & 3) * 8;
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
        T a[4], b[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = A[(r0 + i) * TP + k];
#pragma unroll
        for (int j = 0; j < 8; ++j) b[j] = B[k * TP + c0 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
}

template <typename T>
__device__ __forceinline__ void warp_store32(T *C, const T (&acc)[4][8], int lane, T scale) {
    const int r0 = (lane >> 2) * 4, c0 = (lane & 3) * 8;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) C[(r0 + i) * TP + c0 + j] = scale * acc[i][j];
}

// In-place inverse of a lower 32 x 32 tile by one warp (column recurrence; lane j owns
// column j).  Returns the first row (< valid) whose pivot is zero or non-finite, or 32.
template <typename T>
__device__ __forceinline__ int warp_tile_inverse(T *t, int lane, int valid) {
    T x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] = T(0);
    int bad = 32;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const T tkk = t[k * TP + k];
        if (k < valid && bad == 32 && (tkk == T(0) || !isfinite(tkk))) bad = k;
        const T dk = T(1) / tkk;
        // row k of the inverse becomes final
        if (lane == k) x[k] = dk;
        else if (lane < k) x[k] = -x[k] * dk;
        // pending rows: x_ij += t_ik x_kj  (lanes j > k hold x_kj = 0)
#pragma unroll
        for (int i = k + 1; i < 32; ++i) x[i] = fma(t[i * TP + k], x[k], x[i]);
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 32; ++i) t[i * TP + lane] = (i >= lane) ? x[i] : T(0);
    __syncwarp();
    return bad;
}

// Inverts one block held in global memory (column-major view, order d.n <= 32 * MAXT) in
// shared memory and writes the lower triangle back.  row0 >= 0: the block is the
// diagonal block starting at row row0 of a larger matrix (pivot errors report the row,
// and the BF16 hi/mid/lo planes of the whole block are written when p0 != nullptr);
// row0 < 0: a block of a batch (pivot errors report d.index).
// Inverts the nt x nt lower tiles in place (W scratch `wt`: (nt/2)^2 tiles), with all
// NT threads of the block.  n: order of the valid part (rows >= n are identity padding).
// Returns the first row < n with a zero or non-finite pivot, or -1.  Ends with a barrier.
template <typename T, int NT>
__device__ __forceinline__ int invert_tiles(T *tiles, T *wt, int nt, int n) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = NT / 32;
    __shared__ int s_bad;
    if (tid == 0) s_bad = 1 << 30;
    __syncthreads();
    for (int I = warp; I < nt; I += nwarps) {
        const int bad = warp_tile_inverse(tile_ptr(tiles, I, I), lane, min(32, n - I * 32));
        if (bad < 32 && lane == 0) atomicMin(&s_bad, I * 32 + bad);
    }
    __syncthreads();
    // Split levels (in tiles): ht = 1, 2, 4.
    for (int ht = 1; ht < nt; ht *= 2) {
        const int pairs = (nt - ht + 2 * ht - 1) / (2 * ht);
        // W_q(Iw, Jw) = sum_{K >= Jw} B(c0 + Iw, a0 + K) X(a0 + K, a0 + Jw)
        int jobs = 0;
        for (int q = 0; q < pairs; ++q) jobs += min(ht, nt - (2 * q * ht + ht)) * ht;
        // Job order within a pair is column-major (Jw outer): a W tile's length ht - Jw
        // depends on its column, and warps w, w + 4, ... share one SM sub-partition, so
        // consecutive warps take tiles of different lengths.  The tile is stored at
        // base + Iw * ht + Jw, where the X21 phase reads it.
        for (int jb = warp; jb < jobs; jb += nwarps) {
            int q = 0, rest = jb, base = 0, hc = 0;
            for (;;) {
                hc = min(ht, nt - (2 * q * ht + ht));
                if (rest < hc * ht) break;
                rest -= hc * ht;
                base += hc * ht;
                ++q;
            }
            const int a0 = 2 * q * ht, c0 = a0 + ht;
            const int Jw = rest / hc, Iw = rest % hc;
            T acc[4][8];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = T(0);
            for (int K = Jw; K < ht; ++K)
                warp_mma32(tile_ptr(tiles, c0 + Iw, a0 + K), tile_ptr(tiles, a0 + K, a0 + Jw), acc, lane);
            warp_store32(wt + (size_t)(base + Iw * ht + Jw) * TE, acc, lane, T(1));
        }
        __syncthreads();
        // B(c0 + Iw, a0 + Jw) <- -sum_{K <= Iw} X_C(c0 + Iw, c0 + K) W_q(K, Jw)
        for (int jb = warp; jb < jobs; jb += nwarps) {
            int q = 0, rest = jb, base = 0;
            for (;;) {
                const int hc = min(ht, nt - (2 * q * ht + ht));
                if (rest < hc * ht) break;
                rest -= hc * ht;
                base += hc * ht;
                ++q;
            }
            const int a0 = 2 * q * ht, c0 = a0 + ht;
            const int Iw = rest / ht, Jw = rest % ht;
            T acc[4][8];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = T(0);
            for (int K = 0; K <= Iw; ++K)
                warp_mma32(tile_ptr(tiles, c0 + Iw, c0 + K), wt + (size_t)(base + K * ht + Jw) * TE, acc, lane);
            warp_store32(tile_ptr(tiles, c0 + Iw, a0 + Jw), acc, lane, T(-1));
        }
        __syncthreads();
    }

    const int r = s_bad;
    __syncthreads();
    return r < (1 << 30) ? r : -1;
}

// invert_tiles for NM independent lower blocks at once (same order nt x nt tiles, same
// valid order n): every stage's warp jobs of all blocks are spread over the NT / 32 warps,
// so small blocks keep more warps busy.  tiles[x] / wt[x]: block x and its W scratch.
// Pivot errors are not reported (the callers check their pivots before).  Ends with a
// barrier.
// p[x] without a dynamically indexed array (which would live in local memory).
template <typename T, int NM>
__device__ __forceinline__ T *pick(T *const (&p)[NM], int x) {
    T *r = p[0];
#pragma unroll
    for (int i = 1; i < NM; ++i) r = (x == i) ? p[i] : r;
    return r;
}

template <typename T, int NT, int NM>
__device__ __forceinline__ void invert_tiles_multi(T *const (&tiles)[NM], T *const (&wt)[NM], int nt, int n) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = NT / 32;
    for (int x = warp; x < NM * nt; x += nwarps) {
        const int mtx = x / nt, I = x % nt;
        warp_tile_inverse(tile_ptr(pick(tiles, mtx), I, I), lane, min(32, n - I * 32));
    }
    __syncthreads();
    for (int ht = 1; ht < nt; ht *= 2) {
        const int pairs = (nt - ht + 2 * ht - 1) / (2 * ht);
        int jobs = 0;
        for (int q = 0; q < pairs; ++q) jobs += min(ht, nt - (2 * q * ht + ht)) * ht;
        for (int x = warp; x < NM * jobs; x += nwarps) {
            const int mtx = x / jobs, jb = x % jobs;
            T *tl = pick(tiles, mtx);
            int q = 0, rest = jb, base = 0, hc = 0;
            for (;;) {
                hc = min(ht, nt - (2 * q * ht + ht));
                if (rest < hc * ht) break;
                rest -= hc * ht;
                base += hc * ht;
                ++q;
            }
            const int a0 = 2 * q * ht, c0 = a0 + ht;
            const int Jw = rest / hc, Iw = rest % hc;   // column-major, as in invert_tiles
            T acc[4][8];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = T(0);
            for (int K = Jw; K < ht; ++K)
                warp_mma32(tile_ptr(tl, c0 + Iw, a0 + K), tile_ptr(tl, a0 + K, a0 + Jw), acc, lane);
            warp_store32(pick(wt, mtx) + (size_t)(base + Iw * ht + Jw) * TE, acc, lane, T(1));
        }
        __syncthreads();
        for (int x = warp; x < NM * jobs; x += nwarps) {
            const int mtx = x / jobs, jb = x % jobs;
            T *tl = pick(tiles, mtx);
            int q = 0, rest = jb, base = 0;
            for (;;) {
                const int hc = min(ht, nt - (2 * q * ht + ht));
                if (rest < hc * ht) break;
                rest -= hc * ht;
                base += hc * ht;
                ++q;
            }
            const int a0 = 2 * q * ht, c0 = a0 + ht;
            const int Iw = rest / ht, Jw = rest % ht;
            T acc[4][8];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = T(0);
            for (int K = 0; K <= Iw; ++K)
                warp_mma32(tile_ptr(tl, c0 + Iw, c0 + K), pick(wt, mtx) + (size_t)(base + K * ht + Jw) * TE, acc, lane);
            warp_store32(tile_ptr(tl, c0 + Iw, a0 + Jw), acc, lane, T(-1));
        }
        __syncthreads();
    }
}

}  // namespace triinv
