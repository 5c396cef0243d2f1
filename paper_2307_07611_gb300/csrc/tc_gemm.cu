// tc_gemm.cu -- K3: split-BF16 products on the 5th-generation tensor cores (tcgen05).
//
// Computes, per output tile, acc = sum_t A_t * B_t with BF16 operands and an FP32
// accumulator in tensor memory, where the A_t / B_t are BF16 "planes" of FP32 matrices
// (x = hi + mid + lo, each piece rounded to BF16).  It serves every dense product of the
// mixed-precision path:
//   level products of the split (block inverse, proof of the main Theorem, Section 3):
//       W = B X_A (3 terms)  and  X21 = -X_C W (3 terms);
//   the Newton-Schulz step X <- X + X (I - T X): R = I - T X (6 terms), X += X R (1 term).
//
// Structure (one CTA per SM, persistent over a host-built tile list, longest first):
//   warp 0      TMA producer: fills a ring of pipeline stages (geometry per mode, see
//               cfg_for): per (k-block, term) an A tile 128 x 64 (two 64 x 64 boxes,
//               MN-major) + a B tile 256 x 64 (K-major), or for R = I - T X per 32-wide
//               k-step all three A and three B plane tiles at once.
//   warp 1      allocates 512 TMEM columns (two 128x256 FP32 accumulators), one lane
//               issues tcgen05.mma (M=128, N=256, K=16) and commits slots / accumulators.
//   warps 2..9  epilogue: tcgen05.ld of the accumulator (two warps per 32-lane quarter,
//               128 columns each), split / update / store, then release the accumulator.
// The epilogue of tile i overlaps the main loop of tile i+1 (double-buffered TMEM).
// Every mbarrier wait is bounded (globaltimer); on timeout the kernel records the status,
// drains its in-flight copies and products, frees TMEM and returns.
//
// Operand layouts in shared memory (canonical tcgen05 layouts):
//   A (MN-major, 128-byte swizzle): atom = 64 M-elements (128 B) x 8 K-rows; the two
//                 64-row atoms ks * 128 B apart (LBO), K atoms 1024 B apart (SBO).  One MMA
//                 (K = 16) spans two K atoms (2048 B).
//   B (K-major, 128- or 64-byte swizzle for ks = 64 / 32): atom = 8 N-rows x ks
//                 K-elements; N atoms ks * 16 B apart (SBO); the k-offset inside the row
//                 advances the start address by 32 B per K = 16.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "tc_ptx.cuh"

namespace triinv {
namespace tc {
namespace {

struct Maps {
    CUtensorMap a[3];
    CUtensorMap b[3];
};

// Stores NC accumulator columns gn0..gn0+NC-1 of row gm (one thread = one row).
// Column-major targets advance by one leading dimension per column, so the 32 threads of
// a warp (32 consecutive rows) write contiguous bytes for every column.
// zero (MODE_RES): write R = 0 (the matrix skips its Newton-Schulz step).
template <int MODE, bool TRANS, bool UNIT, int NC>
__device__ __forceinline__ void epilogue_cols(const Epi &ep, int64_t xb, int64_t ob, int64_t gm, int64_t gn0,
                                              const uint32_t (&r)[NC], bool zero = false) {
    if (gm >= ep.mlim) return;
    const int64_t left = ep.nlim - gn0;
    // the six-term level products store exactly like their three-term forms
    constexpr bool W = MODE == MODE_W || MODE == MODE_W6, X21 = MODE == MODE_X21 || MODE == MODE_X216;
    if (W || X21 || MODE == MODE_RES) {
        int64_t off = ob + gm + gn0 * ep.ldo;
        int64_t xo = xb + vidx<TRANS>(gm, gn0, ep.ldx);
        const int64_t xstep = TRANS ? 1 : ep.ldx;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            if (j < left) {
                const float acc = __uint_as_float(r[j]);
                float v = acc;
                if (X21) {
                    v = -acc;
                    ep.x[xo] = v;
                } else if (MODE == MODE_RES) {
                    const int64_t gn = gn0 + j;
                    v = (gm >= gn && !zero) ? ((gm == gn ? 1.f : 0.f) - acc) : 0.f;
                }
                const __nv_bfloat16 h = __float2bfloat16_rn(v);
                const float r1 = v - __bfloat162float(h);
                const __nv_bfloat16 m = __float2bfloat16_rn(r1);
                ep.o0[off] = h;
                if (MODE != MODE_RES || ep.o1) ep.o1[off] = m;
                if (X21 || MODE == MODE_W6) ep.o2[off] = __float2bfloat16_rn(r1 - __bfloat162float(m));
            }
            off += ep.ldo;
            xo += xstep;
        }
    } else if (MODE == MODE_UPD) {
        int64_t xo = xb + vidx<TRANS>(gm, gn0, ep.ldx);
        const int64_t xstep = TRANS ? 1 : ep.ldx;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const int64_t gn = gn0 + j;
            if (j < left && (gm > gn || (!UNIT && gm == gn))) ep.x[xo] += __uint_as_float(r[j]);
            xo += xstep;
        }
    } else if (MODE == MODE_GEN || MODE == MODE_GENP) {
        int64_t xo = xb + gm + gn0 * ep.ldx;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const int64_t gn = gn0 + j;
            const bool low = ep.cmask == 1 || ep.cmask == 3, up = ep.cmask == 2 || ep.cmask == 4;
            const bool keep = j < left && !(low && gn > gm) && !(up && gm > gn);
            if (keep) {
                float v = ep.alpha * __uint_as_float(r[j]);
                if (gm == gn) v += ep.dadd;
                if (ep.cmask >= 3 && gm == gn) ep.x[xo] = 0.f;     // strict triangle: zero diagonal
                else ep.x[xo] = ep.beta == 0.f ? v : fmaf(ep.beta, ep.x[xo], v);
            }
            xo += ep.ldx;
        }
    } else {
        int64_t xo = xb + gm + gn0 * ep.ldx;
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            if (j < left) ep.x[xo] = __uint_as_float(r[j]);
            xo += ep.ldx;
        }
    }
}

// X values of row gm, columns gn0..gn0+15, that the update touches (lower triangle,
// and the diagonal unless unit); others read as 0 and are not stored.
template <bool TRANS, bool UNIT>
__device__ __forceinline__ void load_x16(const Epi &ep, int64_t xb, int64_t gm, int64_t gn0, float (&xv)[16]) {
    int64_t xo = xb + vidx<TRANS>(gm, gn0, ep.ldx);
    const int64_t xstep = TRANS ? 1 : ep.ldx;
    const bool row_ok = gm < ep.mlim;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int64_t gn = gn0 + j;
        xv[j] = (row_ok && gn < ep.nlim && (gm > gn || (!UNIT && gm == gn))) ? ep.x[xo] : 0.f;
        xo += xstep;
    }
}

template <bool TRANS, bool UNIT>
__device__ __forceinline__ void store_upd16(const Epi &ep, int64_t xb, int64_t gm, int64_t gn0,
                                            const float (&xv)[16], const uint32_t (&r)[16]) {
    if (gm >= ep.mlim) return;
    int64_t xo = xb + vidx<TRANS>(gm, gn0, ep.ldx);
    const int64_t xstep = TRANS ? 1 : ep.ldx;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int64_t gn = gn0 + j;
        if (gn < ep.nlim && (gm > gn || (!UNIT && gm == gn))) ep.x[xo] = xv[j] + __uint_as_float(r[j]);
        xo += xstep;
    }
}

// Pipeline geometry per mode.
//   ks       k per stage: 64 (B tiles 256 x 64 with 128-byte swizzle) or 32 (256 x 32,
//            64-byte swizzle).  A tiles are 128 x ks, two 64-row boxes with 128-byte swizzle.
//   fused    true: a stage holds every distinct plane tile the terms read and the MMA
//            issuer runs all terms on it (each plane crosses L2 once per k-step); false:
//            a stage holds the A / B pair of one term (loop: chunk, term, k).
//   promote  MODE_RES, MODE_GENP: 64-wide k-blocks accumulated in tensor memory before
//            the epilogue adds them into FP32 registers.  The accumulator truncates every
//            add, so a product added after the large hi*hi term loses up to one unit in
//            the last place of the partial sum; the chunk length bounds that loss.
// R = I - T X and the general six-term products read 3 + 3 planes: fused 32-wide stages
// (72 KB, 3 deep) halve their L2 traffic; one-term and three-term products keep 64-wide
// per-term stages (48 KB, 4 deep), which measured faster for them.
struct Cfg {
    int ks;
    bool fused;
    int promote;
};
__host__ __device__ constexpr Cfg cfg_for(int mode) {
    return (mode == MODE_RES || mode == MODE_GENP || mode == MODE_W6 || mode == MODE_X216) ? Cfg{32, true, 1}
                                                                                         : Cfg{64, false, 0};
}

constexpr int STAGE_BUDGET = 216 * 1024;
constexpr int MAX_STAGES = 9;
constexpr int GEMM_SMEM_BYTES = STAGE_BUDGET + 1024 + 512;

// Stage layout of one launch (host-computed from the terms and the mode's geometry).
struct Pipe {
    int na, nb;          // A / B tiles per stage
    int stages;          // ring depth
    int stage_bytes;     // na * BM * ks * 2 + nb * BN * ks * 2
    int batched;         // maps are 3-D (batch outermost): loads take the tile's matrix
};

// BNT: columns of an output tile (UMMA N = 256, 128 or 64).  Narrower tiles give the
// small products of the low split levels more, shorter tiles (more SMs busy, a shorter
// longest tile); the widest tile moves the fewest operand bytes per flop.
template <int MODE, bool TRANS, bool UNIT, int BNT>
__global__ void __launch_bounds__(NTHREADS, 1)
tc_gemm_kernel(const __grid_constant__ Maps maps, const Terms terms, const Pipe pipe,
               const Tile *__restrict__ tiles, const int *__restrict__ cta_off, const Epi ep,
               int *gtimeout) {
    constexpr bool PROMOTE = (MODE == MODE_RES || MODE == MODE_GENP || MODE == MODE_W6 || MODE == MODE_X216);
    constexpr Cfg CF = cfg_for(MODE);
    constexpr int KS = CF.ks;
    constexpr int A_TILE = BM * KS * 2, B_TILE = BNT * KS * 2;
    constexpr uint32_t IDESC = idesc_for(BNT);
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int STAGES = pipe.stages;
    const uint32_t stage_bytes = (uint32_t)pipe.stage_bytes;
    uint64_t *bars = (uint64_t *)(smem + STAGE_BUDGET);
    // bars: full[MAX_STAGES], empty[MAX_STAGES], tfull[2], tempty[2], drain
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * MAX_STAGES + 5);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (MAX_STAGES + s); };
    auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * MAX_STAGES + a); };
    auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * MAX_STAGES + 2 + a); };
    const uint32_t drain_bar = bar0 + 8u * (2 * MAX_STAGES + 4);
    // 64-wide k-blocks per accumulation chunk: one chunk per tile unless promoting.
    auto chunk_blocks = [&](const Tile &tl) { return PROMOTE ? CF.promote : (tl.kb1 - tl.kb0); };
    // One stage: load A tiles ia[0..na) and B tiles ib[0..nb) at k.
    auto load_stage = [&](uint32_t st, uint32_t bar, const Tile &tl, int k, int ia0, int ib0, int na, int nb) {
        mbar_arrive_expect_tx(bar, (uint32_t)(na * A_TILE + nb * B_TILE));
        for (int i = 0; i < na; ++i) {
            const uint32_t dst = st + (uint32_t)(i * A_TILE);
#pragma unroll
            for (int c = 0; c < BM / 64; ++c) {
                if (pipe.batched)
                    tma_load_3d(dst + (uint32_t)(c * KS * 128), &maps.a[ia0 + i], tl.am + 64 * c, tl.ak + k, tl.b, bar);
                else
                    tma_load_2d(dst + (uint32_t)(c * KS * 128), &maps.a[ia0 + i], tl.am + 64 * c, tl.ak + k, bar);
            }
        }
        for (int i = 0; i < nb; ++i) {
            const uint32_t dst = st + (uint32_t)(na * A_TILE + i * B_TILE);
            if (pipe.batched) tma_load_3d(dst, &maps.b[ib0 + i], tl.bk + k, tl.bn, tl.b, bar);
            else tma_load_2d(dst, &maps.b[ib0 + i], tl.bk + k, tl.bn, bar);
        }
    };
    // MMAs of one term on stage tiles sa / sb (KS / 16 steps of K = 16).
    auto mma_term = [&](uint32_t d, uint32_t sa, uint32_t sb, uint32_t &accumulate) {
#pragma unroll
        for (int kk = 0; kk < KS / 16; ++kk) {
            // A: MN-major, 64-row chunks KS * 128 B apart (LBO), 8-row k groups 1024 B
            // apart (SBO); a k-step of 16 = 2048 B.  B: K-major, 8-row groups KS * 16 B
            // apart; a k-step of 16 = 32 B inside the swizzled row.
            const uint64_t da = smem_desc(sa + kk * 2048, KS * 128, 1024, kSwizzle128);
            const uint64_t db = smem_desc(sb + kk * 32, 16, KS * 16, KS == 64 ? kSwizzle128 : kSwizzle64);
            tc_mma(d, da, db, IDESC, accumulate);
            accumulate = 1;
        }
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull_bar(a), 1);
            mbar_init(tempty_bar(a), EPI_WARPS);
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        for (int i = 0; i < 3; ++i) {
            prefetch_map(&maps.a[i]);
            prefetch_map(&maps.b[i]);
        }
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int t_begin = cta_off[blockIdx.x], t_end = cta_off[blockIdx.x + 1];   // plan data: constant
    // Programmatic dependent launch: the set-up above may overlap the previous kernel on
    // the stream; no global data it produces (or reads) is touched before this wait.  The
    // trigger lets the next kernel's CTAs start their own set-up as SMs free up; it can
    // only take effect once every CTA of this grid has started.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (threadIdx.x == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            // Ring position kept incrementally (slot, phase, address): no division by the
            // runtime ring depth in the issue loop.
            uint32_t it = 0, ph = 0, st = smem_u32(smem);
            int s = 0;
            bool ok = true;
            for (int t = t_begin; t < t_end && ok; ++t) {
                const Tile tl = tiles[t];
                const int cb = chunk_blocks(tl);
                for (int c0 = tl.kb0; c0 < tl.kb1 && ok; c0 += cb) {
                    const int c1 = min(c0 + cb, tl.kb1);
                    // fused: one pass with every plane; else one pass per term (smallest first)
                    for (int j = CF.fused ? 0 : terms.n - 1; j >= 0 && ok; --j) {
                        for (int kb = c0; kb < c1 && ok; ++kb) {
                            for (int hk = 0; hk < BK / KS; ++hk) {
                                if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, gtimeout)) {
                                    ok = false;
                                    break;
                                }
                                const int k = kb * BK + hk * KS;
                                if (CF.fused) load_stage(st, full_bar(s), tl, k, 0, 0, pipe.na, pipe.nb);
                                else load_stage(st, full_bar(s), tl, k, terms.a[j], terms.b[j], 1, 1);
                                ++it;
                                if (++s == STAGES) {
                                    s = 0;
                                    ph ^= 1u;
                                    st = smem_u32(smem);
                                } else {
                                    st += stage_bytes;
                                }
                            }
                        }
                    }
                }
            }
            if (!ok) {
                // Let the copies already issued land before the CTA exits.
                const uint32_t first = it > (uint32_t)STAGES ? it - STAGES : 0u;
                for (uint32_t j = first; j < it; ++j) mbar_wait_drain(full_bar(j % STAGES), (j / STAGES) & 1u);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            uint32_t lc = 0, ph = 0, st = smem_u32(smem);
            int s = 0;
            bool ok = true, issued = false;
            for (int t = t_begin; t < t_end && ok; ++t) {
                const Tile tl = tiles[t];
                const int cb = chunk_blocks(tl);
                for (int c0 = tl.kb0; c0 < tl.kb1 && ok; c0 += cb, ++lc) {
                    const int c1 = min(c0 + cb, tl.kb1);
                    const uint32_t a = lc & 1u, use = lc >> 1;
                    if (!mbar_wait(tempty_bar(a), (use & 1u) ^ 1u, abort_flag, gtimeout)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem_base + a * (uint32_t)BNT;
                    uint32_t accumulate = 0;
                    for (int jj = CF.fused ? 0 : terms.n - 1; jj >= 0 && ok; --jj) {
                        for (int kb = c0; kb < c1 && ok; ++kb) {
                            for (int hk = 0; hk < BK / KS; ++hk) {
                                if (!mbar_wait(full_bar(s), ph, abort_flag, gtimeout)) {
                                    ok = false;
                                    break;
                                }
                                tc_fence_after();
                                if (CF.fused) {
                                    // terms from the smallest pieces to hi * hi
                                    for (int j = terms.n - 1; j >= 0; --j)
                                        mma_term(d, st + (uint32_t)(terms.a[j] * A_TILE),
                                                 st + (uint32_t)(pipe.na * A_TILE + terms.b[j] * B_TILE), accumulate);
                                } else {
                                    mma_term(d, st, st + (uint32_t)A_TILE, accumulate);
                                }
                                issued = true;
                                tc_commit(empty_bar(s));
                                if (++s == STAGES) {
                                    s = 0;
                                    ph ^= 1u;
                                    st = smem_u32(smem);
                                } else {
                                    st += stage_bytes;
                                }
                            }
                        }
                    }
                    if (ok) tc_commit(tfull_bar(a));
                }
            }
            if (!ok && issued) {
                // Wait until every product issued so far has completed.
                tc_commit(drain_bar);
                mbar_wait_drain(drain_bar, 0);
            }
        }
    } else {
        // ---------------- epilogue (warps 2..9) ----------------
        // Warp w reads TMEM lane quarter (w % 4); warps 2-5 take columns 0-127 and warps
        // 6-9 columns 128-255 of the accumulator.
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row = quarter * 32 + lane;
        uint32_t lc = 0;
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; ++t) {
            const Tile tl = tiles[t];
            const int cb = chunk_blocks(tl);
            const int64_t gm = (int64_t)tl.om + row;
            const int64_t xb = (int64_t)tl.b * ep.xs, ob = (int64_t)tl.b * ep.os;
            float sum[PROMOTE ? BNT / 2 : 1];
            if (PROMOTE) {
#pragma unroll
                for (int i = 0; i < BNT / 2; ++i) sum[i] = 0.f;
            }
            // The update reads X: fetch the first 16 columns before the accumulator is ready.
            const int64_t gcol0 = (int64_t)tl.on + half * (BNT / 2);
            float xv[MODE == MODE_UPD ? 16 : 1];
            if (MODE == MODE_UPD) load_x16<TRANS, UNIT>(ep, xb, gm, gcol0, *(float(*)[16])xv);
            for (int c0 = tl.kb0; c0 < tl.kb1; c0 += cb, ++lc) {
                const uint32_t a = lc & 1u, use = lc >> 1;
                if (!mbar_wait(tfull_bar(a), use & 1u, abort_flag, gtimeout)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem_base + a * (uint32_t)BNT + (uint32_t)(half * (BNT / 2)) +
                                       ((uint32_t)(quarter * 32) << 16);
                if (PROMOTE) {
#pragma unroll
                    for (int q = 0; q < BNT / 32; ++q) {
                        uint32_t r[16];
                        tmem_ld16(taddr + q * 16, r);
#pragma unroll
                        for (int i = 0; i < 16; ++i) sum[q * 16 + i] += __uint_as_float(r[i]);
                    }
                } else if (MODE == MODE_UPD) {
                    // Software pipeline: the next 16 X values are in flight while the
                    // current ones are added and stored.
#pragma unroll 1
                    for (int q = 0; q < BNT / 32; ++q) {
                        float xn[16];
                        if (q + 1 < BNT / 32)
                            load_x16<TRANS, UNIT>(ep, xb, gm, gcol0 + (q + 1) * 16, xn);
                        uint32_t r[16];
                        tmem_ld16(taddr + q * 16, r);
                        store_upd16<TRANS, UNIT>(ep, xb, gm, gcol0 + q * 16, *(float(*)[16])xv, r);
                        if (q + 1 < BNT / 32) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) xv[i] = xn[i];
                        }
                    }
                } else {
#pragma unroll 1
                    for (int q = 0; q < BNT / 16; ++q) {
                        uint32_t r[8];
                        tmem_ld8(taddr + q * 8, r);
                        epilogue_cols<MODE, TRANS, UNIT, 8>(ep, xb, ob, gm, gcol0 + q * 8, r);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty_bar(a));
            }
            if (PROMOTE && ok) {
                // a matrix whose diagonal block needed the FP64 fallback skips its step
                bool zero = false;
                if (MODE == MODE_RES && ep.skip) {
                    int f = 0;
                    for (int i = lane; i < ep.skip_n; i += 32) f |= ep.skip[(int64_t)tl.b * ep.skip_n + i];
                    zero = __any_sync(0xffffffffu, f != 0);
                }
#pragma unroll
                for (int q = 0; q < BNT / 32; ++q) {
                    uint32_t r[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) r[i] = __float_as_uint(sum[q * 16 + i]);
                    epilogue_cols<MODE, TRANS, UNIT, 16>(ep, xb, ob, gm, (int64_t)tl.on + half * (BNT / 2) + q * 16, r,
                                                         zero);
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

// ---- host side ------------------------------------------------------------------------

template <int MODE, bool TRANS, bool UNIT, int BNT = BN>
cudaError_t launch_t(const Ctx &c, const Maps &maps, const Terms &terms, const Pipe &pipe, const Tile *d_tiles,
                     const int *d_off, int ctas, const Epi &epi) {
    auto kern = tc_gemm_kernel<MODE, TRANS, UNIT, BNT>;
    static bool attr_set[64] = {};
    if (!attr_set[c.device]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set[c.device] = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = GEMM_SMEM_BYTES;
    cfg.stream = c.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, maps, terms, pipe, d_tiles, d_off, epi, c.timeout);
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool get_encode() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_encode != nullptr;
}

}  // namespace

// 2-D map over a column-major BF16 plane: inner dimension = rows, 128-byte (or 64-byte)
// swizzle, box = box_rows x box_cols, zero fill outside [0, rows) x [0, cols).
bool encode_plane(CUtensorMap *m, const Plane &p, int box_rows, int box_cols, bool swizzle64) {
    if (!get_encode()) return false;
    if (((uintptr_t)p.p & 15) || (p.ld * 2) % 16 || p.rows <= 0 || p.cols <= 0 || p.batch < 1) return false;
    if (p.batch > 1 && ((p.bstride * 2) % 16 || p.bstride < p.ld * p.cols)) return false;
    const cuuint32_t rank = p.batch > 1 ? 3 : 2;
    cuuint64_t dims[3] = {(cuuint64_t)p.rows, (cuuint64_t)p.cols, (cuuint64_t)p.batch};
    cuuint64_t strides[2] = {(cuuint64_t)(p.ld * 2), (cuuint64_t)(p.bstride * 2)};
    cuuint32_t box[3] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank, (void *)p.p, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE,
                          swizzle64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int schedule_lpt(std::vector<Tile> &tiles, int terms, int ctas, std::vector<int> &offsets) {
    const int nt = (int)tiles.size();
    if (ctas > nt) ctas = nt;
    if (ctas < 1) ctas = 1;
    constexpr int kEpilogueCost = 8;   // pipeline-slot equivalents per tile
    auto cost = [&](const Tile &t) { return (t.kb1 - t.kb0) * terms + kEpilogueCost; };
    std::vector<int> order(nt);
    for (int i = 0; i < nt; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return cost(tiles[x]) > cost(tiles[y]); });
    // min-heap of (load, cta)
    std::vector<std::pair<long long, int>> heap;
    for (int b = 0; b < ctas; ++b) heap.push_back({0, b});
    auto cmp = [](const std::pair<long long, int> &x, const std::pair<long long, int> &y) {
        return x.first > y.first || (x.first == y.first && x.second > y.second);
    };
    std::make_heap(heap.begin(), heap.end(), cmp);
    std::vector<std::vector<int>> lists(ctas);
    for (int i : order) {
        std::pop_heap(heap.begin(), heap.end(), cmp);
        auto &top = heap.back();
        lists[top.second].push_back(i);
        top.first += cost(tiles[i]);
        std::push_heap(heap.begin(), heap.end(), cmp);
    }
    std::vector<Tile> out;
    out.reserve(nt);
    offsets.assign(ctas + 1, 0);
    for (int b = 0; b < ctas; ++b) {
        offsets[b] = (int)out.size();
        for (int i : lists[b]) out.push_back(tiles[i]);
    }
    offsets[ctas] = (int)out.size();
    tiles.swap(out);
    return ctas;
}

cudaError_t launch_tc(const Ctx &c, int mode, bool trans, bool unit, const Plane *aplanes, int na,
                      const Plane *bplanes, int nb, const Terms &terms, const Tile *d_tiles,
                      const int *d_off, int ctas, const Epi &epi, double flops,
                      const char *trace_name, int bn) {
    if (ctas <= 0) return cudaSuccess;
    if (na < 1 || na > 3 || nb < 1 || nb > 3 || terms.n < 1 || terms.n > 6) return cudaErrorInvalidValue;
    // narrow tiles are built for the level products only
    const bool level = mode == MODE_W || mode == MODE_X21 || mode == MODE_W6 || mode == MODE_X216;
    if (bn != BN && !((bn == 128 || bn == 64) && level)) return cudaErrorInvalidValue;
    Maps maps;
    memset(&maps, 0, sizeof(maps));
    const Cfg cf = cfg_for(mode);
    for (int i = 0; i < 3; ++i) {
        const Plane &pa = aplanes[i < na ? i : 0];
        const Plane &pb = bplanes[i < nb ? i : 0];
        if (!encode_plane(&maps.a[i], pa, 64, cf.ks)) return cudaErrorInvalidValue;
        if (!encode_plane(&maps.b[i], pb, cf.ks, bn, cf.ks == 32)) return cudaErrorInvalidValue;
    }
    // Stage layout: every distinct plane the terms read (fused), or one term's pair.
    Pipe pipe{1, 1, 0, 0, 0};
    for (int j = 0; j < terms.n; ++j) {
        if (terms.a[j] < 0 || terms.a[j] >= na || terms.b[j] < 0 || terms.b[j] >= nb) return cudaErrorInvalidValue;
        if (cf.fused) {
            pipe.na = std::max(pipe.na, terms.a[j] + 1);
            pipe.nb = std::max(pipe.nb, terms.b[j] + 1);
        }
    }
    pipe.stage_bytes = (pipe.na * BM + pipe.nb * bn) * cf.ks * 2;
    pipe.batched = aplanes[0].batch > 1 ? 1 : 0;
    for (int i = 0; i < na; ++i)
        if ((aplanes[i].batch > 1) != (pipe.batched != 0)) return cudaErrorInvalidValue;
    for (int i = 0; i < nb; ++i)
        if ((bplanes[i].batch > 1) != (pipe.batched != 0)) return cudaErrorInvalidValue;
    pipe.stages = std::min(MAX_STAGES, STAGE_BUDGET / pipe.stage_bytes);
    TraceScope ts(c.stream, trace_name, flops, 0.0);
#define TRI_TC_CASE_N(M, N)                                                                   \
        if (trans) return unit ? launch_t<M, true, true, N>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi)   \
                               : launch_t<M, true, false, N>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi); \
        return unit ? launch_t<M, false, true, N>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi)             \
                    : launch_t<M, false, false, N>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi);
#define TRI_TC_CASE(M) \
    case M:            \
        TRI_TC_CASE_N(M, BN)
#define TRI_TC_CASE_LEVEL(M)                 \
    case M:                                  \
        if (bn == 64) { TRI_TC_CASE_N(M, 64) } \
        if (bn == 128) { TRI_TC_CASE_N(M, 128) } \
        TRI_TC_CASE_N(M, BN)
    switch (mode) {
        TRI_TC_CASE_LEVEL(MODE_W)
        TRI_TC_CASE_LEVEL(MODE_X21)
        TRI_TC_CASE_LEVEL(MODE_W6)
        TRI_TC_CASE_LEVEL(MODE_X216)
        TRI_TC_CASE(MODE_RES)
        TRI_TC_CASE(MODE_UPD)
        case MODE_F32:
            return launch_t<MODE_F32, false, false>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi);
        case MODE_GEN:
            return launch_t<MODE_GEN, false, false>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi);
        case MODE_GENP:
            return launch_t<MODE_GENP, false, false>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi);
        default:
            return cudaErrorInvalidValue;
    }
#undef TRI_TC_CASE
#undef TRI_TC_CASE_LEVEL
#undef TRI_TC_CASE_N
}

}  // namespace tc
}  // namespace triinv

// Verification entry point: the product kernel on plain column-major BF16 operands.
extern "C" tri_status tri_tc_gemm_bf16(int64_t m, int64_t n, int64_t k, int nterms,
                                       const void *const *a_planes, int64_t lda,
                                       const void *const *b_planes, int64_t ldb, float *c,
                                       int64_t ldc, void *stream) {
    using namespace triinv;
    if (m < 0 || n < 0 || k < 0 || nterms < 1 || nterms > 3 || !a_planes || !b_planes) return TRI_ERR_ARG;
    if (m == 0 || n == 0) return TRI_OK;
    if (k == 0 || !c || ldc < m || lda < m || ldb < k || (lda % 8) || (ldb % 8)) return TRI_ERR_ARG;
    if (m > (1ll << 30) || n > (1ll << 30) || k > (1ll << 30)) return TRI_ERR_ARG;
    tc::Plane ap[3], bp[3];
    for (int i = 0; i < nterms; ++i) {
        if (!a_planes[i] || !b_planes[i] || ((uintptr_t)a_planes[i] & 15) || ((uintptr_t)b_planes[i] & 15))
            return TRI_ERR_ARG;
        ap[i] = tc::Plane{(const __nv_bfloat16 *)a_planes[i], m, k, lda};
        bp[i] = tc::Plane{(const __nv_bfloat16 *)b_planes[i], k, n, ldb};
    }
    Ctx ctx;
    tri_status st = device_ctx_public((cudaStream_t)stream, &ctx);
    if (st != TRI_OK) return st;
    std::vector<tc::Tile> v;
    const int64_t kb = (k + tc::BK - 1) / tc::BK;
    for (int64_t tm = 0; tm * tc::BM < m; ++tm)
        for (int64_t tn = 0; tn * tc::BN < n; ++tn)
            v.push_back(tc::Tile{(int)(tm * tc::BM), 0, 0, (int)(tn * tc::BN), 0, (int)kb, (int)(tm * tc::BM),
                                 (int)(tn * tc::BN)});
    std::vector<int> off;
    const int ctas = tc::schedule_lpt(v, nterms, ctx.sm_count, off);
    const size_t tbytes = v.size() * sizeof(tc::Tile), obytes = off.size() * sizeof(int);
    uint8_t *d = nullptr;
    if (lib_malloc_async((void **)&d, tbytes + obytes, ctx.stream) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_NOMEM;
    }
    if (cudaMemcpyAsync(d, v.data(), tbytes, cudaMemcpyHostToDevice, ctx.stream) != cudaSuccess ||
        cudaMemcpyAsync(d + tbytes, off.data(), obytes, cudaMemcpyHostToDevice, ctx.stream) != cudaSuccess)
        return TRI_ERR_CUDA;
    tc::Terms terms{nterms, {0, 1, 2}, {0, 1, 2}};
    tc::Epi ep{c, ldc, nullptr, nullptr, nullptr, 0, m, n};
    cudaError_t e = tc::launch_tc(ctx, tc::MODE_F32, false, false, ap, nterms, bp, nterms, terms,
                                  (const tc::Tile *)d, (const int *)(d + tbytes), ctas, ep,
                                  2.0 * m * n * k * nterms, "tc_gemm:f32");
    cudaFreeAsync(d, ctx.stream);
    return e == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
}
