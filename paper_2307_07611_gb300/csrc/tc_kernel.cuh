// tc_kernel.cuh -- the tcgen05 split-BF16 product kernel, shared by the single-CTA
// launcher (tc_gemm.cu) and the CTA-pair launcher (tc_gemm_pair.cu).
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
//               MN-major) + a B tile BN x 64 (K-major), or for the six-term products per
//               32-wide k-step all three A and three B plane tiles at once.
//   warp 1      allocates 512 TMEM columns (two 128 x BN FP32 accumulators), one lane
//               issues tcgen05.mma (M = 128, N = BN, K = 16) and commits slots / accumulators.
//   warps 2..9  epilogue: tcgen05.ld of the accumulator (two warps per 32-lane quarter,
//               BN / 2 columns each), split / update / store, then release the accumulator.
// The epilogue of tile i overlaps the main loop of tile i+1 (double-buffered TMEM).
//
// CTA pairs (PAIR): a cluster of two CTAs on two SMs computes a 256 x BN tile with one
// tcgen05.mma.cta_group::2 (M = 256) per K = 16 step.  Each CTA stages its own 128 rows of
// A and its own half (BN / 2 rows) of the B tile, so a CTA moves 16 + 16 KB per 64-wide
// k-block instead of 16 + 32 KB, for the same 128 x BN share of the products.  Roles:
//   even CTA    producer for its halves, expecting the bytes of both CTAs on its stage
//               barrier; the MMA issuer (frees both CTAs' slots and accumulators by
//               multicast commits); epilogue of rows 0-127 of the tile.
//   odd CTA     producer for its halves, its copies completing on the even CTA's stage
//               barrier (cp.async.bulk.tensor.cta_group::2); epilogue of rows 128-255,
//               releasing the accumulator on the even CTA's barrier.
// Every mbarrier wait is bounded (globaltimer); on timeout the kernel records the status,
// drains its in-flight copies and products, frees TMEM and returns (a pair meets at a
// cluster barrier first, so that neither SM leaves while the other may still touch its
// shared or tensor memory).
//
// Operand layouts in shared memory (canonical tcgen05 layouts):
//   A (MN-major, 128-byte swizzle): atom = 64 M-elements (128 B) x 8 K-rows; the two
//                 64-row atoms ks * 128 B apart (LBO), K atoms 1024 B apart (SBO).  One MMA
//                 (K = 16) spans two K atoms (2048 B).
//   B (K-major, 128- or 64-byte swizzle for ks = 64 / 32): atom = 8 N-rows x ks
//                 K-elements; N atoms ks * 16 B apart (SBO); the k-offset inside the row
//                 advances the start address by 32 B per K = 16.
#pragma once

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "tc_ptx.cuh"

namespace triinv {
namespace tc {

struct Maps {
    CUtensorMap a[4];
    CUtensorMap b[4];
};

// Pipeline geometry per mode.
//   ks       k per stage: 64 (B tiles 64 wide with 128-byte swizzle) or 32 (64-byte
//            swizzle).  A tiles are 128 x ks, two 64-row boxes with 128-byte swizzle.
//   fused    true: a stage holds every distinct plane tile the terms read and the MMA
//            issuer runs all terms on it (each plane crosses L2 once per k-step); false:
//            a stage holds the A / B pair of one term (loop: chunk, term, k).
//   promote  MODE_RES, MODE_GENP, MODE_W6, MODE_X216: 64-wide k-blocks accumulated in
//            tensor memory before the epilogue adds them into FP32 registers.  The
//            accumulator truncates every add, so a product added after the large hi*hi
//            term loses up to one unit in the last place of the partial sum; the chunk
//            length bounds that loss.
// R = I - T X and the general six-term products read 3 + 3 planes: fused 32-wide stages
// (72 KB, 3 deep) halve their L2 traffic.  The three-term level products with 64- or
// 128-wide output tiles take fused 64-wide stages (both planes of each operand, 12 MMAs
// per stage; 48 / 64 KB, 4 / 3 deep); with 256-wide tiles such a stage is 96 KB and only
// two fit, so they, the update and the other products keep 64-wide per-term stages
// (48 KB, 4 deep).  Each choice measured fastest at n = 8192 (more tensor work per stage
// helps while the ring stays at least three deep).
struct Cfg {
    int ks;
    bool fused;
    int promote;
};
__host__ __device__ constexpr Cfg cfg_for(int mode, int bn = BN) {
    return (mode == MODE_RES || mode == MODE_GENP || mode == MODE_W6 || mode == MODE_X216) ? Cfg{32, true, 1}
           : ((mode == MODE_W || mode == MODE_X21 || mode == MODE_LVL) && bn <= 128) ? Cfg{64, true, 0}
                                                                                  : Cfg{64, false, 0};
}

constexpr int STAGE_BUDGET = 216 * 1024;
constexpr int MAX_STAGES = 9;
constexpr int GEMM_SMEM_BYTES = STAGE_BUDGET + 1024 + 512;

// Stage layout of one launch (host-computed from the terms and the mode's geometry).
struct Pipe {
    int na, nb;          // A / B tiles per stage
    int stages;          // ring depth
    int stage_bytes;     // (na * BM + nb * B rows staged per CTA) * ks * 2
    int batched;         // maps are 3-D (batch outermost): loads take the tile's matrix
};

// CTA-pair launch of the products of the mixed path (tc_gemm_pair.cu): `ctas` = 2 x the
// pairs, CTA pair p processes the 256-row tiles d_tiles[d_off[p] .. d_off[p+1]).
cudaError_t launch_pair(const Ctx &c, int mode, bool trans, bool unit, const Maps &maps, const Terms &terms,
                        const Pipe &pipe, const Tile *d_tiles, const int *d_off, int ctas, const Epi &epi);

namespace {

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

// Dependency counters of MODE_LVL (global memory, written by other CTAs of the launch).
__device__ __forceinline__ int dep_ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void dep_red_release_add(int *p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void dep_fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
// Bounded wait until *c >= need.  False if the CTA is aborting or the deadline passed (then
// it raises the abort flag and the device timeout word).
__device__ __forceinline__ bool dep_wait(const int *c, int need, volatile int *abort_flag, int *gtimeout) {
    if (dep_ld_acquire(c) >= need) return true;
    const uint64_t t0 = gtimer();
    for (uint32_t i = 1;; ++i) {
        __nanosleep(64);
        if (dep_ld_acquire(c) >= need) return true;
        if ((i & 15) == 0) {
            if (*abort_flag) return false;
            if (gtimer() - t0 > kWaitLimitNs) {
                *abort_flag = 1;
                atomicExch(gtimeout, 1);
                return false;
            }
        }
    }
}

// Drain wait after an abort: gives up at `deadline` (globaltimer ns).
__device__ __forceinline__ void mbar_wait_drain_until(uint32_t bar, uint32_t parity, uint64_t deadline) {
    while (!mbar_try_wait(bar, parity)) {
        if (gtimer() > deadline) return;
    }
}

// BNT: columns of an output tile (UMMA N = 256, 128 or 64).  Narrower tiles give the
// small products of the low split levels more, shorter tiles (more SMs busy, a shorter
// longest tile); the widest tile moves the fewest operand bytes per flop.
// PAIR: 256 x BNT tiles, each computed by the two CTAs of a cluster (see above).
template <int MODE, bool TRANS, bool UNIT, int BNT, bool PAIR = false>
__global__ void __launch_bounds__(NTHREADS, 1)
tc_gemm_kernel(const __grid_constant__ Maps maps, const Terms terms, const Pipe pipe,
               const Tile *__restrict__ tiles, const int *__restrict__ cta_off, const Epi ep,
               const Epi ep2, int *gtimeout) {
    constexpr bool PROMOTE = (MODE == MODE_RES || MODE == MODE_GENP || MODE == MODE_W6 || MODE == MODE_X216);
    constexpr Cfg CF = cfg_for(MODE, BNT);
    constexpr int KS = CF.ks;
    constexpr int BNL = PAIR ? BNT / 2 : BNT;   // B columns this CTA stages
    constexpr int A_TILE = BM * KS * 2, B_TILE = BNL * KS * 2;
    constexpr uint32_t IDESC = idesc_for(BNT, PAIR ? 2 * BM : BM);
    constexpr uint16_t PAIR_MASK = 0x3;         // both CTAs of the cluster
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
    const uint32_t rank = PAIR ? cluster_rank() : 0u;   // 0: the CTA that issues the products
    const bool leader = rank == 0;
    const int owner = PAIR ? (int)cluster_id_x() : (int)blockIdx.x;   // index of the tile list
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (MAX_STAGES + s); };
    auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * MAX_STAGES + a); };
    auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * MAX_STAGES + 2 + a); };
    const uint32_t drain_bar = bar0 + 8u * (2 * MAX_STAGES + 4);
    auto wait = [&](uint32_t bar, uint32_t parity) { return mbar_wait(bar, parity, abort_flag, gtimeout); };
    auto commit = [&](uint32_t bar) {
        if constexpr (PAIR) tc_commit_pair_mc(bar, PAIR_MASK);
        else tc_commit(bar);
    };
    // 64-wide k-blocks per accumulation chunk: one chunk per tile unless promoting.
    auto chunk_blocks = [&](const Tile &tl) { return PROMOTE ? CF.promote : (tl.kb1 - tl.kb0); };
    // One stage: load A tiles ia[0..na) and B tiles ib[0..nb) at k (this CTA's rows of A,
    // its half of the B columns in a pair).  A pair's stage completes on the even CTA's
    // barrier, which expects both CTAs' bytes; the odd CTA's copies signal it remotely.
    auto load_stage = [&](uint32_t st, uint32_t bar, const Tile &tl, int k, int ia0, int ib0, int na, int nb) {
        const uint32_t bytes = (uint32_t)(na * A_TILE + nb * B_TILE);
        const bool remote = PAIR && !leader;
        if (!remote) mbar_arrive_expect_tx(bar, PAIR ? 2 * bytes : bytes);
        const uint32_t rbar = remote ? cluster_addr(bar, 0) : bar;
        auto load2 = [&](uint32_t dst, const CUtensorMap *m, int x, int y) {
            if (remote) tma_load_2d_pair(dst, m, x, y, rbar);
            else tma_load_2d(dst, m, x, y, bar);
        };
        auto load3 = [&](uint32_t dst, const CUtensorMap *m, int x, int y, int z) {
            if (remote) tma_load_3d_pair(dst, m, x, y, z, rbar);
            else tma_load_3d(dst, m, x, y, z, bar);
        };
        const int am = tl.am + (int)rank * BM, bn = tl.bn + (int)rank * BNL;
        for (int i = 0; i < na; ++i) {
            const uint32_t dst = st + (uint32_t)(i * A_TILE);
#pragma unroll
            for (int c = 0; c < BM / 64; ++c) {
                if (pipe.batched) load3(dst + (uint32_t)(c * KS * 128), &maps.a[ia0 + i], am + 64 * c, tl.ak + k, tl.b);
                else load2(dst + (uint32_t)(c * KS * 128), &maps.a[ia0 + i], am + 64 * c, tl.ak + k);
            }
        }
        for (int i = 0; i < nb; ++i) {
            const uint32_t dst = st + (uint32_t)(na * A_TILE + i * B_TILE);
            if (pipe.batched) load3(dst, &maps.b[ib0 + i], tl.bk + k, bn, tl.b);
            else load2(dst, &maps.b[ib0 + i], tl.bk + k, bn);
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
            if constexpr (PAIR) tc_mma_pair(d, da, db, IDESC, accumulate);
            else tc_mma(d, da, db, IDESC, accumulate);
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
            mbar_init(tempty_bar(a), PAIR ? 2 * EPI_WARPS : EPI_WARPS);
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        for (int i = 0; i < 4; ++i) {
            prefetch_map(&maps.a[i]);
            prefetch_map(&maps.b[i]);
        }
    }
    if (warp == 1) {
        // a pair allocates the same columns on both SMs: one warp of each CTA takes part
        if constexpr (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    tc_fence_before();
    // a pair: the other CTA's barriers are initialised before any arrive from this one
    if constexpr (PAIR) {
        __syncwarp();
        cluster_sync_all();
    } else {
        __syncthreads();
    }
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int t_begin = cta_off[owner], t_end = cta_off[owner + 1];   // plan data: constant
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
                // MODE_LVL: X21 tiles read the X21 planes' maps (two further on)
                const int toff = (MODE == MODE_LVL && tl.kind) ? 2 : 0;
                if (MODE == MODE_LVL && (tl.wait0 >= 0 || tl.wait1 >= 0)) {
                    // operands written by other CTAs of this launch (generic-proxy stores,
                    // published with release adds): acquire, then order the async-proxy reads
                    if (tl.wait0 >= 0) ok = dep_wait(ep.cnt + tl.wait0, tl.need0, abort_flag, gtimeout);
                    if (ok && tl.wait1 >= 0) ok = dep_wait(ep.cnt + tl.wait1, tl.need1, abort_flag, gtimeout);
                    if (!ok) break;
                    __threadfence();
                    dep_fence_proxy_async_global();
                }
                for (int c0 = tl.kb0; c0 < tl.kb1 && ok; c0 += cb) {
                    const int c1 = min(c0 + cb, tl.kb1);
                    // fused: one pass with every plane; else one pass per term (smallest first)
                    for (int j = CF.fused ? 0 : terms.n - 1; j >= 0 && ok; --j) {
                        for (int kb = c0; kb < c1 && ok; ++kb) {
                            for (int hk = 0; hk < BK / KS; ++hk) {
                                if (!wait(empty_bar(s), ph ^ 1u)) {
                                    ok = false;
                                    break;
                                }
                                const int k = kb * BK + hk * KS;
                                if (CF.fused) load_stage(st, full_bar(s), tl, k, toff, toff, pipe.na, pipe.nb);
                                else load_stage(st, full_bar(s), tl, k, terms.a[j] + toff, terms.b[j] + toff, 1, 1);
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
                // Let the copies already issued land before the CTA exits.  A pair's stages
                // complete on the even CTA's barriers: there they also wait for the other
                // CTA's bytes, which may never come (the whole drain is bounded by one wait
                // limit); the odd CTA cannot watch them and gives its copies a fixed 200 us.
                if (PAIR && !leader) {
                    const uint64_t t0 = gtimer();
                    while (gtimer() - t0 < 200000ull) {
                    }
                } else {
                    const uint64_t deadline = gtimer() + kWaitLimitNs;
                    const uint32_t first = it > (uint32_t)STAGES ? it - STAGES : 0u;
                    for (uint32_t j = first; j < it; ++j)
                        mbar_wait_drain_until(full_bar(j % STAGES), (j / STAGES) & 1u, deadline);
                }
            }
        }
    } else if (warp == 1) {
        if (PAIR && !leader) {
            // the odd CTA of a pair issues no products
        } else if (lane == 0) {
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
                    if (!wait(tempty_bar(a), (use & 1u) ^ 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem_base + a * (uint32_t)BNT;
                    uint32_t accumulate = 0;
                    for (int jj = CF.fused ? 0 : terms.n - 1; jj >= 0 && ok; --jj) {
                        for (int kb = c0; kb < c1 && ok; ++kb) {
                            for (int hk = 0; hk < BK / KS; ++hk) {
                                if (!wait(full_bar(s), ph)) {
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
                                commit(empty_bar(s));
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
                    if (ok) commit(tfull_bar(a));
                }
            }
            if (!ok && issued) {
                // Wait until every product issued so far has completed.
                if constexpr (PAIR) tc_commit_pair(drain_bar);
                else tc_commit(drain_bar);
                mbar_wait_drain(drain_bar, 0);
            }
        }
    } else {
        // ---------------- epilogue (warps 2..9) ----------------
        // Warp w reads TMEM lane quarter (w % 4); warps 2-5 take columns 0 .. BNT/2 - 1 and
        // warps 6-9 columns BNT/2 .. BNT - 1 of the accumulator.  In a pair, this CTA's
        // accumulator holds rows 128 * rank .. + 127 of the tile.
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row = quarter * 32 + lane;
        // a pair releases the accumulator on the issuing CTA's barrier
        const uint32_t tempty_rel0 = PAIR ? cluster_addr(tempty_bar(0), 0) : tempty_bar(0);
        uint32_t lc = 0;
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; ++t) {
            const Tile tl = tiles[t];
            const int cb = chunk_blocks(tl);
            const int64_t gm = (int64_t)tl.om + (int64_t)rank * BM + row;
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
                if (!wait(tfull_bar(a), use & 1u)) {
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
                } else if (MODE == MODE_LVL) {
                    if (tl.kind) {
                        const int64_t xb2 = (int64_t)tl.b * ep2.xs, ob2 = (int64_t)tl.b * ep2.os;
#pragma unroll 1
                        for (int q = 0; q < BNT / 16; ++q) {
                            uint32_t r[8];
                            tmem_ld8(taddr + q * 8, r);
                            epilogue_cols<MODE_X21, TRANS, UNIT, 8>(ep2, xb2, ob2, gm, gcol0 + q * 8, r);
                        }
                    } else {
#pragma unroll 1
                        for (int q = 0; q < BNT / 16; ++q) {
                            uint32_t r[8];
                            tmem_ld8(taddr + q * 8, r);
                            epilogue_cols<MODE_W, TRANS, UNIT, 8>(ep, xb, ob, gm, gcol0 + q * 8, r);
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
                if (lane == 0) {
                    if constexpr (PAIR) mbar_arrive_cluster(tempty_rel0 + 8u * a);
                    else mbar_arrive(tempty_bar(a));
                }
            }
            if (MODE == MODE_LVL && ok && tl.pub >= 0) {
                // Publish this warp's part of the tile: its generic-proxy stores visible at
                // GPU scope and to later async-proxy (TMA) reads, then one release add.
                dep_fence_proxy_async_global();
                __threadfence();
                __syncwarp();
                if (lane == 0) dep_red_release_add(ep.cnt + tl.pub, 1);
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
    // a pair: neither SM leaves (and frees its tensor or shared memory) before the other
    // has finished with them
    if constexpr (PAIR) {
        __syncwarp();
        cluster_sync_all();
    } else {
        __syncthreads();
    }
    if (warp == 1) {
        tc_fence_after();
        if constexpr (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                         : "memory");
    }
}

// Launch of `ctas` persistent CTAs (PAIR: ctas / 2 clusters of two).
template <int MODE, bool TRANS, bool UNIT, int BNT = BN, bool PAIR = false>
cudaError_t launch_t(const Ctx &c, const Maps &maps, const Terms &terms, const Pipe &pipe, const Tile *d_tiles,
                     const int *d_off, int ctas, const Epi &epi, const Epi &epi2) {
    auto kern = tc_gemm_kernel<MODE, TRANS, UNIT, BNT, PAIR>;
    static bool attr_set[64] = {};
    if (!attr_set[c.device]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set[c.device] = true;
    }
    if (PAIR && (ctas & 1)) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = GEMM_SMEM_BYTES;
    cfg.stream = c.stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (PAIR) {
        attr[1].id = cudaLaunchAttributeClusterDimension;
        attr[1].val.clusterDim.x = 2;
        attr[1].val.clusterDim.y = 1;
        attr[1].val.clusterDim.z = 1;
        cfg.numAttrs = 2;
    }
    return cudaLaunchKernelEx(&cfg, kern, maps, terms, pipe, d_tiles, d_off, epi, epi2, c.timeout);
}

}  // namespace
}  // namespace tc
}  // namespace triinv
