// tc_graph.cu -- every tensor-core product of the mixed-precision inverse in one
// persistent launch that follows the data dependencies tile by tile.
//
// The products of the recursive split (block inverse of the proof of the main Theorem,
// Section 3) form a DAG.  At level h, pair (A, B, C) needs
//     W   = B X_A      X_A: inverse of the upper-left block (lower levels of that block)
//     X21 = -X_C W     X_C: inverse of the lower-right block
// and the Newton-Schulz step R = I - T X, X += X R reads finished rows and columns of X
// and R.  With one launch per product every level waits for the whole previous one, and
// the small levels (h = 256 .. 1024: a few dozen tiles each) leave most SMs idle.  Here
// the host builds the tile DAG once per order n and list-schedules it onto one persistent
// CTA per SM, longest remaining path first.  Each CTA walks its list:
//   * the producer warp waits (ld.acquire, bounded) until every 128 x 256 region the
//     tile's operands read is complete, then issues the TMA loads;
//   * after storing a tile, each epilogue warp adds 1 (red.release) to the ready counter
//     of the region it wrote; a region is complete at EPI_WARPS.
// The list order is a topological order of the DAG and all CTAs are resident (grid <=
// SM count, one CTA per SM), so every wait ends; all waits are nevertheless bounded and
// abort the launch (timeout word) when the bound is hit.
//
// Regions: 128 rows x 256 columns of an n x n plane; counters for three planes, X
// (inverse: FP32 + BF16 planes), W (level products, stored where the B block of T sits)
// and R (Newton-Schulz residual).  X regions inside the 256 x 256 diagonal blocks are
// written before the launch (diagonal-block kernel) and have no counter wait.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <queue>
#include <vector>

#include "tc_graph.cuh"
#include "tc_ptx.cuh"

namespace triinv {
namespace tc {
namespace {

constexpr int kPromote = 4;   // k-blocks per FP32 promotion of the residual (see tc_gemm.cu)

// Operand planes: A maps T0 T1 T2 X0 X1 X2 (box 64 x 64), B maps X0 X1 X2 W0 W1 R0
// (box 64 x 256).  Terms of each product, as 2-bit digits (smallest pieces last):
//   W:   T_h X_h, T_h X_m, T_m X_h          X21: X_h W_h, X_h W_m, X_m W_h
//   RES: hh, hm, mh, hl, mm, lh             UPD: X_h R_h
struct GMaps {
    CUtensorMap a[6];
    CUtensorMap b[6];
};

__device__ __forceinline__ int op_terms(int op) { return op == G_RES ? 6 : (op == G_UPD ? 1 : 3); }

__device__ __forceinline__ void op_term(int op, int j, int &ia, int &ib) {
    constexpr uint32_t kA3 = 0u | (0u << 2) | (1u << 4), kB3 = 0u | (1u << 2) | (0u << 4);
    constexpr uint32_t kA6 = 0u | (0u << 2) | (1u << 4) | (0u << 6) | (1u << 8) | (2u << 10);
    constexpr uint32_t kB6 = 0u | (1u << 2) | (0u << 4) | (2u << 6) | (1u << 8) | (0u << 10);
    if (op == G_RES) {
        ia = (kA6 >> (2 * j)) & 3u;
        ib = (kB6 >> (2 * j)) & 3u;
    } else if (op == G_UPD) {
        ia = 3;
        ib = 5;
    } else {
        const int base = op == G_X21 ? 3 : 0;
        ia = base + (int)((kA3 >> (2 * j)) & 3u);
        ib = base + (int)((kB3 >> (2 * j)) & 3u);
    }
}

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(int *p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Bounded wait until region counter *f reaches EPI_WARPS.  False if this CTA or the
// launch is aborting or the deadline passed (then it raises both abort words and the
// device timeout word).
__device__ bool wait_ready(const int *f, volatile int *abort_flag, int *abort_word, int *gtimeout,
                           unsigned long long limit_ns) {
    if (ld_acquire(f) >= EPI_WARPS) return true;
    const uint64_t t0 = gtimer();
    for (uint32_t i = 1;; ++i) {
        __nanosleep(100);
        if (ld_acquire(f) >= EPI_WARPS) return true;
        if ((i & 15) == 0) {
            if (*abort_flag || *(volatile int *)abort_word) {
                *abort_flag = 1;
                return false;
            }
            if (gtimer() - t0 > limit_ns) {
                *abort_flag = 1;
                atomicExch(abort_word, 1);
                atomicExch(gtimeout, 1);
                return false;
            }
        }
    }
}

// One BF16 piece of v and the remainder.
__device__ __forceinline__ __nv_bfloat16 piece(float &v) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    v -= __bfloat162float(h);
    return h;
}

template <bool TRANS, bool UNIT>
// 10 warps: three share one SM sub-partition (16K registers), so at most 168 per thread.
__global__ void __launch_bounds__(NTHREADS, 1)
tc_graph_kernel(const __grid_constant__ GMaps maps, const GTile *__restrict__ tiles,
                const int *__restrict__ cta_off, const int *__restrict__ deps, const GEpi ep,
                int *gtimeout) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(smem + STAGES * STAGE_BYTES);
    uint32_t *tmem_slot = (uint32_t *)(bars + 2 * STAGES + 5);
    volatile int *abort_flag = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
    auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * STAGES + a); };
    auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * STAGES + 2 + a); };
    const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 4);
    auto chunk_blocks = [&](const GTile &tl) { return tl.op == G_RES ? kPromote : (tl.kb1 - tl.kb0); };

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
        for (int i = 0; i < 6; ++i) {
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
    const int t_begin = cta_off[blockIdx.x], t_end = cta_off[blockIdx.x + 1];
    // Programmatic dependent launch: nothing produced by earlier work on the stream (the
    // planes, the zeroed counters) is read before this wait.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (threadIdx.x == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    if (warp == 0) {
        // ---------------- producer: dependency waits (all lanes), TMA (lane 0) ----------------
        uint32_t it = 0;
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; ++t) {
            const GTile tl = tiles[t];
            unsigned long long *rec = ep.timeline ? ep.timeline + (size_t)t * kTimelineWords : nullptr;
            if (rec && lane == 0) {
                rec[0] = (unsigned long long)blockIdx.x | ((unsigned long long)tl.op << 16) |
                         ((unsigned long long)(tl.kb1 - tl.kb0) << 20) |
                         ((unsigned long long)(tl.om / BM) << 32) | ((unsigned long long)(tl.on / BN) << 48);
                rec[1] = gtimer();
            }
            bool dok = true;
            for (int d = tl.dep0 + lane; d < tl.dep1 && dok; d += 32)
                dok = wait_ready(ep.flags + deps[d], abort_flag, ep.abort_word, gtimeout, ep.limit_ns);
            __syncwarp();
            ok = __all_sync(0xffffffffu, dok);
            if (!ok) break;
            if (lane == 0) {
                // The regions were written through the generic proxy by other CTAs; order
                // the acquires above before the async-proxy (TMA) reads below.
                __threadfence();
                fence_proxy_async_global();
                if (rec) rec[2] = gtimer();
                const int cb = chunk_blocks(tl), nterm = op_terms(tl.op);
                for (int c0 = tl.kb0; c0 < tl.kb1 && ok; c0 += cb) {
                    const int c1 = min(c0 + cb, tl.kb1);
                    for (int j = nterm - 1; j >= 0 && ok; --j) {
                        int ia, ib;
                        op_term(tl.op, j, ia, ib);
                        const CUtensorMap *am = &maps.a[ia];
                        const CUtensorMap *bm = &maps.b[ib];
                        for (int kb = c0; kb < c1; ++kb) {
                            const int s = it % STAGES;
                            const uint32_t ph = (it / STAGES) & 1u;
                            if (!mbar_wait(empty_bar(s), ph ^ 1u, abort_flag, gtimeout, ep.limit_ns)) {
                                ok = false;
                                break;
                            }
                            const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
                            const uint32_t sb = sa + A_BYTES;
                            mbar_arrive_expect_tx(full_bar(s), STAGE_BYTES);
                            const int k = kb * BK;
                            tma_load_2d(sa, am, tl.am, tl.ak + k, full_bar(s));
                            tma_load_2d(sa + A_BYTES / 2, am, tl.am + 64, tl.ak + k, full_bar(s));
                            tma_load_2d(sb, bm, tl.bk + k, tl.bn, full_bar(s));
                            ++it;
                        }
                    }
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
        }
        if (!ok && lane == 0) {
            const uint32_t first = it > (uint32_t)STAGES ? it - STAGES : 0u;
            for (uint32_t j = first; j < it; ++j) mbar_wait_drain(full_bar(j % STAGES), (j / STAGES) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            uint32_t it = 0, lc = 0;
            bool ok = true, issued = false;
            for (int t = t_begin; t < t_end && ok; ++t) {
                const GTile tl = tiles[t];
                const int cb = chunk_blocks(tl), nterm = op_terms(tl.op);
                unsigned long long *rec = ep.timeline ? ep.timeline + (size_t)t * kTimelineWords : nullptr;
                if (rec) rec[3] = gtimer();
                for (int c0 = tl.kb0; c0 < tl.kb1 && ok; c0 += cb, ++lc) {
                    const int c1 = min(c0 + cb, tl.kb1);
                    const uint32_t a = lc & 1u, use = lc >> 1;
                    if (!mbar_wait(tempty_bar(a), (use & 1u) ^ 1u, abort_flag, gtimeout, ep.limit_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem_base + a * (uint32_t)BN;
                    uint32_t accumulate = 0;
                    for (int j = nterm - 1; j >= 0 && ok; --j) {
                        for (int kb = c0; kb < c1; ++kb) {
                            const int s = it % STAGES;
                            const uint32_t ph = (it / STAGES) & 1u;
                            if (!mbar_wait(full_bar(s), ph, abort_flag, gtimeout, ep.limit_ns)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);
                            const uint32_t sb = sa + A_BYTES;
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk) {
                                const uint64_t da = smem_desc(sa + kk * 2048, 8192, 1024);
                                const uint64_t db = smem_desc(sb + kk * 32, 16, 1024);
                                tc_mma(d, da, db, kIdesc, accumulate);
                                accumulate = 1;
                            }
                            issued = true;
                            tc_commit(empty_bar(s));
                            ++it;
                        }
                    }
                    if (ok) tc_commit(tfull_bar(a));
                }
                if (rec) rec[4] = gtimer();
            }
            if (!ok && issued) {
                tc_commit(drain_bar);
                mbar_wait_drain(drain_bar, 0);
            }
        }
    } else {
        // ---------------- epilogue (warps 2..9) ----------------
        // Warp w reads TMEM lane quarter (w % 4); warps 2-5 take columns 0-127 and warps
        // 6-9 columns 128-255 of the accumulator.  Thread = one output row.
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row = quarter * 32 + lane;
        const int64_t n = ep.n, ldp = ep.ldp;
        const int64_t xstep = TRANS ? 1 : ep.ldx;
        uint32_t lc = 0;
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; ++t) {
            const GTile tl = tiles[t];
            const int cb = chunk_blocks(tl);
            const int64_t gm = (int64_t)tl.om + row;
            const int64_t gn0 = (int64_t)tl.on + half * (BN / 2);
            const bool row_ok = gm < n;
            if (tl.op == G_RES) {
                float sum[BN / 2];
#pragma unroll
                for (int i = 0; i < BN / 2; ++i) sum[i] = 0.f;
                for (int c0 = tl.kb0; c0 < tl.kb1; c0 += cb, ++lc) {
                    const uint32_t a = lc & 1u, use = lc >> 1;
                    if (!mbar_wait(tfull_bar(a), use & 1u, abort_flag, gtimeout, ep.limit_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t taddr = tmem_base + a * (uint32_t)BN + (uint32_t)(half * (BN / 2)) +
                                           ((uint32_t)(quarter * 32) << 16);
#pragma unroll
                    for (int q = 0; q < BN / 32; ++q) {
                        uint32_t r[16];
                        tmem_ld16(taddr + q * 16, r);
#pragma unroll
                        for (int i = 0; i < 16; ++i) sum[q * 16 + i] += __uint_as_float(r[i]);
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tempty_bar(a));
                }
                if (!ok) break;
                // R = I - T X on the lower triangle, 0 above; hi piece only.
                if (row_ok) {
                    int64_t off = gm + gn0 * ldp;
#pragma unroll
                    for (int j = 0; j < BN / 2; ++j) {
                        const int64_t gn = gn0 + j;
                        if (gn < n) {
                            const float v = gm >= gn ? ((gm == gn ? 1.f : 0.f) - sum[j]) : 0.f;
                            ep.rp[off] = __float2bfloat16_rn(v);
                        }
                        off += ldp;
                    }
                }
            } else if (tl.op == G_UPD) {
                if (tl.xin_flag >= 0) {
                    bool r = true;
                    if (lane == 0) r = wait_ready(ep.flags + tl.xin_flag, abort_flag, ep.abort_word, gtimeout, ep.limit_ns);
                    ok = __shfl_sync(0xffffffffu, r, 0);
                    __syncwarp();
                    if (!ok) break;
                }
                const uint32_t a = lc & 1u, use = lc >> 1;
                ++lc;
                // X values this thread updates: lower triangle (and the diagonal unless unit).
                auto upd_mask = [&](int64_t gn) { return row_ok && gn < n && (gm > gn || (!UNIT && gm == gn)); };
                float xv[16];
                {
                    int64_t xo = vidx<TRANS>(gm, gn0, ep.ldx);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        xv[j] = upd_mask(gn0 + j) ? ep.x[xo] : 0.f;
                        xo += xstep;
                    }
                }
                if (!mbar_wait(tfull_bar(a), use & 1u, abort_flag, gtimeout, ep.limit_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem_base + a * (uint32_t)BN + (uint32_t)(half * (BN / 2)) +
                                       ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
                for (int q = 0; q < BN / 32; ++q) {
                    const int64_t c = gn0 + q * 16;
                    float xn[16];
                    if (q + 1 < BN / 32) {
                        int64_t xo = vidx<TRANS>(gm, c + 16, ep.ldx);
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            xn[j] = upd_mask(c + 16 + j) ? ep.x[xo] : 0.f;
                            xo += xstep;
                        }
                    }
                    uint32_t r[16];
                    tmem_ld16(taddr + q * 16, r);
                    int64_t xo = vidx<TRANS>(gm, c, ep.ldx);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (upd_mask(c + j)) ep.x[xo] = xv[j] + __uint_as_float(r[j]);
                        xo += xstep;
                    }
                    if (q + 1 < BN / 32) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) xv[j] = xn[j];
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty_bar(a));
            } else {
                // W (hi / mid pieces into the W planes) or X21 (X = -acc in FP32 and its
                // hi / mid / lo pieces).
                const uint32_t a = lc & 1u, use = lc >> 1;
                ++lc;
                if (!mbar_wait(tfull_bar(a), use & 1u, abort_flag, gtimeout, ep.limit_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem_base + a * (uint32_t)BN + (uint32_t)(half * (BN / 2)) +
                                       ((uint32_t)(quarter * 32) << 16);
                const bool x21 = tl.op == G_X21;
#pragma unroll 1
                for (int q = 0; q < BN / 16; ++q) {
                    uint32_t r[8];
                    tmem_ld8(taddr + q * 8, r);
                    const int64_t c = gn0 + q * 8;
                    if (!row_ok) continue;
                    int64_t off = gm + c * ldp;
                    int64_t xo = vidx<TRANS>(gm, c, ep.ldx);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        if (c + j < n) {
                            float v = __uint_as_float(r[j]);
                            if (x21) {
                                v = -v;
                                ep.x[xo] = v;
                                ep.xp0[off] = piece(v);
                                ep.xp1[off] = piece(v);
                                ep.xp2[off] = __float2bfloat16_rn(v);
                            } else {
                                ep.wp0[off] = piece(v);
                                ep.wp1[off] = __float2bfloat16_rn(v);
                            }
                        }
                        off += ldp;
                        xo += xstep;
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty_bar(a));
            }
            if (tl.out_flag >= 0) {
                // Publish this warp's part of the region: generic-proxy stores made visible
                // at GPU scope (and to later async-proxy reads), then one release per warp.
                fence_proxy_async_global();
                __threadfence();
                __syncwarp();
                if (lane == 0 && tl.out_flag != ep.withhold) red_release_add(ep.flags + tl.out_flag, 1);
            }
            if (ep.timeline && warp == 2 && lane == 0) ep.timeline[(size_t)t * kTimelineWords + 5] = gtimer();
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

template <bool TRANS, bool UNIT>
cudaError_t launch_g(const Ctx &c, const GMaps &maps, const GraphPlan &p, const GEpi &ep) {
    auto kern = tc_graph_kernel<TRANS, UNIT>;
    static bool attr_set[64] = {};
    if (!attr_set[c.device]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set[c.device] = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p.ctas);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = c.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, maps, (const GTile *)p.d_tiles, (const int *)p.d_off,
                              (const int *)p.d_deps, ep, c.timeout);
}

// ---- host: the tile DAG and its schedule -----------------------------------------------

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

struct Dag {
    std::vector<GTile> tiles;
    std::vector<std::vector<int>> flag_deps;   // flag indices per tile
    std::vector<std::vector<int>> preds;       // producing tiles per tile
    std::vector<int> kcost;                    // k-blocks x terms
};

// Builds the tiles of every product in a topological order (levels by increasing h, W
// before X21, then R, then the update) with their region dependencies.
bool build_dag(int64_t n, Dag &g, int &nrb, int &ncb, double &flops) {
    nrb = (int)cdiv(n, BM);
    ncb = (int)cdiv(n, BN);
    const int NR = nrb * ncb;
    std::vector<int> prod(3 * NR, -1);   // producing tile of each counter
    flops = 0.0;
    auto region = [&](int kind, int64_t r, int64_t cc) { return kind * NR + (int)(r / BM) * ncb + (int)(cc / BN); };
    auto pre_ready = [&](int kind, int64_t r, int64_t cc) { return kind == 0 && (r / 256) == (cc / BN); };
    bool bad = false;
    // Adds the regions of `kind` covering rows [r0, r1) x columns [c0, c1) to tile t.
    auto need = [&](int t, int kind, int64_t r0, int64_t r1, int64_t c0, int64_t c1) {
        r1 = std::min(r1, n);
        c1 = std::min(c1, n);
        for (int64_t r = r0 / BM * BM; r < r1; r += BM)
            for (int64_t cc = c0 / BN * BN; cc < c1; cc += BN) {
                if (pre_ready(kind, r, cc)) continue;
                const int f = region(kind, r, cc);
                if (prod[f] < 0) {
                    bad = true;
                    continue;
                }
                g.flag_deps[t].push_back(f);
                g.preds[t].push_back(prod[f]);
            }
    };
    auto add = [&](int op, int64_t am, int64_t ak, int64_t bk, int64_t bn, int64_t kb0, int64_t kb1, int64_t om,
                   int64_t on, int out_kind) {
        GTile tl{};
        tl.am = (int)am;
        tl.ak = (int)ak;
        tl.bk = (int)bk;
        tl.bn = (int)bn;
        tl.kb0 = (int)kb0;
        tl.kb1 = (int)kb1;
        tl.om = (int)om;
        tl.on = (int)on;
        tl.op = op;
        tl.out_flag = -1;
        tl.xin_flag = -1;
        g.tiles.push_back(tl);
        g.flag_deps.emplace_back();
        g.preds.emplace_back();
        const int terms = op == G_RES ? 6 : (op == G_UPD ? 1 : 3);
        g.kcost.push_back((int)(kb1 - kb0) * terms);
        const int t = (int)g.tiles.size() - 1;
        if (out_kind >= 0) {
            const int f = region(out_kind, om, on);
            g.tiles[t].out_flag = f;
            if (prod[f] >= 0) bad = true;   // every region has one producer
            prod[f] = t;
        }
        return t;
    };
    for (int64_t h = 256; h < n; h *= 2) {
        const int64_t P = level_pairs(n, h);
        for (int64_t q = 0; q < P; ++q) {
            const int64_t a0 = q * 2 * h, c0 = a0 + h, hc = std::min(h, n - c0);
            flops += 3.0 * (double)hc * h * (h + 1);
            // W = B X_A: rows of B (c0 ..), columns of X_A from the tile's column block.
            for (int64_t tn = 0; tn < h / BN; ++tn)
                for (int64_t tm = 0; tm < cdiv(hc, BM); ++tm) {
                    const int64_t kb0 = tn * BN / BK, kb1 = h / BK;
                    const int t = add(G_W, c0 + tm * BM, a0, a0, a0 + tn * BN, kb0, kb1, c0 + tm * BM,
                                      a0 + tn * BN, 1);
                    need(t, 0, a0 + kb0 * BK, a0 + kb1 * BK, a0 + tn * BN, a0 + tn * BN + BN);
                }
        }
        for (int64_t q = 0; q < P; ++q) {
            const int64_t a0 = q * 2 * h, c0 = a0 + h, hc = std::min(h, n - c0);
            flops += 3.0 * (double)h * hc * (hc + 1);
            // X21 = -X_C W: X_C rows of the tile, k over [c0, c0 + kend); W rows k.
            for (int64_t tm = 0; tm < cdiv(hc, BM); ++tm) {
                const int64_t kend = std::min((tm + 1) * BM, hc), kb1 = cdiv(kend, BK);
                for (int64_t tn = 0; tn < h / BN; ++tn) {
                    const int t = add(G_X21, c0 + tm * BM, c0, c0, a0 + tn * BN, 0, kb1, c0 + tm * BM,
                                      a0 + tn * BN, 0);
                    need(t, 0, c0 + tm * BM, c0 + tm * BM + BM, c0, c0 + kb1 * BK);
                    need(t, 1, c0, c0 + kb1 * BK, a0 + tn * BN, a0 + tn * BN + BN);
                }
            }
        }
    }
    // Newton-Schulz: R = I - T X (T needs no wait), then X += X R.
    const double lower_prod = (double)n * (n + 1) * (n + 2) / 3.0;
    flops += 7.0 * lower_prod;
    for (int pass = 0; pass < 2; ++pass)
        for (int64_t tm = 0; tm < cdiv(n, BM); ++tm) {
            const int64_t kend = std::min((tm + 1) * BM, n), kb1 = cdiv(kend, BK);
            for (int64_t tn = 0; tn * BN < kend; ++tn) {
                const int64_t kb0 = tn * BN / BK;
                if (pass == 0) {
                    const int t = add(G_RES, tm * BM, 0, 0, tn * BN, kb0, kb1, tm * BM, tn * BN, 2);
                    need(t, 0, kb0 * BK, kb1 * BK, tn * BN, tn * BN + BN);
                } else {
                    const int t = add(G_UPD, tm * BM, 0, 0, tn * BN, kb0, kb1, tm * BM, tn * BN, -1);
                    need(t, 0, tm * BM, tm * BM + BM, kb0 * BK, kb1 * BK);
                    need(t, 2, kb0 * BK, kb1 * BK, tn * BN, tn * BN + BN);
                    if (!pre_ready(0, tm * BM, tn * BN)) g.tiles[t].xin_flag = region(0, tm * BM, tn * BN);
                }
            }
        }
    return !bad;
}

// Critical-path list scheduling onto `ctas` persistent CTAs.  Cost model, in units of
// one pipeline slot (a 128 x 256 x 64 product): a tile occupies its CTA for its slots
// plus a small switch cost (the epilogue overlaps the next tile), and its region is
// ready for readers after its slots, its epilogue and the counter latency.  Returns the
// per-CTA lists (each a subsequence of one global topological order) and the makespan;
// *critical = longest dependency path, *work = total busy slots / ctas (both lower bounds).
double list_schedule(const Dag &g, int ctas, std::vector<std::vector<int>> &lists, double *critical,
                     double *work) {
    const int nt = (int)g.tiles.size();
    auto epi = [&](int op) { return op == G_X21 ? 10 : (op == G_UPD ? 12 : 6); };
    constexpr int kSwitch = 2, kLatency = 4;
    std::vector<std::vector<int>> succ(nt);
    std::vector<int> npred(nt, 0);
    for (int t = 0; t < nt; ++t) {
        std::vector<int> p = g.preds[t];
        std::sort(p.begin(), p.end());
        p.erase(std::unique(p.begin(), p.end()), p.end());
        npred[t] = (int)p.size();
        for (int x : p) succ[x].push_back(t);
    }
    // bottom level: longest path to the end, own cost included (tiles are topologically ordered)
    std::vector<double> bl(nt, 0.0);
    for (int t = nt - 1; t >= 0; --t) {
        double m = 0.0;
        for (int s : succ[t]) m = std::max(m, bl[s]);
        bl[t] = g.kcost[t] + epi(g.tiles[t].op) + kLatency + m;
    }
    *critical = 0.0;
    *work = 0.0;
    for (int t = 0; t < nt; ++t) {
        *critical = std::max(*critical, bl[t]);
        *work += (double)(g.kcost[t] + kSwitch) / ctas;
    }
    std::vector<double> ready_at(nt, 0.0);
    using RQ = std::pair<double, int>;   // (ready time, tile), min first
    std::priority_queue<RQ, std::vector<RQ>, std::greater<RQ>> pending;
    using AQ = std::pair<double, int>;   // (bottom level, -tile), max first
    std::priority_queue<AQ> avail;
    for (int t = 0; t < nt; ++t)
        if (npred[t] == 0) pending.push({0.0, t});
    std::priority_queue<RQ, std::vector<RQ>, std::greater<RQ>> procs;
    for (int b = 0; b < ctas; ++b) procs.push({0.0, b});
    lists.assign(ctas, {});
    double makespan = 0.0;
    for (int done = 0; done < nt; ++done) {
        RQ pr = procs.top();
        procs.pop();
        double now = pr.first;
        while (!pending.empty() && pending.top().first <= now) {
            avail.push({bl[pending.top().second], -pending.top().second});
            pending.pop();
        }
        if (avail.empty()) {
            now = pending.top().first;
            while (!pending.empty() && pending.top().first <= now) {
                avail.push({bl[pending.top().second], -pending.top().second});
                pending.pop();
            }
        }
        const int t = -avail.top().second;
        avail.pop();
        lists[pr.second].push_back(t);
        const double busy = now + g.kcost[t] + kSwitch;
        const double ready = now + g.kcost[t] + epi(g.tiles[t].op) + kLatency;
        makespan = std::max(makespan, ready);
        procs.push({busy, pr.second});
        for (int s : succ[t]) {
            ready_at[s] = std::max(ready_at[s], ready);
            if (--npred[s] == 0) pending.push({ready_at[s], s});
        }
    }
    return makespan;
}

// Host half of a plan: per-CTA lists (concatenated), offsets and counter indices.
struct HostPlan {
    std::vector<GTile> tiles;
    std::vector<int> off, deps;
    int ctas = 0, nrb = 0, ncb = 0, edges = 0;
    double flops = 0.0, makespan = 0.0, critical = 0.0, work = 0.0;
};

bool make_host_plan(int64_t n, int sm_count, HostPlan &hp) {
    Dag g;
    if (!build_dag(n, g, hp.nrb, hp.ncb, hp.flops)) return false;
    const int nt = (int)g.tiles.size();
    hp.ctas = std::max(1, std::min(sm_count, nt));
    std::vector<std::vector<int>> lists;
    hp.makespan = list_schedule(g, hp.ctas, lists, &hp.critical, &hp.work);
    hp.tiles.clear();
    hp.off.clear();
    hp.deps.clear();
    hp.tiles.reserve(nt);
    for (int b = 0; b < hp.ctas; ++b) {
        hp.off.push_back((int)hp.tiles.size());
        for (int t : lists[b]) {
            GTile tl = g.tiles[t];
            std::vector<int> f = g.flag_deps[t];
            std::sort(f.begin(), f.end());
            f.erase(std::unique(f.begin(), f.end()), f.end());
            tl.dep0 = (int)hp.deps.size();
            hp.deps.insert(hp.deps.end(), f.begin(), f.end());
            tl.dep1 = (int)hp.deps.size();
            hp.tiles.push_back(tl);
        }
    }
    hp.off.push_back((int)hp.tiles.size());
    hp.edges = (int)hp.deps.size();
    return true;
}

// Replays the lists as the device runs them (each CTA strictly in order, a tile may
// start once every counter it waits on is complete) and reports whether all tiles
// finish: the lists admit no circular wait when all CTAs are resident.
bool replay_ok(const HostPlan &hp) {
    std::vector<char> done_flag(3 * (size_t)hp.nrb * hp.ncb + 1, 0);
    std::vector<int> pos(hp.ctas);
    for (int b = 0; b < hp.ctas; ++b) pos[b] = hp.off[b];
    size_t left = hp.tiles.size();
    while (left > 0) {
        bool progress = false;
        for (int b = 0; b < hp.ctas; ++b) {
            while (pos[b] < hp.off[b + 1]) {
                const GTile &tl = hp.tiles[pos[b]];
                bool ready = true;
                for (int d = tl.dep0; d < tl.dep1 && ready; ++d) ready = done_flag[hp.deps[d]] != 0;
                if (tl.xin_flag >= 0 && !done_flag[tl.xin_flag]) ready = false;
                if (!ready) break;
                if (tl.out_flag >= 0) {
                    if (done_flag[tl.out_flag]) return false;   // two producers
                    done_flag[tl.out_flag] = 1;
                }
                ++pos[b];
                --left;
                progress = true;
            }
        }
        if (!progress) return false;
    }
    return true;
}

std::mutex g_mu;
std::map<std::pair<int, int64_t>, GraphPlan> g_plans;

// Device timeline of the last graph launch made while tracing.
struct Timeline {
    unsigned long long *d = nullptr;
    int ntiles = 0, dev = -1;
};
std::mutex g_tl_mu;
std::map<std::pair<int, int64_t>, Timeline> g_timelines;
Timeline g_last_tl;

}  // namespace

size_t graph_flag_bytes(int64_t n) {
    const int64_t nrb = cdiv(n, BM), ncb = cdiv(n, BN);
    return (size_t)(3 * nrb * ncb + 1) * sizeof(int);
}

tri_status graph_plan(int dev, int sm_count, int64_t n, const GraphPlan **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_pair(dev, n);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) {
        *out = &it->second;
        return TRI_OK;
    }
    HostPlan hp;
    if (!make_host_plan(n, sm_count, hp)) return TRI_ERR_UNSUPPORTED;
    GraphPlan p;
    p.nrb = hp.nrb;
    p.ncb = hp.ncb;
    p.flops = hp.flops;
    p.model_makespan = hp.makespan;
    if (hp.deps.empty()) hp.deps.push_back(0);
    const size_t tb = hp.tiles.size() * sizeof(GTile), ob = hp.off.size() * sizeof(int),
                 db = hp.deps.size() * sizeof(int);
    uint8_t *d = nullptr;
    if (cudaMalloc(&d, tb + ob + db) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_NOMEM;
    }
    if (cudaMemcpy(d, hp.tiles.data(), tb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d + tb, hp.off.data(), ob, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d + tb + ob, hp.deps.data(), db, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return TRI_ERR_CUDA;
    }
    p.d_tiles = (GTile *)d;
    p.d_off = (int *)(d + tb);
    p.d_deps = (int *)(d + tb + ob);
    p.ctas = hp.ctas;
    p.ntiles = (int)hp.tiles.size();
    auto res = g_plans.emplace(key, p);
    *out = &res.first->second;
    return TRI_OK;
}

cudaError_t launch_graph(const Ctx &c, bool trans, bool unit, int64_t n, const GraphPlan &p,
                         const __nv_bfloat16 *const tpl[3], const GEpi &ep) {
    const int64_t ldp = ep.ldp;
    GMaps maps;
    memset(&maps, 0, sizeof(maps));
    const __nv_bfloat16 *bsrc[6] = {ep.xp0, ep.xp1, ep.xp2, ep.wp0, ep.wp1, ep.rp};
    const __nv_bfloat16 *asrc[6] = {tpl[0], tpl[1], tpl[2], ep.xp0, ep.xp1, ep.xp2};
    for (int i = 0; i < 6; ++i) {
        if (!encode_plane(&maps.a[i], Plane{asrc[i], n, n, ldp}, 64, 64)) return cudaErrorInvalidValue;
        if (!encode_plane(&maps.b[i], Plane{bsrc[i], n, n, ldp}, 64, BN)) return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaMemsetAsync(ep.flags, 0, graph_flag_bytes(n), c.stream);
    if (e != cudaSuccess) return e;
    GEpi epl = ep;
    epl.timeline = nullptr;
    // Failure-path test knobs (unset in normal use): TRI_DEBUG_WITHHOLD = a ready counter
    // that is never published, TRI_DEBUG_WAIT_LIMIT_US = the deadline of every wait.
    if (const char *w = std::getenv("TRI_DEBUG_WITHHOLD")) epl.withhold = std::atoi(w);
    if (const char *l = std::getenv("TRI_DEBUG_WAIT_LIMIT_US")) {
        const long long us = std::atoll(l);
        if (us > 0) epl.limit_ns = (unsigned long long)us * 1000ull;
    }
    if (trace_on()) {
        std::lock_guard<std::mutex> lk(g_tl_mu);
        Timeline &tl = g_timelines[std::make_pair(c.device, n)];
        if (!tl.d) {
            if (cudaMalloc(&tl.d, (size_t)p.ntiles * kTimelineWords * 8) != cudaSuccess) {
                cudaGetLastError();
                tl.d = nullptr;
            }
            tl.ntiles = p.ntiles;
            tl.dev = c.device;
        }
        if (tl.d) {
            epl.timeline = tl.d;
            g_last_tl = tl;
        }
    }
    TraceScope ts(c.stream, "tc_graph", p.flops, 0.0);
    if (trans) return unit ? launch_g<true, true>(c, maps, p, epl) : launch_g<true, false>(c, maps, p, epl);
    return unit ? launch_g<false, true>(c, maps, p, epl) : launch_g<false, false>(c, maps, p, epl);
}

}  // namespace tc
}  // namespace triinv

// Host-only inspection of the mixed path's tensor-core schedule (no device needed).
extern "C" tri_status tri_mixed_schedule_stats(int64_t n, int ctas, double *stats, int nstats) {
    using namespace triinv::tc;
    if (n <= 256 || ctas < 1 || !stats || nstats < 8) return TRI_ERR_ARG;
    if (n > (1ll << 20)) return TRI_ERR_UNSUPPORTED;
    HostPlan hp;
    if (!make_host_plan(n, ctas, hp)) return TRI_ERR_UNSUPPORTED;
    stats[0] = (double)hp.tiles.size();
    stats[1] = (double)hp.edges;
    stats[2] = hp.makespan;
    stats[3] = hp.critical;
    stats[4] = hp.work;
    stats[5] = replay_ok(hp) ? 1.0 : 0.0;
    stats[6] = hp.flops;
    stats[7] = (double)hp.ctas;
    return TRI_OK;
}

// Copies the per-tile timeline of the last mixed-path launch made while tracing.
extern "C" int64_t tri_trace_timeline(unsigned long long *buf, size_t cap_words) {
    using namespace triinv::tc;
    Timeline tl;
    {
        std::lock_guard<std::mutex> lk(g_tl_mu);
        tl = g_last_tl;
    }
    if (!tl.d) return 0;
    const size_t words = (size_t)tl.ntiles * kTimelineWords;
    if (buf && cap_words) {
        int cur = 0;
        if (cudaGetDevice(&cur) != cudaSuccess || cudaSetDevice(tl.dev) != cudaSuccess) return -1;
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(buf, tl.d, std::min(words, cap_words) * 8, cudaMemcpyDeviceToHost);
        cudaSetDevice(cur);
        if (e != cudaSuccess) return -1;
    }
    return (int64_t)tl.ntiles;
}
