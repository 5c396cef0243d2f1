// tc_gemm.cu -- K3 host side: tensor maps, longest-first tile schedules and the launch of
// the tcgen05 split-BF16 product kernel (tc_kernel.cuh) for every mode; the CTA-pair
// launches are instantiated in tc_gemm_pair.cu.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "tc_kernel.cuh"

namespace triinv {
namespace tc {
namespace {

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

int schedule_lpt_groups(std::vector<Tile> &tiles, const std::vector<int> &group, int terms, int ctas,
                        std::vector<int> &offsets) {
    const int nt = (int)tiles.size();
    if (ctas > nt) ctas = nt;
    if (ctas < 1) ctas = 1;
    constexpr int kEpilogueCost = 8;   // pipeline-slot equivalents per tile (as schedule_lpt)
    auto cost = [&](int i) { return (tiles[i].kb1 - tiles[i].kb0) * terms + kEpilogueCost; };
    std::vector<int> order(nt);
    for (int i = 0; i < nt; ++i) order[i] = i;
    // by group, then longest first
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return group[x] != group[y] ? group[x] < group[y] : cost(x) > cost(y);
    });
    std::vector<std::pair<long long, int>> heap;
    for (int b = 0; b < ctas; ++b) heap.push_back({0, b});
    auto cmp = [](const std::pair<long long, int> &x, const std::pair<long long, int> &y) {
        return x.first > y.first || (x.first == y.first && x.second > y.second);
    };
    std::make_heap(heap.begin(), heap.end(), cmp);
    std::vector<std::vector<int>> lists(ctas);
    for (int i : order) {   // each CTA's list stays in group order
        std::pop_heap(heap.begin(), heap.end(), cmp);
        auto &top = heap.back();
        lists[top.second].push_back(i);
        top.first += cost(i);
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
                      const char *trace_name, int bn, bool pair, const Epi *epi2) {
    if (ctas <= 0) return cudaSuccess;
    const bool lvl = mode == MODE_LVL;
    if (lvl ? (na != 4 || nb != 4 || bn != 128 || pair || !epi2 || !epi.cnt)
            : (na < 1 || na > 3 || nb < 1 || nb > 3))
        return cudaErrorInvalidValue;
    if (terms.n < 1 || terms.n > 6 || (lvl && terms.n != 3)) return cudaErrorInvalidValue;
    const Epi &e2 = epi2 ? *epi2 : epi;
    // narrow tiles are built for the level products only
    const bool level = mode == MODE_W || mode == MODE_X21 || mode == MODE_W6 || mode == MODE_X216 || lvl;
    if (bn != BN && !((bn == 128 || bn == 64) && level)) return cudaErrorInvalidValue;
    // CTA pairs: the products of the mixed path, full-width tiles
    if (pair && !(bn == BN && (mode == MODE_W || mode == MODE_X21 || mode == MODE_RES || mode == MODE_UPD)))
        return cudaErrorInvalidValue;
    const int bcols = pair ? bn / 2 : bn;   // B columns one CTA stages
    Maps maps;
    memset(&maps, 0, sizeof(maps));
    const Cfg cf = cfg_for(mode, bn);
    for (int i = 0; i < 4; ++i) {
        const Plane &pa = aplanes[i < na ? i : 0];
        const Plane &pb = bplanes[i < nb ? i : 0];
        if (!encode_plane(&maps.a[i], pa, 64, cf.ks)) return cudaErrorInvalidValue;
        if (!encode_plane(&maps.b[i], pb, cf.ks, bcols, cf.ks == 32)) return cudaErrorInvalidValue;
    }
    // Stage layout: every distinct plane the terms read (fused), or one term's pair.
    Pipe pipe{1, 1, 0, 0, 0};
    for (int j = 0; j < terms.n; ++j) {
        // MODE_LVL: the X21 tiles use the W terms' planes shifted by two
        const int ra = lvl ? na - 2 : na, rb = lvl ? nb - 2 : nb;
        if (terms.a[j] < 0 || terms.a[j] >= ra || terms.b[j] < 0 || terms.b[j] >= rb) return cudaErrorInvalidValue;
        if (cf.fused) {
            pipe.na = std::max(pipe.na, terms.a[j] + 1);
            pipe.nb = std::max(pipe.nb, terms.b[j] + 1);
        }
    }
    pipe.stage_bytes = (pipe.na * BM + pipe.nb * bcols) * cf.ks * 2;
    pipe.batched = aplanes[0].batch > 1 ? 1 : 0;
    for (int i = 0; i < na; ++i)
        if ((aplanes[i].batch > 1) != (pipe.batched != 0)) return cudaErrorInvalidValue;
    for (int i = 0; i < nb; ++i)
        if ((bplanes[i].batch > 1) != (pipe.batched != 0)) return cudaErrorInvalidValue;
    pipe.stages = std::min(MAX_STAGES, STAGE_BUDGET / pipe.stage_bytes);
    TraceScope ts(c.stream, trace_name, flops, 0.0);
    if (pair) return launch_pair(c, mode, trans, unit, maps, terms, pipe, d_tiles, d_off, ctas, epi);
#define TRI_TC_CASE_N(M, N)                                                                   \
        if (trans) return unit ? launch_t<M, true, true, N>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi, e2)   \
                               : launch_t<M, true, false, N>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi, e2); \
        return unit ? launch_t<M, false, true, N>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi, e2)             \
                    : launch_t<M, false, false, N>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi, e2);
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
        case MODE_LVL:
            TRI_TC_CASE_N(MODE_LVL, 128)
        TRI_TC_CASE(MODE_RES)
        TRI_TC_CASE(MODE_UPD)
        case MODE_F32:
            return launch_t<MODE_F32, false, false>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi, e2);
        case MODE_GEN:
            return launch_t<MODE_GEN, false, false>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi, e2);
        case MODE_GENP:
            return launch_t<MODE_GENP, false, false>(c, maps, terms, pipe, d_tiles, d_off, ctas, epi, e2);
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
