// gemm_tc.cu -- the generic product C = alpha * A * B + beta * C on the tensor cores with
// split-BF16 operands (mixed precision).  Both FP32 operands are split into BF16 planes
// (x = hi + mid [+ lo]) with the operand's triangle applied, and the requested pieces are
// accumulated in FP32: 1 term hi*hi, 3 terms hi*hi + hi*mid + mid*hi (about 2^-16
// relative), 6 terms adding hi*lo + mid*mid + lo*hi (about 2^-24; all six read from
// one fused pipeline stage, partial sums promoted to FP32 registers every 64 k).
// Tile lists depend on the shape and the triangle kinds only and are cached per device.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "gemm.cuh"
#include "tc_gemm.cuh"

namespace triinv {

cudaError_t launch_split_rect(const Ctx &c, const float *a, int64_t lds, int64_t rows, int64_t cols,
                              int kind, __nv_bfloat16 *p0, __nv_bfloat16 *p1, __nv_bfloat16 *p2,
                              int64_t ldp, bool trans, int64_t batch, int64_t as_, int64_t ps);

namespace {

int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
size_t al256(size_t x) { return (x + 255) / 256 * 256; }

struct TileList {
    tc::Tile *d_tiles;
    int *d_off;
    int ctas;
};

std::mutex g_tl_mu;
std::map<std::tuple<int, int64_t, int64_t, int64_t, int, int, int, int, int64_t>, TileList> g_tl;

// Matrices per chunk of a batched product: operand planes of at most kChunkBytes at a time.
constexpr size_t kChunkBytes = size_t(4) << 30;

bool is_low(int k) { return k == OP_LOWER || k == OP_LOWER_UNIT; }
bool is_up(int k) { return k == OP_UPPER || k == OP_UPPER_UNIT; }

cudaError_t tile_list(const Ctx &c, const GemmArgs &g, int terms, int64_t batch, TileList *out) {
    auto key = std::make_tuple(c.device, g.m, g.n, g.k, g.akind, g.bkind, g.cmask, terms, batch);
    std::lock_guard<std::mutex> lk(g_tl_mu);
    auto it = g_tl.find(key);
    if (it != g_tl.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    std::vector<tc::Tile> v;
    for (int64_t m0 = 0; m0 < g.m; m0 += tc::BM) {
        for (int64_t n0 = 0; n0 < g.n; n0 += tc::BN) {
            if ((g.cmask == OP_LOWER || g.cmask == OP_LOWER_UNIT) && n0 > m0 + tc::BM - 1) continue;
            if ((g.cmask == OP_UPPER || g.cmask == OP_UPPER_UNIT) && m0 > n0 + tc::BN - 1) continue;
            int64_t kbeg = 0, kend = g.k;
            if (is_low(g.akind)) kend = std::min(kend, m0 + tc::BM);
            if (is_up(g.akind)) kbeg = std::max(kbeg, m0);
            if (is_low(g.bkind)) kbeg = std::max(kbeg, n0);
            if (is_up(g.bkind)) kend = std::min(kend, n0 + tc::BN);
            const int kb0 = (int)(kbeg / tc::BK), kb1 = (int)((kend + tc::BK - 1) / tc::BK);
            if (kb0 >= kb1) return cudaErrorInvalidValue;   // no product has an empty k range
            v.push_back(tc::Tile{(int)m0, 0, 0, (int)n0, kb0, kb1, (int)m0, (int)n0});
        }
    }
    const size_t one = v.size();
    for (int64_t b = 1; b < batch; ++b)
        for (size_t i = 0; i < one; ++i) {
            tc::Tile t = v[i];
            t.b = (int)b;
            v.push_back(t);
        }
    std::vector<int> off;
    const int ctas = tc::schedule_lpt(v, terms, c.sm_count, off);
    const size_t tb = v.size() * sizeof(tc::Tile), ob = off.size() * sizeof(int);
    uint8_t *d = nullptr;
    if (cudaMalloc(&d, tb + ob) != cudaSuccess) return cudaErrorMemoryAllocation;
    if (cudaMemcpy(d, v.data(), tb, cudaMemcpyHostToDevice) != cudaSuccess) return cudaErrorUnknown;
    if (cudaMemcpy(d + tb, off.data(), ob, cudaMemcpyHostToDevice) != cudaSuccess) return cudaErrorUnknown;
    TileList t{(tc::Tile *)d, (int *)(d + tb), ctas};
    g_tl.emplace(key, t);
    *out = t;
    return cudaSuccess;
}

}  // namespace

namespace {

size_t per_matrix_ws(int64_t m, int64_t n, int64_t k) {
    const int64_t lda = rup(std::max<int64_t>(m, 1), 64), ldb = rup(std::max<int64_t>(k, 1), 64);
    return 3 * al256((size_t)lda * k * 2) + 3 * al256((size_t)ldb * n * 2);
}

int64_t chunk_of(int64_t m, int64_t n, int64_t k, int64_t batch) {
    return std::max<int64_t>(1, std::min<int64_t>(batch, (int64_t)(kChunkBytes / per_matrix_ws(m, n, k))));
}

}  // namespace

size_t gemm_tc_ws_bytes(int64_t m, int64_t n, int64_t k, int64_t batch) {
    return per_matrix_ws(m, n, k) * (size_t)chunk_of(m, n, k, std::max<int64_t>(batch, 1));
}

cudaError_t gemm_tc(const Ctx &c, const GemmArgs &g, int terms, void *ws, const char *trace_name) {
    if (g.m <= 0 || g.n <= 0 || g.batch <= 0) return cudaSuccess;
    if (g.batch2 > 1) return cudaErrorInvalidValue;
    if (terms != 1 && terms != 3 && terms != 6) return cudaErrorInvalidValue;
    if (g.batch > 65535) return cudaErrorInvalidValue;
    // Each chunk of the batch: split every operand of the chunk into planes (one launch per
    // operand), then one persistent tensor-core launch over the tiles of all its matrices.
    const int64_t cb = chunk_of(g.m, g.n, g.k, g.batch);
    const int64_t lda = rup(g.m, 64), ldb = rup(g.k, 64);
    const size_t pa = al256((size_t)lda * g.k * 2), pb = al256((size_t)ldb * g.n * 2);
    for (int64_t b0 = 0; b0 < g.batch; b0 += cb) {
        const int64_t nb = std::min(cb, g.batch - b0);
        uint8_t *base = (uint8_t *)ws;
        __nv_bfloat16 *A[3], *B[3];
        for (int i = 0; i < 3; ++i) {
            A[i] = (__nv_bfloat16 *)(base + (size_t)i * nb * pa);
            B[i] = (__nv_bfloat16 *)(base + 3 * (size_t)nb * pa + (size_t)i * nb * pb);
        }
        const bool three = terms == 6;
        const float *ga = (const float *)g.a + b0 * g.sa, *gb = (const float *)g.b + b0 * g.sb;
        float *gc = (float *)g.c + b0 * g.sc;
        cudaError_t e = launch_split_rect(c, ga, g.lda, g.m, g.k, g.akind, A[0], A[1], three ? A[2] : nullptr, lda,
                                          g.ta, nb, g.sa, (int64_t)(pa / 2));
        if (e != cudaSuccess) return e;
        e = launch_split_rect(c, gb, g.ldb, g.k, g.n, g.bkind, B[0], B[1], three ? B[2] : nullptr, ldb, g.tb, nb, g.sb,
                              (int64_t)(pb / 2));
        if (e != cudaSuccess) return e;
        TileList tl;
        e = tile_list(c, g, terms, nb, &tl);
        if (e != cudaSuccess) return e;
        tc::Plane ap[3], bp[3];
        for (int i = 0; i < 3; ++i) {
            ap[i] = tc::Plane{A[i], g.m, g.k, lda};
            bp[i] = tc::Plane{B[i], g.k, g.n, ldb};
            ap[i].batch = bp[i].batch = nb;
            ap[i].bstride = (int64_t)(pa / 2);
            bp[i].bstride = (int64_t)(pb / 2);
        }
        tc::Terms t1{1, {0}, {0}};
        tc::Terms t3{3, {0, 0, 1}, {0, 1, 0}};
        tc::Terms t6{6, {0, 0, 1, 0, 1, 2}, {0, 1, 0, 2, 1, 0}};
        const tc::Terms &tt = terms == 1 ? t1 : (terms == 3 ? t3 : t6);
        tc::Epi ep{gc, g.ldc, nullptr, nullptr, nullptr, 0, g.m, g.n};
        ep.alpha = (float)g.alpha;
        ep.beta = (float)g.beta;
        ep.cmask = g.cmask;
        ep.dadd = (float)g.dadd;
        ep.xs = g.sc;
        e = tc::launch_tc(c, three ? tc::MODE_GENP : tc::MODE_GEN, false, false, ap, three ? 3 : 2, bp,
                          three ? 3 : 2, tt, tl.d_tiles, tl.d_off, tl.ctas, ep, (double)nb * terms * gemm_flops(g),
                          trace_name);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace triinv
