// gemm_tc.cu -- the generic product C = alpha * A * B + beta * C on the tensor cores with
// split-BF16 operands (mixed precision).  Both FP32 operands are split into BF16 planes
// (x = hi + mid [+ lo]) with the operand's triangle applied, and the requested pieces are
// accumulated in FP32: 1 term hi*hi, 3 terms hi*hi + hi*mid + mid*hi (about 2^-16
// relative), 6 terms adding hi*lo + mid*mid + lo*hi (about 2^-24).
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
                              int64_t ldp, bool trans);

namespace {

int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
size_t al256(size_t x) { return (x + 255) / 256 * 256; }

struct TileList {
    tc::Tile *d_tiles;
    int *d_off;
    int ctas;
};

std::mutex g_tl_mu;
std::map<std::tuple<int, int64_t, int64_t, int64_t, int, int, int, int>, TileList> g_tl;

bool is_low(int k) { return k == OP_LOWER || k == OP_LOWER_UNIT; }
bool is_up(int k) { return k == OP_UPPER || k == OP_UPPER_UNIT; }

cudaError_t tile_list(const Ctx &c, const GemmArgs &g, int terms, TileList *out) {
    auto key = std::make_tuple(c.device, g.m, g.n, g.k, g.akind, g.bkind, g.cmask, terms);
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

size_t gemm_tc_ws_bytes(int64_t m, int64_t n, int64_t k) {
    const int64_t lda = rup(std::max<int64_t>(m, 1), 64), ldb = rup(std::max<int64_t>(k, 1), 64);
    return 3 * al256((size_t)lda * k * 2) + 3 * al256((size_t)ldb * n * 2);
}

cudaError_t gemm_tc(const Ctx &c, const GemmArgs &g, int terms, void *ws, const char *trace_name) {
    if (g.m <= 0 || g.n <= 0) return cudaSuccess;
    if (g.batch > 1) {
        // One product per batch element (the planes of one element at a time).
        GemmArgs one = g;
        one.batch = 1;
        for (int64_t b = 0; b < g.batch; ++b) {
            one.a = (const uint8_t *)g.a + b * g.sa * 4;
            one.b = (const uint8_t *)g.b + b * g.sb * 4;
            one.c = (uint8_t *)g.c + b * g.sc * 4;
            cudaError_t e = gemm_tc(c, one, terms, ws, trace_name);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (terms != 1 && terms != 3 && terms != 6) return cudaErrorInvalidValue;
    const int64_t lda = rup(g.m, 64), ldb = rup(g.k, 64);
    uint8_t *base = (uint8_t *)ws;
    const size_t pa = al256((size_t)lda * g.k * 2), pb = al256((size_t)ldb * g.n * 2);
    __nv_bfloat16 *A[3], *B[3];
    for (int i = 0; i < 3; ++i) {
        A[i] = (__nv_bfloat16 *)(base + i * pa);
        B[i] = (__nv_bfloat16 *)(base + 3 * pa + i * pb);
    }
    const bool three = terms == 6;
    cudaError_t e = launch_split_rect(c, (const float *)g.a, g.lda, g.m, g.k, g.akind, A[0], A[1],
                                      three ? A[2] : nullptr, lda, g.ta);
    if (e != cudaSuccess) return e;
    e = launch_split_rect(c, (const float *)g.b, g.ldb, g.k, g.n, g.bkind, B[0], B[1],
                          three ? B[2] : nullptr, ldb, g.tb);
    if (e != cudaSuccess) return e;
    TileList tl;
    e = tile_list(c, g, terms, &tl);
    if (e != cudaSuccess) return e;
    tc::Plane ap[3], bp[3];
    for (int i = 0; i < 3; ++i) {
        ap[i] = tc::Plane{A[i], g.m, g.k, lda};
        bp[i] = tc::Plane{B[i], g.k, g.n, ldb};
    }
    tc::Terms t1{1, {0}, {0}};
    tc::Terms t3{3, {0, 0, 1}, {0, 1, 0}};
    tc::Terms t6{6, {0, 0, 1, 0, 1, 2}, {0, 1, 0, 2, 1, 0}};
    const tc::Terms &tt = terms == 1 ? t1 : (terms == 3 ? t3 : t6);
    tc::Epi ep{(float *)g.c, g.ldc, nullptr, nullptr, nullptr, 0, g.m, g.n};
    ep.alpha = (float)g.alpha;
    ep.beta = (float)g.beta;
    ep.cmask = g.cmask;
    return tc::launch_tc(c, tc::MODE_GEN, false, false, ap, three ? 3 : 2, bp, three ? 3 : 2, tt,
                         tl.d_tiles, tl.d_off, tl.ctas, ep, terms * gemm_flops(g), trace_name);
}

}  // namespace triinv
