// mixed.cu -- the TRI_F32_MIXED path: recursive split with split-BF16 tensor-core
// products, followed by one Newton-Schulz step.
//
// 1. T (FP32) -> BF16 planes T_hi, T_mid, T_lo                       (split.cu)
// 2. every 256 x 256 diagonal block is inverted in FP32 by one CTA in shared memory
//    (CRIT leaves of 32, split levels 32..128) and written with its BF16 planes
//    X_hi, X_mid, X_lo                                                 (batched.cu)
// 4. split levels h = 256, 512, ...: for every pair (block inverse of the proof of the
//    main Theorem, Section 3; Algorithm COMBRIT with two blocks, Section 4.1)
//        W   = B X_A       3 terms  hi*hi + hi*mid + mid*hi   -> W_hi, W_mid
//        X21 = -X_C W      3 terms                              -> X (FP32) and its planes
// 5. Newton-Schulz step X <- X (2I - T X) = X + X R:
//        R = I - T X       6 terms (hh, hm, mh, hl, mm, lh) with FP32 promotion of the
//                          tensor-core partial sums every 64 k: R is a difference of
//                          nearly equal terms and needs ~2^-24 relative accuracy
//        X += X R          1 term: R is as small as the forward residual (~3e-8
//                          normwise at n = 8192), so the BF16 error 2^-8 |X R| of the
//                          update adds ~1e-10, far below FP32 rounding
// Direct recipe (tri_set_mixed_recipe(TRI_RECIPE_DIRECT)): the level products of step 4
// take all six terms with FP32 promotion every 64 k (FP32-class products, W with its lo
// plane) and step 5 is left out.
// Steps 4 and 5 run either as one persistent tensor-core launch per product (default),
// with the low levels h = 256 .. 1024 in one dependency-ordered launch
// (TRI_MIXED_SCHEDULE=merged), or as a single launch that follows the data dependencies
// tile by tile (tc_graph.cu, TRI_MIXED_SCHEDULE=graph).  Tile lists and schedules depend
// on n only and are built once per (device, n).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <mutex>
#include <vector>

#include "tc_graph.cuh"
#include "tc_ptx.cuh"

namespace triinv {

cudaError_t launch_split_planes(const Ctx &c, bool trans, bool unit, bool diag_only, int64_t n,
                                const float *a, int64_t lda, __nv_bfloat16 *p0, __nv_bfloat16 *p1,
                                __nv_bfloat16 *p2, int64_t ldp, bool skip_diag, int64_t batch, int64_t as_,
                                int64_t ps, int lmin = 0, int lmax = 62);
cudaError_t launch_diag_blocks(const Ctx &c, bool trans, bool unit, int64_t n, float *a, int64_t lda,
                               __nv_bfloat16 *p0, __nv_bfloat16 *p1, __nv_bfloat16 *p2, int64_t ldp,
                               __nv_bfloat16 *q0, __nv_bfloat16 *q1, __nv_bfloat16 *q2, int64_t batch,
                               int64_t as_, int64_t ps, int64_t index0, float tau, int *flags);

// Per-device side stream and events used to run two independent kernels concurrently
// (fork / join through events, so the pair also works inside stream capture).
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, join2 = nullptr;
    cudaEvent_t lev[24] = {};   // per split level, when the input arrives by level (InputFeed)
};
std::mutex g_side_mu;
SideStream g_side[64];

// Caller holds g_side_mu for the whole fork / launch / join sequence, so concurrent
// calls from several host threads never interleave their event records.
bool side_stream(int dev, SideStream **out) {
    SideStream &ss = g_side[dev];
    if (!ss.s) {
        if (cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking) != cudaSuccess) return false;
        if (cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming) != cudaSuccess) return false;
        if (cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming) != cudaSuccess) return false;
        if (cudaEventCreateWithFlags(&ss.join2, cudaEventDisableTiming) != cudaSuccess) return false;
        for (cudaEvent_t &e : ss.lev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
    }
    *out = &ss;
    return true;
}

namespace {

constexpr int64_t kDiag = 256;      // diagonal blocks inverted on CUDA cores
constexpr int64_t kLeaf = 64;

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
int64_t cdiv(int64_t x, int64_t m) { return (x + m - 1) / m; }

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// Matrices per workspace chunk of a batch: the planes of at most kChunkBytes at a time.
constexpr size_t kChunkBytes = size_t(8) << 30;

struct Layout {
    int64_t ldp;
    size_t plane;                 // bytes of one plane of one matrix (256-aligned)
    int64_t batch;                // matrices whose planes the workspace holds
    size_t off_t, off_x, off_r, off_w, off_f, off_g, off_c, off_m, total;
    size_t mplane;                // bytes of one merged-level W plane of one matrix
};

// Under the "merged" schedule the low split levels h = 256 .. kMergedMax (h < n) run as
// one launch whose tiles wait on dependency counters: two per pair and level (its W tiles
// done, its X21 tiles done).
constexpr int64_t kMergedMax = 1024;
bool use_merged_levels();
int64_t merged_counters(int64_t n) {
    if (!use_merged_levels()) return 0;
    int64_t c = 0;
    for (int64_t h = kDiag; h <= kMergedMax && h < n; h *= 2) c += 2 * level_pairs(n, h);
    return c;
}
// W of the merged levels: one wld x wcols matrix (ld = wld), level h in columns of its own.
void merged_w_dims(int64_t n, int64_t *wld, int64_t *wcols) {
    *wld = 0;
    *wcols = 0;
    if (!use_merged_levels()) return;
    for (int64_t h = kDiag; h <= kMergedMax && h < n; h *= 2) {
        *wld = h;
        *wcols += level_pairs(n, h) * h;
    }
}

// Workspace: T planes (3), X planes (3), R plane, W planes (3; single matrix: at the
// positions of the B blocks of T; batch: the compact h x P*h level layout), each a group of
// `batch` planes, then the ready counters of the single-launch schedule, then one growth
// flag per diagonal block of every matrix, then the dependency counters of the merged
// low levels of every matrix, then their two W planes (hi, mid) per matrix.
Layout layout(int64_t n, int64_t batch = 1) {
    Layout L{};
    L.ldp = round_up(std::max<int64_t>(n, 1), 64);
    L.plane = al256((size_t)L.ldp * (size_t)n * 2);
    L.batch = batch;
    const size_t g = L.plane * (size_t)batch;
    L.off_t = 0;
    L.off_x = L.off_t + 3 * g;
    L.off_r = L.off_x + 3 * g;
    L.off_w = L.off_r + g;
    L.off_f = L.off_w + 3 * g;
    L.off_g = L.off_f + al256(tc::graph_flag_bytes(n));
    L.off_c = L.off_g + al256((size_t)((n + kDiag - 1) / kDiag) * (size_t)batch * sizeof(int));
    L.off_m = L.off_c + al256((size_t)merged_counters(n) * (size_t)batch * sizeof(int));
    int64_t wld = 0, wcols = 0;
    merged_w_dims(n, &wld, &wcols);
    L.mplane = al256((size_t)wld * (size_t)wcols * 2);
    L.total = L.off_m + 2 * L.mplane * (size_t)batch;
    return L;
}

int64_t chunk_matrices(int64_t n, int64_t batch) {
    const size_t per = 10 * layout(n).plane;
    return std::max<int64_t>(1, std::min<int64_t>(batch, (int64_t)(kChunkBytes / per)));
}

struct Launch {
    int first, ctas, off_first;   // tiles from `first`, CTA offsets from `off_first`
    double flops;
    int bn = tc::BN;              // output tile width the tiles were cut with
    bool pair = false;            // 256-row tiles for clusters of two CTAs
};

// Products run by CTA pairs (tc_gemm_pair.cu, tri_set_cta_pairs).
constexpr int kPairLevels = TRI_PAIR_LEVELS, kPairRes = TRI_PAIR_RES, kPairUpd = TRI_PAIR_UPD;

// Output tile width of the level products at split half-size h.  A level's products
// are P = n / 2h pairs of h x h "triangular x full" products; with 128 x 256 tiles the low
// levels have few tiles (h = 256: 32 tiles for 152 SMs) whose k range sets the launch's
// length, so narrower tiles spread them over more SMs and shorten the longest tile.
// TRI_LEVEL_TILE_N="h:bn,..." (bn in {64, 128, 256}) overrides the table, read once.
int level_tile_n(int64_t h) {
    static const std::vector<std::pair<int64_t, int>> table = [] {
        // measured at n = 8192 (one GB300, untraced step): all 256 wide 1.436 ms; this
        // table 1.416 ms; 128 wide from h = 2048 up, or 64 wide at h = 1024, were slower
        std::vector<std::pair<int64_t, int>> t = {{256, 64}, {512, 128}, {1024, 128}};
        if (const char *e = std::getenv("TRI_LEVEL_TILE_N")) {
            t.clear();
            long long hh = 0;
            int bn = 0, used = 0;
            while (std::sscanf(e, "%lld:%d%n", &hh, &bn, &used) == 2) {
                if (bn == 64 || bn == 128 || bn == 256) t.push_back({(int64_t)hh, bn});
                e += used;
                if (*e != ',') break;
                ++e;
            }
        }
        return t;
    }();
    for (const auto &p : table)
        if (p.first == h) return p.second;
    return tc::BN;
}

struct Plan {
    tc::Tile *d_tiles = nullptr;
    int *d_off = nullptr;
    std::vector<Launch> w, x21;   // per tc level (the levels after the merged ones)
    Launch res{}, upd{};
    std::vector<Launch> res_parts, upd_parts;   // both products in column groups, rightmost first
    std::vector<int64_t> upd_lo, upd_hi;
    Launch lvl{};                 // merged low levels (MODE_LVL), if merged_levels > 0
    int merged_levels = 0;        // h = 256 .. 256 * 2^(merged_levels - 1)
    int64_t wld = 0, wcols = 0;   // W layout of the merged levels: wld x wcols, ld = wld
};

// Schedule of the tensor-core products: "levels" (default) launches one persistent kernel
// per product (W and X21 per level, R, the update); "graph" runs them all in one launch
// that follows the tile dependencies (tc_graph.cu).  Chosen once per process from the
// environment variable TRI_MIXED_SCHEDULE; batches always use "levels".
bool use_graph_schedule() {
    static const bool g = [] {
        const char *e = std::getenv("TRI_MIXED_SCHEDULE");
        return e && std::strcmp(e, "graph") == 0;
    }();
    return g;
}

// Split levels whose B blocks are split beside the diagonal-block kernel (the rest follow
// on the side stream while those levels run).  TRI_SPLIT_HEAD_LEVELS (>= 1) overrides
// the default of 2 (h = 256 and 512), read once; a large value splits all of T first.
int split_head_levels() {
    static const int v = [] {
        const char *e = std::getenv("TRI_SPLIT_HEAD_LEVELS");
        const int x = e ? std::atoi(e) : 2;
        return x >= 1 ? x : 2;
    }();
    return v;
}

// "merged" (TRI_MIXED_SCHEDULE=merged): the low levels (h <= kMergedMax) share one
// dependency-ordered launch (MODE_LVL); by default every level has launches of its own.
// Measured at n = 8192: 1.420 ms per step merged against 1.404 ms per level (with
// programmatic dependent launch the per-level boundaries cost little, and the merged
// tiles wait on their pairs).
bool use_merged_levels() {
    static const bool m = [] {
        const char *e = std::getenv("TRI_MIXED_SCHEDULE");
        return e && std::strcmp(e, "merged") == 0;
    }();
    return m;
}

std::mutex g_plan_mu;
std::map<std::tuple<int, int64_t, int64_t, int, int, int>, Plan> g_plans;

// Tile lists of every product for `batch` matrices of order n (each product's tiles of
// all matrices in one longest-first schedule).  recipe TRI_RECIPE_DIRECT: the level
// products take six terms (longest-first costs follow) and there is no Newton-Schulz step.
tri_status build_plan(int dev, int sm_count, int pairs, int pm, int64_t n, int64_t batch, int recipe, Plan **out,
                      int ugroups = 1) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    const bool direct = recipe == TRI_RECIPE_DIRECT;
    const int lterms = direct ? 6 : 3;
    if (direct) pm = 0;
    if (direct || ugroups < 2) ugroups = 1;
    auto key = std::make_tuple(dev, n, batch, recipe, pm, ugroups);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) {
        *out = &it->second;
        return TRI_OK;
    }
    Plan p;
    std::vector<tc::Tile> v;
    std::vector<int> offs;
    auto add = [&](std::vector<Launch> *vec, Launch *one, size_t from, double flops, int terms, int bn = tc::BN,
                   bool pair = false) {
        // replicate the single-matrix tiles over the batch
        const size_t one_count = v.size() - from;
        for (int64_t b = 1; b < batch; ++b)
            for (size_t i = 0; i < one_count; ++i) {
                tc::Tile t = v[from + i];
                t.b = (int)b;
                v.push_back(t);
            }
        std::vector<tc::Tile> part(v.begin() + from, v.end());
        std::vector<int> o;
        const int lists = part.empty() ? 0 : tc::schedule_lpt(part, terms, pair ? pairs : sm_count, o);
        std::copy(part.begin(), part.end(), v.begin() + from);
        Launch l{(int)from, pair ? 2 * lists : lists, (int)offs.size(), flops * (double)batch, bn, pair};
        for (int x : o) offs.push_back(x);
        if (vec) vec->push_back(l);
        else *one = l;
    };
    // Merged low levels (three-term recipe): W and X21 tiles of h = 256 .. kMergedMax in one
    // launch.  Each tile waits on the counters of the tiles that write its operands:
    //   W(h, q)    reads X_A, the inverse of [a0, a0 + h): complete once the X21 tiles of
    //              pair 2q at level h / 2 are (they waited on everything below them);
    //   X21(h, q)  reads W(h, q) and X_C, the inverse of [c0, c0 + hc): complete once the
    //              X21 tiles of the largest lower level's pair starting at c0 are.
    // Each level's W has its own columns of one wld x wcols matrix (ld = wld) in the W planes.
    const bool merged = use_merged_levels() && !direct && n > kDiag;
    int64_t hnext = kDiag;   // first level with launches of its own
    if (merged) {
        std::vector<int64_t> hs, coff, pbase;
        int64_t cols = 0, pb = 0;
        for (int64_t h = kDiag; h <= kMergedMax && h < n; h *= 2) {
            hs.push_back(h);
            coff.push_back(cols);
            pbase.push_back(pb);
            cols += level_pairs(n, h) * h;
            pb += level_pairs(n, h);
        }
        hnext = hs.back() * 2;
        p.merged_levels = (int)hs.size();
        merged_w_dims(n, &p.wld, &p.wcols);
        const int ncnt = (int)(2 * pb);
        auto widx = [&](size_t l, int64_t q) { return (int)(2 * (pbase[l] + q)); };
        auto xidx = [&](size_t l, int64_t q) { return (int)(2 * (pbase[l] + q) + 1); };
        constexpr int64_t bnl = 128;
        // pass 0 counts the tiles behind every counter, pass 1 emits the tiles with waits
        std::vector<int> count(ncnt, 0);
        std::vector<tc::Tile> lt;
        std::vector<int> grp;
        double fl = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
            for (size_t l = 0; l < hs.size(); ++l) {
                const int64_t h = hs[l], P = level_pairs(n, h);
                for (int64_t q = 0; q < P; ++q) {
                    const int64_t a0 = q * 2 * h, c0 = a0 + h, hc = std::min(h, n - c0);
                    int xa = -1, xc = -1;   // counters of X_A and X_C (-1: complete before the launch)
                    if (l > 0) xa = xidx(l - 1, 2 * q);
                    for (size_t m = l; m-- > 0;)
                        if (c0 + hs[m] < n) {
                            xc = xidx(m, c0 / (2 * hs[m]));
                            break;
                        }
                    if (pass == 1) fl += 3.0 * ((double)hc * h * (h + 1) + (double)h * hc * (hc + 1));
                    for (int64_t tn = 0; tn < h / bnl; ++tn)
                        for (int64_t tm = 0; tm < cdiv(hc, tc::BM); ++tm) {
                            if (pass == 0) {
                                ++count[widx(l, q)];
                                continue;
                            }
                            tc::Tile t{(int)(c0 + tm * tc::BM), (int)a0, (int)a0, (int)(a0 + tn * bnl),
                                       (int)(tn * bnl / tc::BK), (int)(h / tc::BK), (int)(tm * tc::BM),
                                       (int)(coff[l] + q * h + tn * bnl)};
                            t.kind = 0;
                            t.pub = widx(l, q);
                            if (xa >= 0) {
                                t.wait0 = xa;
                                t.need0 = tc::EPI_WARPS * count[xa];
                            }
                            lt.push_back(t);
                            grp.push_back((int)(2 * l));
                        }
                    for (int64_t tm = 0; tm < cdiv(hc, tc::BM); ++tm) {
                        const int64_t kend = std::min((tm + 1) * tc::BM, hc);
                        for (int64_t tn = 0; tn < h / bnl; ++tn) {
                            if (pass == 0) {
                                ++count[xidx(l, q)];
                                continue;
                            }
                            tc::Tile t{(int)(c0 + tm * tc::BM), (int)c0, 0, (int)(coff[l] + q * h + tn * bnl), 0,
                                       (int)cdiv(kend, tc::BK), (int)(c0 + tm * tc::BM), (int)(a0 + tn * bnl)};
                            t.kind = 1;
                            t.pub = xidx(l, q);
                            t.wait0 = widx(l, q);
                            t.need0 = tc::EPI_WARPS * count[widx(l, q)];
                            if (xc >= 0) {
                                t.wait1 = xc;
                                t.need1 = tc::EPI_WARPS * count[xc];
                            }
                            lt.push_back(t);
                            grp.push_back((int)(2 * l + 1));
                        }
                    }
                }
            }
        }
        // replicate over the batch: matrix b's tiles use its own counters
        const size_t one = lt.size();
        for (int64_t b = 1; b < batch; ++b)
            for (size_t i = 0; i < one; ++i) {
                tc::Tile t = lt[i];
                t.b = (int)b;
                const int o = (int)b * ncnt;
                t.pub += o;
                if (t.wait0 >= 0) t.wait0 += o;
                if (t.wait1 >= 0) t.wait1 += o;
                lt.push_back(t);
                grp.push_back(grp[i]);
            }
        std::vector<int> o;
        // one CTA per SM at most: a tile waits on tiles of other CTAs, all resident
        const int ctas = lt.empty() ? 0 : tc::schedule_lpt_groups(lt, grp, 3, sm_count, o);
        p.lvl = Launch{(int)v.size(), ctas, (int)offs.size(), fl * (double)batch, (int)bnl, false};
        v.insert(v.end(), lt.begin(), lt.end());
        for (int x : o) offs.push_back(x);
    }
    for (int64_t h = hnext; h < n; h *= 2) {
        const int64_t P = level_pairs(n, h);
        const int bn = level_tile_n(h);   // divides h (h is 256 * 2^s)
        // full-width three-term level products may run on CTA pairs (256-row tiles)
        const bool lp = (pm & kPairLevels) && bn == tc::BN;
        const int64_t bm = lp ? tc::PAIR_BM : tc::BM;
        // W = B X_A  (W is h x P*h, pair q in columns [q*h, q*h + h))
        size_t from = v.size();
        double fl = 0.0;
        for (int64_t q = 0; q < P; ++q) {
            const int64_t a0 = q * 2 * h, c0 = a0 + h, hc = std::min(h, n - c0);
            fl += lterms * (double)hc * h * (h + 1);
            for (int64_t tn = 0; tn < h / bn; ++tn)
                for (int64_t tm = 0; tm < cdiv(hc, bm); ++tm)
                    v.push_back(tc::Tile{(int)(c0 + tm * bm), (int)a0, (int)a0, (int)(a0 + tn * bn),
                                         (int)(tn * bn / tc::BK), (int)(h / tc::BK),
                                         (int)(tm * bm), (int)(q * h + tn * bn)});
        }
        add(&p.w, nullptr, from, fl, lterms, bn, lp);
        // X21 = -X_C W
        from = v.size();
        fl = 0.0;
        for (int64_t q = 0; q < P; ++q) {
            const int64_t a0 = q * 2 * h, c0 = a0 + h, hc = std::min(h, n - c0);
            fl += lterms * (double)h * hc * (hc + 1);
            for (int64_t tm = 0; tm < cdiv(hc, bm); ++tm) {
                const int64_t kend = std::min((tm + 1) * bm, hc);
                for (int64_t tn = 0; tn < h / bn; ++tn)
                    v.push_back(tc::Tile{(int)(c0 + tm * bm), (int)c0, 0, (int)(q * h + tn * bn), 0,
                                         (int)cdiv(kend, tc::BK), (int)(c0 + tm * bm),
                                         (int)(a0 + tn * bn)});
            }
        }
        add(&p.x21, nullptr, from, fl, lterms, bn, lp);
    }
    // Newton-Schulz: lower x lower products over the whole matrix.
    const double lower_prod = (double)n * (n + 1) * (n + 2) / 3.0;   // 2 * sum_{i>=j} (i-j+1)
    for (int pass = 0; pass < (direct ? 0 : 2); ++pass) {
        const size_t from = v.size();
        const bool pp = (pm & (pass == 0 ? kPairRes : kPairUpd)) != 0;
        const int64_t bm = pp ? tc::PAIR_BM : tc::BM;
        for (int64_t tm = 0; tm < cdiv(n, bm); ++tm) {
            const int64_t kend = std::min((tm + 1) * bm, n);
            for (int64_t tn = 0; tn * tc::BN < kend; ++tn)
                v.push_back(tc::Tile{(int)(tm * bm), 0, 0, (int)(tn * tc::BN), (int)(tn * tc::BN / tc::BK),
                                     (int)cdiv(kend, tc::BK), (int)(tm * bm), (int)(tn * tc::BN)});
        }
        add(nullptr, pass == 0 ? &p.res : &p.upd, from, (pass == 0 ? 6.0 : 1.0) * lower_prod,
            pass == 0 ? 6 : 1, tc::BN, pp);
    }
    if (!direct && ugroups > 1) {
        // Both Newton-Schulz products again, in ugroups column groups (rightmost first):
        // tile columns [tc0, tc1) of 256.  Columns j of X R need only columns j of R, and R
        // reads only planes that the update does not write, so group by group the residual
        // and then the update finish those columns of the result.  Flops 2 (i - j + 1) per
        // term for each lower entry (i, j) of the group.
        const int64_t tcn = cdiv(n, tc::BN);
        // group boundaries in tile columns: for four groups at 1/8, 3/8 and 5/8 of the
        // columns (the leftmost group, whose copy back is not overlapped, holds the longest
        // columns; measured at n = 8192: 2.35 ms end to end against 2.51 for equal widths),
        // else equal widths; TRI_HOST_BOUNDS="f1,f2,..." (ugroups - 1 increasing fractions of
        // n) overrides
        std::vector<int64_t> bnd(ugroups + 1);
        for (int g = 0; g <= ugroups; ++g) bnd[g] = tcn * g / ugroups;
        if (ugroups == 4) {
            bnd[1] = (tcn + 4) / 8;
            bnd[2] = std::max(bnd[1], (3 * tcn + 4) / 8);
            bnd[3] = std::max(bnd[2], (5 * tcn + 4) / 8);
        }
        if (const char *e = std::getenv("TRI_HOST_BOUNDS")) {
            std::vector<double> f;
            for (const char *q = e; *q;) {
                char *end = nullptr;
                const double x = std::strtod(q, &end);
                if (end == q) break;
                f.push_back(x);
                q = *end == ',' ? end + 1 : end;
            }
            if ((int)f.size() == ugroups - 1)
                for (int g = 1; g < ugroups; ++g)
                    bnd[g] = std::max(bnd[g - 1], std::min(tcn, (int64_t)(f[g - 1] * (double)tcn + 0.5)));
        }
        for (int g = ugroups - 1; g >= 0; --g) {
            const int64_t tc0 = bnd[g], tc1 = bnd[g + 1];
            if (tc1 <= tc0) continue;
            double fl = 0.0;
            for (int64_t j = tc0 * tc::BN; j < std::min(tc1 * tc::BN, n); ++j) fl += (double)(n - j) * (n - j + 1);
            for (int pass = 0; pass < 2; ++pass) {
                const size_t from = v.size();
                for (int64_t tm = 0; tm < cdiv(n, tc::BM); ++tm) {
                    const int64_t kend = std::min((tm + 1) * tc::BM, n);
                    for (int64_t tn = tc0; tn < tc1 && tn * tc::BN < kend; ++tn)
                        v.push_back(tc::Tile{(int)(tm * tc::BM), 0, 0, (int)(tn * tc::BN), (int)(tn * tc::BN / tc::BK),
                                             (int)cdiv(kend, tc::BK), (int)(tm * tc::BM), (int)(tn * tc::BN)});
                }
                add(pass == 0 ? &p.res_parts : &p.upd_parts, nullptr, from, (pass == 0 ? 6.0 : 1.0) * fl,
                    pass == 0 ? 6 : 1);
            }
            p.upd_lo.push_back(tc0 * tc::BN);
            p.upd_hi.push_back(std::min(tc1 * tc::BN, n));
        }
    }
    if (!v.empty()) {
        const size_t tb = v.size() * sizeof(tc::Tile), ob = offs.size() * sizeof(int);
        uint8_t *d = nullptr;
        if (cudaMalloc(&d, tb + ob) != cudaSuccess) {
            cudaGetLastError();
            return TRI_ERR_NOMEM;
        }
        if (cudaMemcpy(d, v.data(), tb, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(d + tb, offs.data(), ob, cudaMemcpyHostToDevice) != cudaSuccess)
            return TRI_ERR_CUDA;
        p.d_tiles = (tc::Tile *)d;
        p.d_off = (int *)(d + tb);
    }
    auto res = g_plans.emplace(key, p);
    *out = &res.first->second;
    return TRI_OK;
}

}  // namespace

size_t mixed_ws_bytes(int64_t n) {
    if (n <= kDiag) {
        size_t best = 0;
        for (int64_t h = kLeaf; h < n; h *= 2) best = std::max(best, (size_t)(level_pairs(n, h) * h * h) * 4);
        return best;
    }
    return layout(n).total;
}

// Workspace of the strided-batched mixed path: the planes of one chunk of matrices.
size_t mixed_batched_ws_bytes(int64_t n, int64_t batch) {
    if (n <= kDiag) return 0;
    return layout(n, chunk_matrices(n, batch)).total;
}

tri_status run_plain_levels(const Ctx &c, tri_dtype dt, bool trans, bool unit, int64_t n, void *a,
                            int64_t lda, void *ws, int64_t hmax);

namespace {

// One chunk of `batch` matrices (stride elements apart) whose planes fit the workspace.
// index0 >= 0: matrices of a batch starting at index index0 (zero pivots report the
// matrix index); -1: a single matrix (zero pivots report the row).
tri_status run_mixed_chunk(const Ctx &c, bool trans, bool unit, int64_t n, float *a, int64_t lda, int64_t stride,
                           int64_t batch, int64_t index0, void *ws, const InputFeed *feed = nullptr,
                           OutputDrain *drain = nullptr) {
    const Layout L = layout(n, batch);
    uint8_t *base = (uint8_t *)ws;
    const size_t g = L.plane * (size_t)batch;   // bytes of one plane group
    const int64_t ps = (int64_t)(L.plane / 2);  // elements between the planes of consecutive matrices
    __nv_bfloat16 *T[3], *X[3], *R[1], *W[3];
    for (int i = 0; i < 3; ++i) {
        T[i] = (__nv_bfloat16 *)(base + L.off_t + i * g);
        X[i] = (__nv_bfloat16 *)(base + L.off_x + i * g);
    }
    R[0] = (__nv_bfloat16 *)(base + L.off_r);
    W[0] = (__nv_bfloat16 *)(base + L.off_w);
    W[1] = (__nv_bfloat16 *)(base + L.off_w + g);
    W[2] = (__nv_bfloat16 *)(base + L.off_w + 2 * g);

    const bool direct = c.recipe == TRI_RECIPE_DIRECT;
    const bool graph = batch == 1 && !direct && use_graph_schedule();
    const tc::GraphPlan *gplan = nullptr;
    Plan *plan = nullptr;
    tri_status st = graph ? tc::graph_plan(c.device, c.sm_count, n, &gplan)
                          : build_plan(c.device, c.sm_count, c.pairs ? tc::pair_lists(c) : 0, c.pairs, n, batch,
                                       c.recipe, &plan, drain ? std::min(drain->groups, 8) : 1);
    if (drain) drain->got = 0;
    if (st != TRI_OK) return st;
    // dependency counters of the merged low levels start at zero
    int *cnt = (int *)(base + L.off_c);
    if (plan && plan->merged_levels > 0 &&
        cudaMemsetAsync(cnt, 0, (size_t)merged_counters(n) * (size_t)batch * sizeof(int), c.stream) != cudaSuccess)
        return TRI_ERR_CUDA;

    // 1. T planes of the off-diagonal part (side stream), concurrently with
    // 2.+3. the FP32 diagonal blocks of 256, each inverted in shared memory by one CTA (CRIT
    //       leaves of 32 and the split levels 32, 64, 128), which also writes the T and X
    //       planes of its block.  The two touch disjoint parts of T.
    //    Only the B blocks of the first kHeadLevels split levels are split beside the
    //    diagonal blocks; the rest (most of T) follows on the side stream while those
    //    levels run, and the main stream waits for it before the next level.  (The split
    //    runs at full HBM bandwidth; beside it the latency-bound diagonal-block kernel
    //    took 90 us against 64 us alone.)
    SideStream *ss = nullptr;
    std::unique_lock<std::mutex> side_lock(g_side_mu);
    if (!side_stream(c.device, &ss)) return TRI_ERR_CUDA;
    // input arriving by parts: the head waits for the diagonal blocks and the first levels
    if (feed && feed->count > 0 && cudaStreamWaitEvent(c.stream, feed->ready[0], 0) != cudaSuccess)
        return TRI_ERR_CUDA;
    if (cudaEventRecord(ss->fork, c.stream) != cudaSuccess || cudaStreamWaitEvent(ss->s, ss->fork, 0) != cudaSuccess)
        return TRI_ERR_CUDA;
    // The diagonal-block kernel goes first: each of its CTAs needs a whole SM's shared
    // memory, so queued behind the split kernel's CTAs it would wait for SMs to drain (the
    // split then fills the SMs it leaves free).
    int *gflags = (int *)(base + L.off_g);   // growth flags (the single-launch schedule takes no fallback)
    const float tau = graph ? 0.f : c.tau;
    if (launch_diag_blocks(c, trans, unit, n, a, lda, X[0], X[1], X[2], L.ldp, T[0], T[1], T[2], batch, stride, ps,
                           index0, tau, tau > 0.f ? gflags : nullptr) != cudaSuccess)
        return TRI_ERR_CUDA;
    Ctx cs = c;
    cs.stream = ss->s;
    const int kHeadLevels = split_head_levels();
    int nlevels = 0;   // split levels h = 256 * 2^l < n
    for (int64_t h = kDiag; h < n; h *= 2) ++nlevels;
    const bool rest = nlevels > kHeadLevels;   // B blocks left for the side stream
    if (launch_split_planes(cs, trans, unit, false, n, a, lda, T[0], T[1], T[2], L.ldp, true, batch, stride, ps, 0,
                            rest ? kHeadLevels - 1 : 62) != cudaSuccess)
        return TRI_ERR_CUDA;
    if (cudaEventRecord(ss->join, ss->s) != cudaSuccess || cudaStreamWaitEvent(c.stream, ss->join, 0) != cudaSuccess)
        return TRI_ERR_CUDA;
    // Input by parts (feed): one split launch per later level, each after its part arrives,
    // each with a join event of its own; otherwise one launch for all later levels.
    const bool by_level = rest && feed && feed->count >= 1 + nlevels - kHeadLevels &&
                          nlevels - kHeadLevels <= (int)(sizeof(ss->lev) / sizeof(ss->lev[0]));
    if (rest && by_level) {
        for (int l = kHeadLevels; l < nlevels; ++l)
            if (cudaStreamWaitEvent(ss->s, feed->ready[1 + l - kHeadLevels], 0) != cudaSuccess ||
                launch_split_planes(cs, trans, unit, false, n, a, lda, T[0], T[1], T[2], L.ldp, true, batch, stride,
                                    ps, l, l) != cudaSuccess ||
                cudaEventRecord(ss->lev[l - kHeadLevels], ss->s) != cudaSuccess)
                return TRI_ERR_CUDA;
    } else if (rest) {
        if (feed)   // parts arrive in order: the last one completes the input
            for (int k = 1; k < feed->count; ++k)
                if (cudaStreamWaitEvent(ss->s, feed->ready[k], 0) != cudaSuccess) return TRI_ERR_CUDA;
        if (launch_split_planes(cs, trans, unit, false, n, a, lda, T[0], T[1], T[2], L.ldp, true, batch, stride, ps,
                                kHeadLevels, 62) != cudaSuccess ||
            cudaEventRecord(ss->join2, ss->s) != cudaSuccess)
            return TRI_ERR_CUDA;
    }
    // The main stream's waits for the planes of level l >= kHeadLevels, enqueued before
    // the level's first product; the side stream's lock is held until the last one.
    int joined = rest ? kHeadLevels : nlevels;   // levels whose planes the main stream has
    auto join_level = [&](int l) -> bool {
        bool ok = true;
        while (joined <= l && joined < nlevels) {
            if (by_level) ok = ok && cudaStreamWaitEvent(c.stream, ss->lev[joined - kHeadLevels], 0) == cudaSuccess;
            else if (joined == kHeadLevels) ok = ok && cudaStreamWaitEvent(c.stream, ss->join2, 0) == cudaSuccess;
            ++joined;
        }
        if (joined >= nlevels && side_lock.owns_lock()) side_lock.unlock();
        return ok;
    };
    auto join_rest = [&]() -> bool { return join_level(nlevels); };
    if (!rest) side_lock.unlock();

    if (graph) {
        if (!join_rest()) return TRI_ERR_CUDA;
        // 4. + 5. as one dependency-driven launch (W planes at the B-block positions)
        int *flags = (int *)(base + L.off_f);
        tc::GEpi ep{a, lda, X[0], X[1], X[2], W[0], W[1], R[0], L.ldp, n, flags,
                    flags + 3 * gplan->nrb * gplan->ncb, nullptr};
        return tc::launch_graph(c, trans, unit, n, *gplan, T, ep) == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
    }
    auto pl = [&](const __nv_bfloat16 *p, int64_t rows, int64_t cols, int64_t ld) {
        tc::Plane q{p, rows, cols, ld};
        q.batch = batch;
        q.bstride = ps;
        return q;
    };
    const tc::Plane tp[3] = {pl(T[0], n, n, L.ldp), pl(T[1], n, n, L.ldp), pl(T[2], n, n, L.ldp)};
    const tc::Plane xp[3] = {pl(X[0], n, n, L.ldp), pl(X[1], n, n, L.ldp), pl(X[2], n, n, L.ldp)};
    const tc::Terms three{3, {0, 0, 1}, {0, 1, 0}};
    const tc::Terms six{6, {0, 0, 1, 0, 1, 2}, {0, 1, 0, 2, 1, 0}};
    // 4. tensor-core levels (direct recipe: six promoted terms, W with its lo plane)
    const int mw = direct ? tc::MODE_W6 : tc::MODE_W, mx = direct ? tc::MODE_X216 : tc::MODE_X21;
    const tc::Terms &lt = direct ? six : three;
    const int nw = direct ? 3 : 2;
    // trace names per split half-size h = 256 * 2^lvl
    static const char *const kWName[] = {"tc_gemm:w:256", "tc_gemm:w:512", "tc_gemm:w:1024", "tc_gemm:w:2048",
                                         "tc_gemm:w:4096", "tc_gemm:w:8192", "tc_gemm:w:16384", "tc_gemm:w"};
    static const char *const kXName[] = {"tc_gemm:x21:256", "tc_gemm:x21:512", "tc_gemm:x21:1024",
                                         "tc_gemm:x21:2048", "tc_gemm:x21:4096", "tc_gemm:x21:8192",
                                         "tc_gemm:x21:16384", "tc_gemm:x21"};
    int64_t hfirst = kDiag;
    if (plan->merged_levels > 0) {
        if (!join_rest()) return TRI_ERR_CUDA;
        // 4a. the low levels in one launch: W tiles (targets ew) and X21 tiles (ex)
        static const char *const kLvlName = "tc_gemm:lvl";
        // the merged levels' W planes: wld x wcols each, mplane bytes per matrix
        const int64_t ms = (int64_t)(L.mplane / 2);
        __nv_bfloat16 *M0 = (__nv_bfloat16 *)(base + L.off_m), *M1 = M0 + ms * batch;
        auto plm = [&](const __nv_bfloat16 *p) {
            tc::Plane q{p, plan->wld, plan->wcols, plan->wld};
            q.batch = batch;
            q.bstride = ms;
            return q;
        };
        const tc::Plane la[4] = {tp[0], tp[1], xp[0], xp[1]};
        const tc::Plane lb[4] = {xp[0], xp[1], plm(M0), plm(M1)};
        tc::Epi ew{nullptr, 0, M0, M1, nullptr, plan->wld, plan->wld, plan->wcols};
        ew.os = ms;
        ew.cnt = cnt;
        ew.xs = 0;
        tc::Epi ex{a, lda, X[0], X[1], X[2], L.ldp, n, n};
        ex.xs = stride;
        ex.os = ps;
        const Launch &ll = plan->lvl;
        if (tc::launch_tc(c, tc::MODE_LVL, trans, unit, la, 4, lb, 4, three, plan->d_tiles + ll.first,
                          plan->d_off + ll.off_first, ll.ctas, ew, ll.flops, kLvlName, ll.bn, false, &ex) !=
            cudaSuccess)
            return TRI_ERR_CUDA;
        hfirst = kDiag << plan->merged_levels;
    }
    int lvl = 0;
    for (int64_t h = hfirst; h < n; h *= 2, ++lvl) {
        const int64_t P = level_pairs(n, h);
        int lv = 0;   // split level: log2(h / 256)
        while ((kDiag << lv) < h) ++lv;
        const int name = std::min(lv, 7);   // trace name index
        if (lv >= kHeadLevels && !join_level(lv)) return TRI_ERR_CUDA;
        const tc::Plane wp[3] = {pl(W[0], h, P * h, h), pl(W[1], h, P * h, h), pl(W[2], h, P * h, h)};
        tc::Epi ew{nullptr, 0, W[0], W[1], direct ? W[2] : nullptr, h, h, P * h};
        ew.os = ps;
        const Launch &lw = plan->w[lvl];
        if (tc::launch_tc(c, mw, trans, unit, tp, 3, xp, 3, lt, plan->d_tiles + lw.first, plan->d_off + lw.off_first,
                          lw.ctas, ew, lw.flops, kWName[name], lw.bn, lw.pair) != cudaSuccess)
            return TRI_ERR_CUDA;
        tc::Epi ex{a, lda, X[0], X[1], X[2], L.ldp, n, n};
        ex.xs = stride;
        ex.os = ps;
        const Launch &lx = plan->x21[lvl];
        if (tc::launch_tc(c, mx, trans, unit, xp, 3, wp, nw, lt, plan->d_tiles + lx.first, plan->d_off + lx.off_first,
                          lx.ctas, ex, lx.flops, kXName[name], lx.bn, lx.pair) != cudaSuccess)
            return TRI_ERR_CUDA;
    }
    if (!join_rest()) return TRI_ERR_CUDA;
    if (direct) return TRI_OK;
    // 5. Newton-Schulz: R = I - T X, then X += X R
    tc::Epi er{nullptr, 0, R[0], nullptr, nullptr, L.ldp, n, n};
    er.os = ps;
    if (tau > 0.f) {
        er.skip = gflags;
        er.skip_n = (int)((n + kDiag - 1) / kDiag);
    }
    const tc::Plane rp[1] = {pl(R[0], n, n, L.ldp)};
    const tc::Terms one{1, {0}, {0}};
    tc::Epi eu{a, lda, nullptr, nullptr, nullptr, 0, n, n};
    eu.xs = stride;
    if (drain && !plan->upd_parts.empty()) {
        // column groups from the right: residual then update of the group; its columns of
        // the result are final after the update
        const int np = (int)plan->upd_parts.size();
        for (int g = 0; g < np; ++g) {
            const Launch &lr = plan->res_parts[g], &lu = plan->upd_parts[g];
            if (tc::launch_tc(c, tc::MODE_RES, trans, unit, tp, 3, xp, 3, six, plan->d_tiles + lr.first,
                              plan->d_off + lr.off_first, lr.ctas, er, lr.flops, "tc_gemm:res") != cudaSuccess ||
                tc::launch_tc(c, tc::MODE_UPD, trans, unit, xp, 1, rp, 1, one, plan->d_tiles + lu.first,
                              plan->d_off + lu.off_first, lu.ctas, eu, lu.flops, "tc_gemm:upd") != cudaSuccess ||
                cudaEventRecord(drain->done[g], c.stream) != cudaSuccess)
                return TRI_ERR_CUDA;
            drain->col_lo[g] = plan->upd_lo[g];
            drain->col_hi[g] = plan->upd_hi[g];
        }
        drain->got = np;
        return TRI_OK;
    }
    if (tc::launch_tc(c, tc::MODE_RES, trans, unit, tp, 3, xp, 3, six, plan->d_tiles + plan->res.first,
                      plan->d_off + plan->res.off_first, plan->res.ctas, er, plan->res.flops, "tc_gemm:res", tc::BN,
                      plan->res.pair) != cudaSuccess)
        return TRI_ERR_CUDA;
    if (tc::launch_tc(c, tc::MODE_UPD, trans, unit, xp, 1, rp, 1, one, plan->d_tiles + plan->upd.first,
                      plan->d_off + plan->upd.off_first, plan->upd.ctas, eu, plan->upd.flops, "tc_gemm:upd", tc::BN,
                      plan->upd.pair) != cudaSuccess)
        return TRI_ERR_CUDA;
    return TRI_OK;
}

}  // namespace

tri_status run_mixed(const Ctx &c, bool trans, bool unit, int64_t n, float *a, int64_t lda, void *ws) {
    if (n <= kDiag) return run_plain_levels(c, TRI_F32, trans, unit, n, a, lda, ws, n);
    return run_mixed_chunk(c, trans, unit, n, a, lda, 0, 1, -1, ws);
}

int mixed_head_levels() { return split_head_levels(); }

// run_mixed with the input arriving by parts (see InputFeed): every part's event is waited
// for before anything reads that part.
tri_status run_mixed_fed(const Ctx &c, bool trans, bool unit, int64_t n, float *a, int64_t lda, void *ws,
                         const InputFeed *feed, OutputDrain *drain) {
    if (drain) drain->got = 0;
    if (n <= kDiag) {
        for (int k = 0; feed && k < feed->count; ++k)
            if (cudaStreamWaitEvent(c.stream, feed->ready[k], 0) != cudaSuccess) return TRI_ERR_CUDA;
        return run_plain_levels(c, TRI_F32, trans, unit, n, a, lda, ws, n);
    }
    return run_mixed_chunk(c, trans, unit, n, a, lda, 0, 1, -1, ws, feed, drain);
}

// `batch` matrices `stride` elements apart (n > 256), in chunks whose planes fit the
// workspace of mixed_batched_ws_bytes(n, batch).
tri_status run_mixed_batched(const Ctx &c, bool trans, bool unit, int64_t n, float *a, int64_t lda, int64_t stride,
                             int64_t batch, void *ws) {
    const int64_t cb = chunk_matrices(n, batch);
    for (int64_t b0 = 0; b0 < batch; b0 += cb) {
        const tri_status st =
            run_mixed_chunk(c, trans, unit, n, a + b0 * stride, lda, stride, std::min(cb, batch - b0), b0, ws);
        if (st != TRI_OK) return st;
    }
    return TRI_OK;
}

}  // namespace triinv
