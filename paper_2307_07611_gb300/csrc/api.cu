// api.cu -- the C ABI (include/triinv.h): argument checks, per-device status words,
// scratch handling, kernel tracing and the level scheduler of the recursive split.
//
// Recursive triangular split (Section 4.1, Algorithm "COMBRIT" with two blocks; block
// inverse from the proof of the main Theorem, Section 3):
//     T = [A 0; B C]  ->  T^-1 = [A^-1 0; -C^-1 B A^-1  C^-1].
// The recursion tree is walked bottom-up by levels.  The matrix is logically padded with
// identity up to leaf * 2^L (the paper pads with canonical-basis columns, Appendix), so
// every level has the same half-size h = leaf * 2^(s-1) and pairs start at multiples of
// 2h; padded rows and columns are never touched (the kernels clip them).
//   level 0: every leaf block is inverted by the CRIT column recurrence (leaf.cu);
//   level s: for every pair, W = B X_A then B <- -X_C W (trmm_simt.cu / tc_gemm.cu).
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"
#include "tc_gemm.cuh"

namespace triinv {

// Device status words: the smallest bad pivot index seen and the timeout flag.  One copy
// per device (module globals are per context); host code reaches them through
// cudaGetSymbolAddress.
__device__ long long g_info_word = LLONG_MAX;
__device__ int g_timeout_word = 0;

namespace {

struct DeviceState {
    bool ready = false;
    long long *info = nullptr;
    int *timeout = nullptr;
    int sm_count = 0;
};

std::mutex g_mu;
DeviceState g_dev[64];

// Growth limit of the FP64 fallback on the single-matrix paths (plain leaves, the mixed
// path's diagonal blocks): max|X| max|T| of a diagonal block's FP32 inverse above it
// triggers an FP64 inverse of that block.  Process-wide; <= 0 disables.
std::atomic<float> g_growth_tau{1.0e4f};

// Recipe of the mixed triangular path (process-wide).
std::atomic<int> g_recipe{TRI_RECIPE_NEWTON_SCHULZ};
std::atomic<int> g_pairs{0};

tri_status device_ctx(cudaStream_t stream, Ctx *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TRI_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceState &d = g_dev[dev];
    if (!d.ready) {
        void *pi = nullptr, *pt = nullptr;
        if (cudaGetSymbolAddress(&pi, g_info_word) != cudaSuccess) return TRI_ERR_CUDA;
        if (cudaGetSymbolAddress(&pt, g_timeout_word) != cudaSuccess) return TRI_ERR_CUDA;
        if (cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return TRI_ERR_CUDA;
        d.info = (long long *)pi;
        d.timeout = (int *)pt;
        d.ready = true;
    }
    out->stream = stream;
    out->info = d.info;
    out->timeout = d.timeout;
    out->sm_count = d.sm_count;
    out->device = dev;
    out->tau = g_growth_tau.load(std::memory_order_relaxed);
    out->recipe = g_recipe.load(std::memory_order_relaxed);
    out->pairs = g_pairs.load(std::memory_order_relaxed);
    return TRI_OK;
}

// ---- library scratch pool -----------------------------------------------------------
// Scratch of the allocating entry points comes from a private stream-ordered pool per
// device, created on the first allocation.  Its release threshold is unlimited, so freed
// blocks stay cached for the next call; the device's default pool, which other code in
// the process (PyTorch, the application) may use, is left as it is.
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64];

cudaError_t lib_pool(cudaMemPool_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

// Per-call status word: the caller's d_info is set to "none" before the call's kernels
// and turned from the internal "none" (LLONG_MAX) into -1 after them.
__global__ void info_begin_kernel(long long *w) { *w = LLONG_MAX; }
__global__ void info_end_kernel(long long *w) {
    if (*w == LLONG_MAX) *w = -1;
}

}  // namespace

tri_status device_ctx_public(cudaStream_t stream, Ctx *out) { return device_ctx(stream, out); }

cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    cudaMemPool_t pool;
    cudaError_t e = lib_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

tri_status info_begin(Ctx &c, int64_t *d_info) {
    if (!d_info) return TRI_OK;
    c.info = (long long *)d_info;
    info_begin_kernel<<<1, 1, 0, c.stream>>>(c.info);
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
}

tri_status info_end(const Ctx &c, int64_t *d_info, tri_status st) {
    if (!d_info || st != TRI_OK) return st;
    info_end_kernel<<<1, 1, 0, c.stream>>>(c.info);
    return cudaGetLastError() == cudaSuccess ? TRI_OK : TRI_ERR_CUDA;
}

namespace {

// ---- tracing -------------------------------------------------------------------------
struct TraceRec {
    std::string kernel;
    cudaEvent_t beg, end;
    double flops, bytes;
};
std::mutex g_trace_mu;
bool g_trace_on = false;
std::vector<TraceRec> g_trace;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event() {
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void clear_trace_locked() {
    for (auto &r : g_trace) {
        g_event_pool.push_back(r.beg);
        g_event_pool.push_back(r.end);
    }
    g_trace.clear();
}

}  // namespace

bool trace_on() {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    return g_trace_on;
}

TraceScope::TraceScope(cudaStream_t stream, const char *kernel, double flops, double bytes)
    : slot(-1), stream_(stream) {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    if (!g_trace_on) return;
    TraceRec r{kernel, take_event(), take_event(), flops, bytes};
    if (!r.beg || !r.end) return;
    cudaEventRecord(r.beg, stream);
    g_trace.push_back(r);
    slot = (int)g_trace.size() - 1;
}

TraceScope::~TraceScope() {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_trace_mu);
    if (slot < (int)g_trace.size()) cudaEventRecord(g_trace[slot].end, stream_);
}

// ---- plans ---------------------------------------------------------------------------
namespace {

// Leaf order of the plain path.  FP64 leaves are 16: GB300 has little FP64 throughput per
// SM, so the serial leaf recurrence is kept short and the work moves into the level
// products, which spread over every SM.
int leaf_plain(tri_dtype dt) { return dt == TRI_F64 ? 16 : 64; }

size_t elem_size(tri_dtype dt) { return dt == TRI_F64 ? 8 : 4; }

// Largest per-level scratch of the plain path: one h x h W block per active pair.
size_t plain_ws_bytes(int64_t n, tri_dtype dt) {
    size_t best = 0;
    for (int64_t h = leaf_plain(dt); h < n; h *= 2) {
        const int64_t p = level_pairs(n, h);
        best = std::max(best, (size_t)p * (size_t)h * (size_t)h * elem_size(dt));
    }
    return best;
}

bool valid_enums(tri_uplo u, tri_diag d, tri_dtype t) {
    return (u == TRI_LOWER || u == TRI_UPPER) && (d == TRI_NONUNIT || d == TRI_UNIT) &&
           (t == TRI_F64 || t == TRI_F32 || t == TRI_F32_MIXED);
}

tri_status from_cuda(cudaError_t e) { return e == cudaSuccess ? TRI_OK : TRI_ERR_CUDA; }

}  // namespace

// Leaf inverses and the split levels with half-size h < hmax (hmax = n: the whole
// recursion; hmax = 256: only the diagonal 256-blocks, as the mixed path needs).
tri_status run_plain_levels(const Ctx &c, tri_dtype dt, bool trans, bool unit, int64_t n, void *a,
                            int64_t lda, void *ws, int64_t hmax) {
    const int leaf = leaf_plain(dt);
    cudaError_t e = launch_leaf(c, dt, trans, unit, n, a, lda, leaf);
    if (e != cudaSuccess) return TRI_ERR_CUDA;
    for (int64_t h = leaf; h < n && h < hmax; h *= 2) {
        e = launch_trmm_level(c, dt, trans, unit, 0, n, a, lda, h, ws);
        if (e != cudaSuccess) return TRI_ERR_CUDA;
        e = launch_trmm_level(c, dt, trans, unit, 1, n, a, lda, h, ws);
        if (e != cudaSuccess) return TRI_ERR_CUDA;
    }
    return TRI_OK;
}

size_t mixed_ws_bytes(int64_t n);
size_t combrit_ws_bytes(int64_t n, tri_dtype dt, int beta);
tri_status run_combrit(const Ctx &c, tri_dtype dt, bool trans, bool unit, int64_t n, void *a, int64_t lda, int beta,
                       void *ws);
size_t gen_inv_ws_bytes(int64_t n, tri_dtype dt);
tri_status run_gen_inv(const Ctx &c, tri_dtype dt, int64_t n, void *a, int64_t lda, void *ws,
                       int64_t info_base = 0);
size_t skul_ws_bytes(int64_t n, tri_dtype dt);
size_t brsi_ws_bytes(int64_t n, int gamma, tri_dtype dt);
tri_status run_brsi(const Ctx &c, tri_dtype dt, int64_t n, void *a, int64_t lda, int gamma, const int64_t *perm,
                    void *ws);
tri_status run_skul(const Ctx &c, tri_dtype dt, int64_t n, void *a, int64_t lda, void *sk, int64_t ldsk, void *ws);
size_t sqr_ws_bytes(int64_t n, tri_dtype dt);
tri_status run_sqr(const Ctx &c, tri_dtype dt, int64_t n, void *a, int64_t lda, void *r, int64_t ldr, void *s,
                   int64_t lds, void *ws);
size_t sqr_inv_ws_bytes(int64_t n, tri_dtype dt);
tri_status run_sqr_inv(const Ctx &c, tri_dtype dt, int64_t n, void *a, int64_t lda, void *ws);
tri_status run_mixed(const Ctx &c, bool trans, bool unit, int64_t n, float *a, int64_t lda, void *ws);

}  // namespace triinv

using namespace triinv;

extern "C" {

const char *tri_status_string(tri_status s) {
    switch (s) {
        case TRI_OK: return "TRI_OK";
        case TRI_ERR_ARG: return "TRI_ERR_ARG: invalid argument";
        case TRI_ERR_SINGULAR: return "TRI_ERR_SINGULAR: zero or non-finite pivot";
        case TRI_ERR_NOMEM: return "TRI_ERR_NOMEM: scratch allocation failed or workspace too small";
        case TRI_ERR_CUDA: return "TRI_ERR_CUDA: CUDA runtime or launch error";
        case TRI_ERR_TIMEOUT: return "TRI_ERR_TIMEOUT: a bounded device wait ran out";
        case TRI_ERR_UNSUPPORTED: return "TRI_ERR_UNSUPPORTED: not provided by this build";
    }
    return "unknown tri_status";
}

const char *tri_version(void) { return "0.1.0 sm_103a"; }

size_t tri_inv_workspace_size(int64_t n, tri_dtype dtype) {
    if (n <= 0) return 0;
    if (dtype == TRI_F64 || dtype == TRI_F32) return plain_ws_bytes(n, dtype);
    if (dtype == TRI_F32_MIXED) return mixed_ws_bytes(n);
    return 0;
}

tri_status tri_inv_ex(tri_uplo uplo, tri_diag diag, int64_t n, void *a, int64_t lda,
                      tri_dtype dtype, void *workspace, size_t ws_bytes, int64_t *d_info, void *stream) {
    if (!valid_enums(uplo, diag, dtype) || n < 0) return TRI_ERR_ARG;
    if (n == 0) return TRI_OK;
    if (!a || lda < std::max<int64_t>(1, n)) return TRI_ERR_ARG;
    const size_t need = tri_inv_workspace_size(n, dtype);
    if (need > 0 && (ws_bytes < need || !workspace || ((uintptr_t)workspace & 255)))
        return TRI_ERR_NOMEM;
    Ctx c;
    tri_status st = device_ctx((cudaStream_t)stream, &c);
    if (st != TRI_OK) return st;
    if ((st = info_begin(c, d_info)) != TRI_OK) return st;
    if (dtype == TRI_F32_MIXED)
        st = run_mixed(c, uplo == TRI_UPPER, diag == TRI_UNIT, n, (float *)a, lda, workspace);
    else
        st = run_plain_levels(c, dtype, uplo == TRI_UPPER, diag == TRI_UNIT, n, a, lda, workspace, n);
    return info_end(c, d_info, st);
}

tri_status tri_inv(tri_uplo uplo, tri_diag diag, int64_t n, void *a, int64_t lda,
                   tri_dtype dtype, void *stream) {
    if (!valid_enums(uplo, diag, dtype) || n < 0) return TRI_ERR_ARG;
    if (n == 0) return TRI_OK;
    if (!a || lda < std::max<int64_t>(1, n)) return TRI_ERR_ARG;
    const size_t need = tri_inv_workspace_size(n, dtype);
    void *ws = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    if (need > 0 && lib_malloc_async(&ws, need, s) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_NOMEM;
    }
    tri_status st = tri_inv_ex(uplo, diag, n, a, lda, dtype, ws, need, nullptr, stream);
    if (ws) {
        cudaError_t e = cudaFreeAsync(ws, s);
        if (st == TRI_OK && e != cudaSuccess) st = TRI_ERR_CUDA;
    }
    return st;
}

// Host-memory form: the referenced triangle travels in 256-column panels (one 2-D copy
// each), so about half of the n x n matrix crosses the host link in each direction.
// Columns [jlo, jhi) only (jlo a multiple of 256) when given.
static int64_t host_panel_copies(bool upper, int64_t n, uint8_t *dev, int64_t ldd, uint8_t *host, int64_t ldh,
                                 size_t es, cudaMemcpyKind kind, cudaStream_t s, cudaError_t *err, int64_t jlo = 0,
                                 int64_t jhi = -1) {
    constexpr int64_t kPanel = 256;
    int64_t bytes = 0;
    if (jhi < 0 || jhi > n) jhi = n;
    for (int64_t j0 = jlo; j0 < jhi && *err == cudaSuccess; j0 += kPanel) {
        const int64_t cols = std::min(kPanel, jhi - j0);
        const int64_t r0 = upper ? 0 : j0, rows = upper ? j0 + cols : n - j0;
        uint8_t *d = dev + ((size_t)j0 * ldd + r0) * es, *h = host + ((size_t)j0 * ldh + r0) * es;
        *err = kind == cudaMemcpyHostToDevice
                   ? cudaMemcpy2DAsync(d, ldd * es, h, ldh * es, rows * es, cols, kind, s)
                   : cudaMemcpy2DAsync(h, ldh * es, d, ldd * es, rows * es, cols, kind, s);
        bytes += rows * cols * (int64_t)es;
    }
    return bytes;
}

// Mixed path: the referenced triangle travels in the order the inverse first reads it, on a
// copy stream of its own: the diagonal 256-blocks and the B blocks of the first split
// levels, then the B blocks of each further level (the blocks of the recursive split tile
// the triangle).  An event after each part lets the inverse start on the first parts while
// the rest is still in flight (run_mixed_fed).
struct HostFeed {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, back = nullptr;
    cudaEvent_t ready[26] = {};
    cudaEvent_t done[8] = {};
};
std::mutex g_feed_mu;
HostFeed g_feed[64];

static int64_t host_block_copies(bool upper, int64_t n, uint8_t *dev, int64_t ldd, uint8_t *host, int64_t ldh,
                                 size_t es, HostFeed &f, int *parts, cudaError_t *err) {
    constexpr int64_t kDiagB = 256;
    const int head = mixed_head_levels();
    int64_t bytes = 0;
    // lower-view block rows [r0, r0 + rows) x columns [c0, c0 + cols); stored transposed
    // for an upper matrix
    auto copy = [&](int64_t r0, int64_t rows, int64_t c0, int64_t cols) {
        if (*err != cudaSuccess || rows <= 0 || cols <= 0) return;
        if (upper) {
            std::swap(r0, c0);
            std::swap(rows, cols);
        }
        *err = cudaMemcpy2DAsync(dev + ((size_t)c0 * ldd + r0) * es, ldd * es, host + ((size_t)c0 * ldh + r0) * es,
                                 ldh * es, rows * es, cols, cudaMemcpyHostToDevice, f.s);
        bytes += rows * cols * (int64_t)es;
    };
    auto level_blocks = [&](int64_t h) {
        for (int64_t q = 0; q < level_pairs(n, h); ++q) {
            const int64_t a0 = 2 * q * h, c0 = a0 + h;
            copy(c0, std::min(h, n - c0), a0, h);
        }
    };
    int k = 0;
    // the first part, as 256-column panels down to the end of each band of 256 * 2^head
    // rows: the diagonal squares and the B blocks of the first `head` levels, in one copy per
    // panel
    const int64_t band = kDiagB << head;
    for (int64_t j0 = 0; j0 < n; j0 += kDiagB)
        copy(j0, std::min(n, (j0 / band + 1) * band) - j0, j0, std::min(kDiagB, n - j0));
    int64_t h = kDiagB << head;
    if (*err == cudaSuccess) *err = cudaEventRecord(f.ready[k++], f.s);
    for (; h < n && k < 26; h *= 2) {
        level_blocks(h);
        if (*err == cudaSuccess) *err = cudaEventRecord(f.ready[k++], f.s);
    }
    *parts = k;
    return bytes;
}

tri_status tri_inv_host(tri_uplo uplo, tri_diag diag, int64_t n, void *a, int64_t lda, tri_dtype dtype,
                        void *stream, int64_t *bytes_moved) {
    if (bytes_moved) *bytes_moved = 0;
    if (!valid_enums(uplo, diag, dtype) || n < 0) return TRI_ERR_ARG;
    if (n == 0) return TRI_OK;
    if (!a || lda < std::max<int64_t>(1, n)) return TRI_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Ctx c;
    tri_status st = device_ctx(s, &c);
    if (st != TRI_OK) return st;
    const size_t es = dtype == TRI_F64 ? 8 : 4;
    const int64_t ldd = (n + 31) / 32 * 32;
    const size_t mat = ((size_t)ldd * n * es + 255) / 256 * 256;
    const size_t need = tri_inv_workspace_size(n, dtype);
    uint8_t *buf = nullptr;
    if (lib_malloc_async((void **)&buf, mat + need, s) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_NOMEM;
    }
    cudaError_t e = cudaSuccess;
    const bool upper = uplo == TRI_UPPER;
    int64_t moved = 0;
    if (dtype == TRI_F32_MIXED && c.device >= 0 && c.device < 64) {
        // copies by parts on the copy stream, the inverse waiting for each part where needed
        std::lock_guard<std::mutex> lk(g_feed_mu);
        HostFeed &f = g_feed[c.device];
        if (!f.s) {
            bool ok = cudaStreamCreateWithFlags(&f.s, cudaStreamNonBlocking) == cudaSuccess &&
                      cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming) == cudaSuccess &&
                      cudaEventCreateWithFlags(&f.back, cudaEventDisableTiming) == cudaSuccess;
            for (cudaEvent_t &ev : f.ready)
                ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
            for (cudaEvent_t &ev : f.done)
                ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
            if (!ok) e = cudaErrorUnknown;
        }
        int parts = 0;
        if (e == cudaSuccess &&
            (e = cudaEventRecord(f.fork, s)) == cudaSuccess &&   // after the buffer's allocation
            (e = cudaStreamWaitEvent(f.s, f.fork, 0)) == cudaSuccess)
            moved = host_block_copies(upper, n, buf, ldd, (uint8_t *)a, lda, es, f, &parts, &e);
        if (e == cudaSuccess) {
            const InputFeed feed{f.ready, parts};
            // the result goes back by column groups, each as soon as the update has
            // finished its columns, on the copy stream beside the later groups' updates
            // (lower storage only: for an upper matrix the columns of the lower view are
            // stored rows, which do not map onto panels of the stored triangle)
            static const int kGroups = [] {   // TRI_HOST_GROUPS (1..8) overrides, read once
                const char *ev = std::getenv("TRI_HOST_GROUPS");
                const int v = ev ? std::atoi(ev) : 4;
                return v >= 1 && v <= 8 ? v : 4;
            }();
            OutputDrain drain{upper ? 1 : kGroups, f.done, 0, {}, {}};
            if ((st = info_begin(c, nullptr)) == TRI_OK)
                st = info_end(c, nullptr,
                              run_mixed_fed(c, upper, diag == TRI_UNIT, n, (float *)buf, ldd, need ? buf + mat : nullptr,
                                            &feed, &drain));
            // every part is in before the result goes back and the buffer is freed
            if (parts > 0 && cudaStreamWaitEvent(s, f.ready[parts - 1], 0) != cudaSuccess) e = cudaErrorUnknown;
            if (st == TRI_OK && e == cudaSuccess) {
                if (drain.got > 0) {
                    for (int g = 0; g < drain.got && e == cudaSuccess; ++g) {
                        if ((e = cudaStreamWaitEvent(f.s, f.done[g], 0)) != cudaSuccess) break;
                        moved += host_panel_copies(upper, n, buf, ldd, (uint8_t *)a, lda, es, cudaMemcpyDeviceToHost,
                                                   f.s, &e, drain.col_lo[g], drain.col_hi[g]);
                    }
                    // the stream sees the copies out (also those queued before a failed one)
                    // before it frees the buffer and returns
                    const cudaError_t eb = cudaEventRecord(f.back, f.s);
                    const cudaError_t ew = eb == cudaSuccess ? cudaStreamWaitEvent(s, f.back, 0) : eb;
                    if (e == cudaSuccess) e = ew;
                } else {
                    moved += host_panel_copies(upper, n, buf, ldd, (uint8_t *)a, lda, es, cudaMemcpyDeviceToHost, s, &e);
                }
            }
        }
    } else {
        moved = host_panel_copies(upper, n, buf, ldd, (uint8_t *)a, lda, es, cudaMemcpyHostToDevice, s, &e);
        if (e == cudaSuccess) {
            st = tri_inv_ex(uplo, diag, n, buf, ldd, dtype, need ? buf + mat : nullptr, need, nullptr, stream);
            if (st == TRI_OK)
                moved += host_panel_copies(upper, n, buf, ldd, (uint8_t *)a, lda, es, cudaMemcpyDeviceToHost, s, &e);
        }
    }
    const cudaError_t ef = cudaFreeAsync(buf, s);
    const cudaError_t es2 = cudaStreamSynchronize(s);
    if (st == TRI_OK && (e != cudaSuccess || ef != cudaSuccess || es2 != cudaSuccess)) st = TRI_ERR_CUDA;
    if (bytes_moved) *bytes_moved = moved;
    return st;
}

tri_status tri_inv_combrit(tri_uplo uplo, tri_diag diag, int64_t n, void *a, int64_t lda, tri_dtype dtype,
                           int beta, void *stream) {
    if (!valid_enums(uplo, diag, dtype) || n < 0 || !(beta == 2 || beta == 4 || beta == 8 || beta == 16)) return TRI_ERR_ARG;
    if (dtype == TRI_F32_MIXED) return TRI_ERR_UNSUPPORTED;
    if (n == 0) return TRI_OK;
    if (!a || lda < std::max<int64_t>(1, n)) return TRI_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Ctx c;
    tri_status st = device_ctx(s, &c);
    if (st != TRI_OK) return st;
    const size_t need = combrit_ws_bytes(n, dtype, beta);
    void *ws = nullptr;
    if (need > 0 && lib_malloc_async(&ws, need, s) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_NOMEM;
    }
    st = run_combrit(c, dtype, uplo == TRI_UPPER, diag == TRI_UNIT, n, a, lda, beta, ws);
    if (ws && cudaFreeAsync(ws, s) != cudaSuccess && st == TRI_OK) st = TRI_ERR_CUDA;
    return st;
}

size_t gen_inv_workspace_size(int64_t n, tri_dtype dtype) {
    if (n <= 0 || !valid_enums(TRI_LOWER, TRI_NONUNIT, dtype)) return 0;
    return gen_inv_ws_bytes(n, dtype);
}

tri_status gen_inv_ex(int64_t n, void *a, int64_t lda, tri_dtype dtype, void *workspace, size_t ws_bytes,
                      int64_t *d_info, void *stream) {
    if (!valid_enums(TRI_LOWER, TRI_NONUNIT, dtype) || n < 0) return TRI_ERR_ARG;
    if (n == 0) return TRI_OK;
    if (!a || lda < std::max<int64_t>(1, n)) return TRI_ERR_ARG;
    if (n > (int64_t)1 << 30) return TRI_ERR_UNSUPPORTED;
    const size_t need = gen_inv_ws_bytes(n, dtype);
    if (ws_bytes < need || !workspace || ((uintptr_t)workspace & 255)) return TRI_ERR_NOMEM;
    Ctx c;
    tri_status st = device_ctx((cudaStream_t)stream, &c);
    if (st != TRI_OK) return st;
    if ((st = info_begin(c, d_info)) != TRI_OK) return st;
    return info_end(c, d_info, run_gen_inv(c, dtype, n, a, lda, workspace));
}

tri_status gen_inv(int64_t n, void *a, int64_t lda, tri_dtype dtype, void *stream) {
    if (!valid_enums(TRI_LOWER, TRI_NONUNIT, dtype) || n < 0) return TRI_ERR_ARG;
    if (n == 0) return TRI_OK;
    if (!a || lda < std::max<int64_t>(1, n)) return TRI_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Ctx c;
    tri_status st = device_ctx(s, &c);
    if (st != TRI_OK) return st;
    const size_t need = gen_inv_ws_bytes(n, dtype);
    void *ws = nullptr;
    if (lib_malloc_async(&ws, need, s) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_NOMEM;
    }
    st = gen_inv_ex(n, a, lda, dtype, ws, need, nullptr, stream);
    cudaError_t e = cudaFreeAsync(ws, s);
    if (st == TRI_OK && e != cudaSuccess) st = TRI_ERR_CUDA;
    return st;
}

size_t brsi_inv_workspace_size(int64_t n, int gamma, tri_dtype dtype) {
    if (n <= 0 || gamma < 2 || gamma > 16 || !valid_enums(TRI_LOWER, TRI_NONUNIT, dtype)) return 0;
    return brsi_ws_bytes(n, gamma, dtype);
}

static bool valid_perm(int64_t n, const int64_t *perm) {
    if (!perm) return true;
    std::vector<char> seen((size_t)n, 0);
    for (int64_t j = 0; j < n; ++j) {
        if (perm[j] < 0 || perm[j] >= n || seen[(size_t)perm[j]]) return false;
        seen[(size_t)perm[j]] = 1;
    }
    return true;
}

tri_status brsi_inv_ex(int64_t n, void *a, int64_t lda, int gamma, const int64_t *perm, tri_dtype dtype,
                       void *workspace, size_t ws_bytes, int64_t *d_info, void *stream) {
    if (!valid_enums(TRI_LOWER, TRI_NONUNIT, dtype) || n < 0 || gamma < 2 || gamma > 16) return TRI_ERR_ARG;
    if (n == 0) return TRI_OK;
    if (!a || lda < std::max<int64_t>(1, n) || !valid_perm(n, perm)) return TRI_ERR_ARG;
    if (n > 65535) return TRI_ERR_UNSUPPORTED;
    const size_t need = brsi_ws_bytes(n, gamma, dtype);
    if (ws_bytes < need || !workspace || ((uintptr_t)workspace & 255)) return TRI_ERR_NOMEM;
    Ctx c;
    tri_status st = device_ctx((cudaStream_t)stream, &c);
    if (st != TRI_OK) return st;
    if ((st = info_begin(c, d_info)) != TRI_OK) return st;
    return info_end(c, d_info, run_brsi(c, dtype, n, a, lda, gamma, perm, workspace));
}

tri_status brsi_inv(int64_t n, void *a, int64_t lda, int gamma, const int64_t *perm, tri_dtype dtype,
                    void *stream) {
    if (!valid_enums(TRI_LOWER, TRI_NONUNIT, dtype) || n < 0 || gamma < 2 || gamma > 16) return TRI_ERR_ARG;
    if (n == 0) return TRI_OK;
    if (!a || lda < std::max<int64_t>(1, n) || !valid_perm(n, perm)) return TRI_ERR_ARG;
    if (n > 65535) return TRI_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    Ctx c;
    tri_status st = device_ctx(s, &c);
    if (st != TRI_OK) return st;
    const size_t need = brsi_ws_bytes(n, gamma, dtype);
    void *ws = nullptr;
    if (lib_malloc_async(&ws, need, s) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_NOMEM;
    }
    st = brsi_inv_ex(n, a, lda, gamma, perm, dtype, ws, need, nullptr, stream);
    cudaError_t e = cudaFreeAsync(ws, s);
    if (st == TRI_OK && e != cudaSuccess) st = TRI_ERR_CUDA;
    return st;
}

size_t skul_workspace_size(int64_t n, tri_dtype dtype) {
    if (n <= 0 || !valid_enums(TRI_LOWER, TRI_NONUNIT, dtype)) return 0;
    return skul_ws_bytes(n, dtype);
}

tri_status skul_ex(int64_t n, void *a, int64_t lda, void *sk, int64_t ldsk, tri_dtype dtype, void *workspace,
                   size_t ws_bytes, int64_t *d_info, void *stream) {
    if (!valid_enums(TRI_LOWER, TRI_NONUNIT, dtype) || n < 0) return TRI_ERR_ARG;
    if (n == 0) return TRI_OK;
    if (!a || !sk || lda < n || ldsk < n || a == sk) return TRI_ERR_ARG;
    if (n > 65535) return TRI_ERR_UNSUPPORTED;
    const size_t need = skul_ws_bytes(n, dtype);
    if (ws_bytes < need || !workspace || ((uintptr_t)workspace & 255)) return TRI_ERR_NOMEM;
    Ctx c;
    tri_status st = device_ctx((cudaStream_t)stream, &c);
    if (st != TRI_OK) return st;
    if ((st = info_begin(c, d_info)) != TRI_OK) return st;
    return info_end(c, d_info, run_skul(c, dtype, n, a, lda, sk, ldsk, workspace));
}

tri_status skul(int64_t n, void *a, int64_t lda, void *sk, int64_t ldsk, tri_dtype dtype, void *stream) {
    if (!valid_enums(TRI_LOWER, TRI_NONUNIT, dtype) || n < 0) return TRI_ERR_ARG;
    if (n == 0) return TRI_OK;
    if (!a || !sk || lda < n || ldsk < n || a == sk) return TRI_ERR_ARG;
    if (n > 65535) return TRI_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    Ctx c;
    tri_status st = device_ctx(s, &c);
    if (st != TRI_OK) return st;
    const size_t need = skul_ws_bytes(n, dtype);
    void *ws = nullptr;
    if (lib_malloc_async(&ws, need, s) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_NOMEM;
    }
    st = skul_ex(n, a, lda, sk, ldsk, dtype, ws, need, nullptr, stream);
    cudaError_t e = cudaFreeAsync(ws, s);
    if (st == TRI_OK && e != cudaSuccess) st = TRI_ERR_CUDA;
    return st;
}

size_t sqr_workspace_size(int64_t n, tri_dtype dtype) {
    if (n <= 0 || !valid_enums(TRI_LOWER, TRI_NONUNIT, dtype)) return 0;
    return sqr_ws_bytes(n, dtype);
}

static bool overlaps(const void *p, int64_t ldp, const void *q, int64_t ldq, int64_t n, size_t es) {
    const uint8_t *a0 = (const uint8_t *)p, *a1 = a0 + ((size_t)(n - 1) * ldp + n) * es;
    const uint8_t *b0 = (const uint8_t *)q, *b1 = b0 + ((size_t)(n - 1) * ldq + n) * es;
    return a0 < b1 && b0 < a1;
}

tri_status sqr_ex(int64_t n, void *a, int64_t lda, void *r, int64_t ldr, void *s, int64_t lds, tri_dtype dtype,
                  void *workspace, size_t ws_bytes, int64_t *d_info, void *stream) {
    if (!valid_enums(TRI_LOWER, TRI_NONUNIT, dtype) || n < 0) return TRI_ERR_ARG;
    if (n == 0) return TRI_OK;
    if (!a || !r || !s || lda < n || ldr < n || lds < n) return TRI_ERR_ARG;
    const size_t es = dtype == TRI_F64 ? 8 : 4;
    if (overlaps(a, lda, r, ldr, n, es) || overlaps(a, lda, s, lds, n, es) || overlaps(r, ldr, s, lds, n, es))
        return TRI_ERR_ARG;
    if (n > 65535) return TRI_ERR_UNSUPPORTED;
    const size_t need = sqr_ws_bytes(n, dtype);
    if (ws_bytes < need || !workspace || ((uintptr_t)workspace & 255)) return TRI_ERR_NOMEM;
    Ctx c;
    tri_status st = device_ctx((cudaStream_t)stream, &c);
    if (st != TRI_OK) return st;
    if ((st = info_begin(c, d_info)) != TRI_OK) return st;
    return info_end(c, d_info, run_sqr(c, dtype, n, a, lda, r, ldr, s, lds, workspace));
}

tri_status sqr(int64_t n, void *a, int64_t lda, void *r, int64_t ldr, void *s, int64_t lds, tri_dtype dtype,
               void *stream) {
    if (!valid_enums(TRI_LOWER, TRI_NONUNIT, dtype) || n < 0) return TRI_ERR_ARG;
    if (n == 0) return TRI_OK;
    cudaStream_t cs = (cudaStream_t)stream;
    if (!a || !r || !s || lda < n || ldr < n || lds < n) return TRI_ERR_ARG;
    if (n > 65535) return TRI_ERR_UNSUPPORTED;
    Ctx c;
    tri_status st = device_ctx(cs, &c);
    if (st != TRI_OK) return st;
    const size_t need = sqr_ws_bytes(n, dtype);
    void *ws = nullptr;
    if (lib_malloc_async(&ws, need, cs) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_NOMEM;
    }
    st = sqr_ex(n, a, lda, r, ldr, s, lds, dtype, ws, need, nullptr, stream);
    cudaError_t e = cudaFreeAsync(ws, cs);
    if (st == TRI_OK && e != cudaSuccess) st = TRI_ERR_CUDA;
    return st;
}

tri_status sqr_inv(int64_t n, void *a, int64_t lda, tri_dtype dtype, void *stream) {
    if (!valid_enums(TRI_LOWER, TRI_NONUNIT, dtype) || n < 0) return TRI_ERR_ARG;
    if (n == 0) return TRI_OK;
    if (!a || lda < n) return TRI_ERR_ARG;
    if (n > 65535) return TRI_ERR_UNSUPPORTED;
    cudaStream_t cs = (cudaStream_t)stream;
    Ctx c;
    tri_status st = device_ctx(cs, &c);
    if (st != TRI_OK) return st;
    const size_t need = sqr_inv_ws_bytes(n, dtype);
    void *ws = nullptr;
    if (lib_malloc_async(&ws, need, cs) != cudaSuccess) {
        cudaGetLastError();
        return TRI_ERR_NOMEM;
    }
    st = run_sqr_inv(c, dtype, n, a, lda, ws);
    cudaError_t e = cudaFreeAsync(ws, cs);
    if (st == TRI_OK && e != cudaSuccess) st = TRI_ERR_CUDA;
    return st;
}

tri_status tri_get_info(void *stream, int64_t *first_bad_index) {
    Ctx c;
    tri_status st = device_ctx((cudaStream_t)stream, &c);
    if (st != TRI_OK) return st;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return TRI_ERR_CUDA;
    long long info = LLONG_MAX;
    int tmo = 0;
    if (cudaMemcpy(&info, c.info, sizeof(info), cudaMemcpyDeviceToHost) != cudaSuccess) return TRI_ERR_CUDA;
    if (cudaMemcpy(&tmo, c.timeout, sizeof(tmo), cudaMemcpyDeviceToHost) != cudaSuccess) return TRI_ERR_CUDA;
    const long long none = LLONG_MAX;
    const int zero = 0;
    if (cudaMemcpy(c.info, &none, sizeof(none), cudaMemcpyHostToDevice) != cudaSuccess) return TRI_ERR_CUDA;
    if (cudaMemcpy(c.timeout, &zero, sizeof(zero), cudaMemcpyHostToDevice) != cudaSuccess) return TRI_ERR_CUDA;
    if (first_bad_index) *first_bad_index = (info == LLONG_MAX) ? -1 : (int64_t)info;
    if (tmo) return TRI_ERR_TIMEOUT;
    if (info != LLONG_MAX) return TRI_ERR_SINGULAR;
    return TRI_OK;
}

tri_status tri_set_growth_limit(double tau) {
    if (tau != tau) return TRI_ERR_ARG;
    g_growth_tau.store(tau > 0.0 ? (float)std::min(tau, 3.0e38) : 0.f, std::memory_order_relaxed);
    return TRI_OK;
}

double tri_growth_limit(void) { return (double)g_growth_tau.load(std::memory_order_relaxed); }

tri_status tri_set_mixed_recipe(int recipe) {
    if (recipe != TRI_RECIPE_NEWTON_SCHULZ && recipe != TRI_RECIPE_DIRECT) return TRI_ERR_ARG;
    g_recipe.store(recipe, std::memory_order_relaxed);
    return TRI_OK;
}

int tri_mixed_recipe(void) { return g_recipe.load(std::memory_order_relaxed); }

tri_status tri_set_cta_pairs(int mask) {
    if (mask & ~(TRI_PAIR_LEVELS | TRI_PAIR_RES | TRI_PAIR_UPD)) return TRI_ERR_ARG;
    g_pairs.store(mask, std::memory_order_relaxed);
    return TRI_OK;
}

int tri_cta_pairs(void) { return g_pairs.load(std::memory_order_relaxed); }

int tri_cta_pair_capacity(void) {
    Ctx c;
    if (device_ctx_public(nullptr, &c) != TRI_OK) return 0;
    return tc::pair_lists(c);
}

tri_status tri_pool_stats(uint64_t *used, uint64_t *used_high, int reset_high) {
    cudaMemPool_t pool;
    if (lib_pool(&pool) != cudaSuccess) return TRI_ERR_CUDA;
    uint64_t v = 0;
    if (used) {
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v) != cudaSuccess) return TRI_ERR_CUDA;
        *used = v;
    }
    if (used_high) {
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v) != cudaSuccess) return TRI_ERR_CUDA;
        *used_high = v;
    }
    if (reset_high) {
        v = 0;
        if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v) != cudaSuccess) return TRI_ERR_CUDA;
    }
    return TRI_OK;
}

void tri_trace_enable(int on) {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    if (on) clear_trace_locked();
    g_trace_on = on != 0;
}

int64_t tri_trace_report(char *buf, size_t cap) {
    struct Agg { std::string k; int64_t launches; double ms, flops, bytes; };
    std::vector<Agg> agg;
    {
        std::lock_guard<std::mutex> lk(g_trace_mu);
        for (auto &r : g_trace) {
            if (cudaEventSynchronize(r.end) != cudaSuccess) return -1;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.beg, r.end) != cudaSuccess) return -1;
            auto it = std::find_if(agg.begin(), agg.end(), [&](const Agg &a) { return a.k == r.kernel; });
            if (it == agg.end()) {
                agg.push_back({r.kernel, 0, 0.0, 0.0, 0.0});
                it = agg.end() - 1;
            }
            it->launches += 1;
            it->ms += ms;
            it->flops += r.flops;
            it->bytes += r.bytes;
        }
    }
    std::string out = "{";
    for (size_t i = 0; i < agg.size(); ++i) {
        char tmp[512];
        snprintf(tmp, sizeof(tmp), "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f, \"flops\": %.6e, \"bytes\": %.6e}",
                 i ? ", " : "", agg[i].k.c_str(), (long long)agg[i].launches, agg[i].ms, agg[i].flops,
                 agg[i].bytes);
        out += tmp;
    }
    out += "}";
    if (buf && cap) {
        size_t m = std::min(cap - 1, out.size());
        memcpy(buf, out.data(), m);
        buf[m] = 0;
    }
    return (int64_t)out.size();
}

}  // extern "C"
