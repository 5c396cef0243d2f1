// internal.cuh -- declarations shared by the library's translation units.
// Not part of the public ABI (include/triinv.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "triinv.h"

namespace triinv {

// Per-call launch context.
struct Ctx {
    cudaStream_t stream;
    long long *info;   // device: smallest bad pivot index seen (LLONG_MAX = none)
    int *timeout;      // device: set to 1 when a bounded wait runs out
    int sm_count;
    int device;
    float tau;         // growth limit of the FP64 fallback for ill-conditioned diagonal
                       // blocks (tri_set_growth_limit; <= 0 disables)
    int recipe;        // TRI_F32_MIXED recipe of the triangular path (tri_set_mixed_recipe)
    int pairs;         // products of the mixed path run on CTA pairs (tri_set_cta_pairs)
};

// Lower-orientation view of a column-major matrix.  For an upper-triangular matrix U
// stored column-major, the lower view is U^T, i.e. element (i, j) of the view lives at
// p[j + i*ld] (trans == true).  Section 2 of the paper: the lower case is the transpose
// of the upper one.
template <bool TRANS>
__host__ __device__ __forceinline__ int64_t vidx(int64_t i, int64_t j, int64_t ld) {
    return TRANS ? (j + i * ld) : (i + j * ld);
}

// Launch context of the calling thread's current device (api.cu).
tri_status device_ctx_public(cudaStream_t stream, Ctx *out);

// Stream-ordered scratch from the library's private pool of the current device (api.cu);
// release it with cudaFreeAsync.
cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t s);

// Per-call status word of the _ex entry points (api.cu).  d_info == nullptr keeps the
// device-wide word of c.  Otherwise info_begin points c.info at the caller's word and
// queues its reset; info_end queues the conversion of "no bad pivot" to -1 (when st is OK)
// and returns st.
tri_status info_begin(Ctx &c, int64_t *d_info);
tri_status info_end(const Ctx &c, int64_t *d_info, tri_status st);

// ---- tracing (api.cu) -------------------------------------------------------------
// While tracing is on, TraceScope records a CUDA event pair around the launches made in
// its lifetime on `stream`, and books the launch's algorithmic flops and bytes.
// True while kernel tracing is enabled (tri_trace_enable).
bool trace_on();

struct TraceScope {
    int slot;
    TraceScope(cudaStream_t stream, const char *kernel, double flops, double bytes);
    ~TraceScope();
    cudaStream_t stream_;
};

// ---- leaf inverse (leaf.cu) -------------------------------------------------------
// Inverts every diagonal block [q*leaf, min(q*leaf+leaf, n)) of the lower view in place
// by the column recurrence.  leaf must be 16, 32 or 64.
// batch > 1: `batch` matrices `bstride` elements apart (grid.y); singular pivots then
// record the matrix index instead of the row.
cudaError_t launch_leaf(const Ctx &c, tri_dtype dt, bool trans, bool unit, int64_t n,
                        void *a, int64_t lda, int leaf, int64_t batch = 1, int64_t bstride = 0);

// ---- SIMT level products (trmm_simt.cu) -------------------------------------------
// One split level with half-size h: for every active pair q (A-block at q*2h, C-block
// at q*2h+h, clipped to n):
//   mode 0:  W_q = B_q * X_A        (B_q: rows of C x cols of A; X_A lower)
//   mode 1:  B_q <- -X_C * W_q      (X_C lower)
// W is column-major with leading dimension h, pair q at offset q*h*h.
// batch > 1: matrices `bstride` elements apart; W of matrix b at b * pairs * h * h.
cudaError_t launch_trmm_level(const Ctx &c, tri_dtype dt, bool trans, bool unit, int mode,
                              int64_t n, void *a, int64_t lda, int64_t h, void *w,
                              int64_t batch = 1, int64_t bstride = 0);

// Copies in flight that write parts of the input matrix of the mixed path (tri_inv_host):
// the inverse waits for each part only where it first reads it.  ready[0]: the diagonal
// 256-blocks and the B blocks of the first mixed_head_levels() split levels; ready[1 + k]:
// the B blocks of level mixed_head_levels() + k (half-size 256 * 2^level).
struct InputFeed {
    const cudaEvent_t *ready;
    int count;
};
// Where the result of the mixed path is final early (tri_inv_host): with groups > 1 the
// Newton-Schulz update runs in column groups from the right, and done[g] is recorded on
// the stream after group g, whose columns [col_lo[g], col_hi[g]) (multiples of 256) are
// then final.  The callee sets `got` (0: no groups, the result is final at the end).
struct OutputDrain {
    int groups;                  // wanted (at most 8)
    const cudaEvent_t *done;     // groups events
    int got;
    int64_t col_lo[8], col_hi[8];
};
int mixed_head_levels();
tri_status run_mixed_fed(const Ctx &c, bool trans, bool unit, int64_t n, float *a, int64_t lda, void *ws,
                         const InputFeed *feed, OutputDrain *drain = nullptr);

// Number of active pairs at split half-size h.
inline int64_t level_pairs(int64_t n, int64_t h) {
    return n > h ? (n - h + 2 * h - 1) / (2 * h) : 0;
}

}  // namespace triinv
