// tc_graph.cuh -- interface of the dependency-driven tensor-core kernel (tc_graph.cu) that
// runs all products of the mixed-precision inverse in one persistent launch.
#pragma once

#include "tc_gemm.cuh"

namespace triinv {
namespace tc {

enum GOp {
    G_W = 0,     // W = B X_A (3 terms)            -> W hi / mid planes
    G_X21 = 1,   // X21 = -X_C W (3 terms)         -> X (FP32) and its hi / mid / lo planes
    G_RES = 2,   // R = I - T X (6 terms, promoted) -> R hi plane
    G_UPD = 3,   // X += X R (1 term)              -> X (FP32)
};

// One 128 x 256 output tile.  Operands as in Tile; deps[dep0 .. dep1) are the ready
// counters it waits on; out_flag the counter it publishes (-1: none); xin_flag the
// counter of the FP32 X region an update tile reads (-1: none or written before launch).
struct GTile {
    int am, ak, bk, bn, kb0, kb1, om, on;
    int op, dep0, dep1, out_flag, xin_flag, pad0, pad1, pad2;
};

// Targets: all planes are n x n column-major BF16 with leading dimension ldp (lower view
// of the matrix); X in FP32 is the caller's matrix (lda, TRANS view).
struct GEpi {
    float *x;
    int64_t ldx;
    __nv_bfloat16 *xp0, *xp1, *xp2, *wp0, *wp1, *rp;
    int64_t ldp, n;
    int *flags;        // 3 * nrb * ncb ready counters (X, W, R), zeroed by launch_graph
    int *abort_word;   // flags[3 * nrb * ncb], zeroed with them
    unsigned long long *timeline;   // per-tile records while tracing (else null)
    // Failure-path testing: the counter index whose publication is withheld (-1: none) and
    // the deadline of every wait (ns).
    int withhold = -1;
    unsigned long long limit_ns = 4000000000ull;
};

// Per-tile timeline record written while tracing (list order, kTimelineWords words):
//   [0] cta | op << 16 | k-blocks << 20 | (om / 128) << 32 | (on / 256) << 48
//   [1] producer starts waiting for the tile's regions, [2] first TMA load issued,
//   [3] MMA issuer starts the tile, [4] last MMA of the tile issued,
//   [5] epilogue warp 2 done (region published); times from %globaltimer (ns).
constexpr int kTimelineWords = 6;

struct GraphPlan {
    GTile *d_tiles = nullptr;   // per-CTA lists, concatenated
    int *d_off = nullptr;       // ctas + 1 list offsets
    int *d_deps = nullptr;      // counter indices
    int ctas = 0, ntiles = 0, nrb = 0, ncb = 0;
    double flops = 0.0;             // algorithmic flops of all products
    double model_makespan = 0.0;    // schedule length in pipeline slots (cost model)
};

// Bytes of the ready counters plus the abort word for order n.
size_t graph_flag_bytes(int64_t n);

// Tile DAG and schedule for order n on `sm_count` CTAs, built once per (device, n).
tri_status graph_plan(int dev, int sm_count, int64_t n, const GraphPlan **out);

// Zeroes the counters on c.stream and launches the kernel.  tpl: T hi / mid / lo planes.
cudaError_t launch_graph(const Ctx &c, bool trans, bool unit, int64_t n, const GraphPlan &p,
                         const __nv_bfloat16 *const tpl[3], const GEpi &ep);

}  // namespace tc
}  // namespace triinv
