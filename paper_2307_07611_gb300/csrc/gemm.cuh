// gemm.cuh -- the generic triangular-aware product used by the general inverse and the
// adjoint: C = alpha * A * B + beta * C, column-major, operands full or triangular.
#pragma once

#include "internal.cuh"

namespace triinv {

enum OpKind {
    OP_FULL = 0,
    OP_LOWER = 1,
    OP_UPPER = 2,
    OP_LOWER_UNIT = 3,   // strict lower part stored, diagonal taken as 1
    OP_UPPER_UNIT = 4,
};

struct GemmArgs {
    int64_t m, n, k;
    double alpha;
    const void *a;
    int64_t lda;
    int akind;
    const void *b;
    int64_t ldb;
    int bkind;
    double beta;
    void *c;
    int64_t ldc;
    int cmask;   // OP_FULL, OP_LOWER or OP_UPPER: which part of C is written;
                 // OP_LOWER_UNIT / OP_UPPER_UNIT: the strict triangle, diagonal set to 0
    bool ta = false, tb = false;              // use A^T / B^T (stored column-major)
    int64_t batch = 1;                        // independent products, pointers advanced by
    int64_t sa = 0, sb = 0, sc = 0;           // these strides (elements)
    int64_t batch2 = 1;                       // an outer batch level (product index =
    int64_t sa2 = 0, sb2 = 0, sc2 = 0;        // inner + batch * outer)
    bool split_k = false;                     // FP32 on CUDA cores: allow splitting a long
                                              // k over CTAs (atomic adds, beta == 0 only;
                                              // FP64 always may)
    double dadd = 0.0;                        // tensor-core path only: added to the diagonal
                                              // of C after the product (R = I - A X)
};

double gemm_flops(const GemmArgs &g);

// CUDA-core product (FP32 or FP64 by dt).
cudaError_t gemm_simt(const Ctx &c, tri_dtype dt, const GemmArgs &g, const char *trace_name);

// Split-BF16 tensor-core product (FP32 data): both operands are split into BF16
// hi/mid(/lo) planes inside `ws` and `terms` (1, 3 or 6) pieces are accumulated in FP32;
// six-term products also promote their partial sums to FP32 registers every 64 k, which
// brings them to about 2^-24 relative (FP32 class).
// ws must hold gemm_tc_ws_bytes(m, n, k, g.batch) bytes: the operand planes of one chunk
// of the batch (all matrices of a chunk in one launch).
size_t gemm_tc_ws_bytes(int64_t m, int64_t n, int64_t k, int64_t batch = 1);
cudaError_t gemm_tc(const Ctx &c, const GemmArgs &g, int terms, void *ws, const char *trace_name);

}  // namespace triinv
