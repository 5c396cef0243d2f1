/*
 * triinv.h -- C ABI of the GB300 (sm_103a) triangular-inversion library.
 *
 * The library inverts a non-singular triangular matrix T by the recursive triangular
 * split of arXiv 2307.07611 (COMBRIT with block count 2, Section 4.1, Algorithm
 * "COMBRIT"; the block inverse of the proof of the main Theorem, Section 3):
 *
 *     T = [A 0; B C]   ->   T^-1 = [A^-1 0; -C^-1 B A^-1  C^-1]
 *
 * The diagonal leaf blocks are inverted by the column recurrence of CRIT (Section 4.2,
 * Algorithm "CRIT", transposed to lower form):
 *     x_jj = 1/t_jj,   x_ij = -(1/t_ii) * sum_{k=j}^{i-1} t_ik x_kj   (i > j)
 * and the off-diagonal blocks by two dense products per split (Section 4.1, Eq.
 * "ptfm" counts one of them as m^3 flops).
 *
 * Conventions shared by every entry point:
 *   - Matrices are COLUMN-MAJOR: element (i, j) of a matrix with leading dimension ld
 *     is ptr[i + j*ld].  Pointers passed as `void*` data are DEVICE pointers unless a
 *     comment says "host".
 *   - Only the triangle named by `uplo` is read and written (LAPACK trtri semantics);
 *     the other triangle is never touched.  With TRI_UNIT the diagonal is taken as 1
 *     and neither read nor written.
 *   - `stream` is a cudaStream_t passed as `void*`; NULL is the legacy default stream.
 *     Every call is asynchronous on `stream`: a returned TRI_OK means the work was
 *     queued (argument errors are detected and returned before anything is queued).
 *   - The caller owns all memory it passes.  The library never frees caller memory.
 *     Internal scratch comes from the `_ex` workspace argument or, in the plain entry
 *     points, from the library's own stream-ordered memory pool on the current device
 *     (created on first use; freed blocks stay cached in it for later calls; the
 *     device's default pool is not touched).  TRI_ERR_NOMEM if that allocation fails.
 *   - A zero or non-finite pivot (t_ii, or a pivot of the LU in gen_inv) does not stop
 *     the queued work; its index is recorded on the device (smallest index wins).  The
 *     result is then unspecified.  No pivoting is done and there is no small-pivot
 *     threshold.  Where the index goes:
 *       * `_ex` entry points with a non-NULL `d_info` (a DEVICE pointer to one int64_t
 *         that the call owns until its work completes): the call queues a reset of
 *         *d_info, its kernels record into it, and a last kernel leaves -1 there if no
 *         pivot was bad.  Nothing else is touched, so calls on different streams with
 *         their own words do not see each other's pivots.  Read it after the stream
 *         has reached the end of the call (e.g. cudaStreamSynchronize, or an event).
 *       * every other call: one status word per device, reported and cleared by
 *         tri_get_info() -- shared by all streams and host threads using the device.
 *   - Every wait inside a kernel is bounded; a wait that runs out records
 *     TRI_ERR_TIMEOUT, reported by tri_get_info().
 */
#ifndef TRIINV_H
#define TRIINV_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TRI_API __attribute__((visibility("default")))
#else
#define TRI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TRI_OK = 0,
    TRI_ERR_ARG = 1,         /* invalid argument (nothing was queued)                    */
    TRI_ERR_SINGULAR = 2,    /* zero or non-finite pivot (from tri_get_info)             */
    TRI_ERR_NOMEM = 3,       /* scratch allocation failed / workspace too small          */
    TRI_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed              */
    TRI_ERR_TIMEOUT = 5,     /* a bounded device wait ran out (from tri_get_info)        */
    TRI_ERR_UNSUPPORTED = 6  /* valid request this build does not provide                */
} tri_status;

typedef enum { TRI_LOWER = 0, TRI_UPPER = 1 } tri_uplo;
typedef enum { TRI_NONUNIT = 0, TRI_UNIT = 1 } tri_diag;

typedef enum {
    TRI_F64 = 0,       /* FP64 storage, FP64 leaf recurrence and DFMA products; small
                          products split k over several CTAs and add the partial sums
                          atomically, so results may differ between runs in the last
                          bits                                                            */
    TRI_F32 = 1,       /* FP32 storage, FP32 leaf recurrence and FFMA products ("plain")  */
    TRI_F32_MIXED = 2  /* FP32 storage; split-BF16 tensor-core products with FP32
                          accumulation, then one Newton-Schulz step X <- X + X(I - TX)    */
} tri_dtype;

/* Human-readable name of a status code (static string, never NULL). */
TRI_API const char *tri_status_string(tri_status s);

/* Library version string, e.g. "0.1.0 sm_103a". */
TRI_API const char *tri_version(void);

/* ---------------------------------------------------------------------------------
 * Single triangular inverse, in place: A <- A^-1 on the `uplo` triangle.
 *   uplo  TRI_LOWER: A is lower triangular; TRI_UPPER: upper (handled as the transpose
 *         of a lower matrix, Section 2 of the paper).
 *   diag  TRI_UNIT: unit diagonal, not referenced.
 *   n     order, n >= 0 (n == 0 is a no-op).
 *   a     device pointer to an lda x n column-major matrix (FP64 for TRI_F64, FP32
 *         otherwise).
 *   lda   leading dimension, lda >= max(1, n).
 * Errors: TRI_ERR_ARG for bad enums, n < 0, lda < max(1,n) or a == NULL with n > 0;
 *         TRI_ERR_NOMEM if scratch cannot be allocated; TRI_ERR_CUDA on a launch error.
 * --------------------------------------------------------------------------------- */
TRI_API tri_status tri_inv(tri_uplo uplo, tri_diag diag, int64_t n, void *a, int64_t lda,
                   tri_dtype dtype, void *stream);

/* Bytes of scratch tri_inv_ex needs for order n (0 if none).  Scratch must be
 * 256-byte aligned device memory and must not be used by anything else until the
 * queued work completes. */
TRI_API size_t tri_inv_workspace_size(int64_t n, tri_dtype dtype);

/* tri_inv with caller-provided scratch and an optional per-call status word.
 * TRI_ERR_NOMEM if ws_bytes is smaller than tri_inv_workspace_size(n, dtype) or
 * `workspace` is not 256-byte aligned.
 *   d_info  NULL (pivots go to the device-wide word of tri_get_info) or a device int64_t
 *           that receives the first bad pivot index, or -1 (see the conventions above).
 *           A bounded wait that runs out is still reported by tri_get_info. */
TRI_API tri_status tri_inv_ex(tri_uplo uplo, tri_diag diag, int64_t n, void *a, int64_t lda,
                              tri_dtype dtype, void *workspace, size_t ws_bytes, int64_t *d_info,
                              void *stream);

/* ---------------------------------------------------------------------------------
 * General inverse, in place: A <- A^-1 for a dense n x n matrix, as A^-1 = U^-1 L^-1 from
 * an unpivoted block LU (BRSI with two blocks reduced to the Schur complement, Section
 * 5.2; inverse factors S = U^-1, K = L^-1 formed alongside the factorisation as in SKUL,
 * Section 5.1, "S K = A^-1").  Intended for matrices that need no pivoting (e.g. diagonally
 * dominant ones); a zero or non-finite pivot is recorded and reported by tri_get_info.
 *   n     order, n >= 0;  a: device pointer, lda x n column-major;  lda >= max(1, n).
 *   dtype TRI_F64 (DFMA), TRI_F32 (FFMA) or TRI_F32_MIXED (split-BF16 tensor-core
 *         products with three terms and FP32 accumulation, FP32 leaves; for n >= 512
 *         followed by one Newton-Schulz step X <- X + X (I - A X) with a six-term
 *         residual, which brings the result to FP32 accuracy).
 * Errors: TRI_ERR_ARG, TRI_ERR_NOMEM (scratch), TRI_ERR_CUDA.
 * --------------------------------------------------------------------------------- */
TRI_API tri_status gen_inv(int64_t n, void *a, int64_t lda, tri_dtype dtype, void *stream);

/* Bytes of 256-byte aligned device scratch gen_inv_ex needs (about 2 n^2 elements, plus
 * for TRI_F32_MIXED the BF16 operand planes of the largest product and, for n >= 512, a
 * copy of A for the Newton-Schulz residual). */
TRI_API size_t gen_inv_workspace_size(int64_t n, tri_dtype dtype);

/* gen_inv with caller scratch (TRI_ERR_NOMEM if too small or misaligned) and an optional
 * per-call status word d_info (as tri_inv_ex). */
TRI_API tri_status gen_inv_ex(int64_t n, void *a, int64_t lda, tri_dtype dtype, void *workspace,
                              size_t ws_bytes, int64_t *d_info, void *stream);

/* ---------------------------------------------------------------------------------
 * BRSI with gamma blocks (Section 5.2, "Steps of BRSI(gamma)"), in place: A <- A^-1.
 * Step 1: A_0 = A P_0 with the caller's column permutation P_0.  Steps 2-5, gamma - 1
 * times: A_l = M_l + N_l (M_l the block upper part of A_l, diagonal blocks included; N_l
 * the strictly block lower part), A_{l+1} = I + M_l^-1 N_l.  Then A P_0 = M_0 ... M_{g-2} L
 * with L = A_{g-1} block lower triangular, and A^-1 = P_0 L^-1 M_{g-2}^-1 ... M_0^-1.  The
 * diagonal blocks of the M_l and L are inverted by gen_inv (the two-block form: the
 * double recursion of Step 4); the rest are block products.  The work grows with gamma.
 *   n      order, 0 <= n <= 65535;  a: device, lda x n column-major, lda >= max(1, n).
 *   gamma  number of blocks, 2..16 (blocks of ceil(n / gamma) rows, the last ragged).
 *   perm   HOST array of n distinct indices (column j of A P_0 is column perm[j] of A), or
 *          NULL for the identity.  The later permutations P_l of the paper ("as necessary")
 *          are the identity: choose P_0 so that the diagonal blocks of every A_l are
 *          non-singular (e.g. block columns swapped when a diagonal block of A is
 *          singular).  With perm the call copies it from host memory (do not capture).
 *   dtype  TRI_F64 / TRI_F32 (CUDA-core products) or TRI_F32_MIXED (three-term split-BF16
 *          tensor-core products, then one Newton-Schulz step against A for n >= 512).
 * A zero or non-finite pivot in a diagonal-block inverse is reported by tri_get_info (or
 * d_info) as the row of A_l where that block's pivot lies; the result is then unspecified.
 * Errors: TRI_ERR_ARG (bad dtype, n < 0, gamma outside 2..16, null a, small lda, perm not
 * a permutation), TRI_ERR_UNSUPPORTED (n > 65535), TRI_ERR_NOMEM, TRI_ERR_CUDA.
 * --------------------------------------------------------------------------------- */
TRI_API tri_status brsi_inv(int64_t n, void *a, int64_t lda, int gamma, const int64_t *perm, tri_dtype dtype,
                            void *stream);
/* Bytes of 256-byte aligned device scratch brsi_inv_ex needs (4 n^2 elements, the gen_inv
 * scratch of one diagonal block, the BF16 planes of an n x n product for mixed). */
TRI_API size_t brsi_inv_workspace_size(int64_t n, int gamma, tri_dtype dtype);
/* brsi_inv with caller scratch and an optional per-call status word (as tri_inv_ex). */
TRI_API tri_status brsi_inv_ex(int64_t n, void *a, int64_t lda, int gamma, const int64_t *perm, tri_dtype dtype,
                               void *workspace, size_t ws_bytes, int64_t *d_info, void *stream);

/* ---------------------------------------------------------------------------------
 * SKUL (Algorithm SKUL, Section 5.1): the unpivoted Crout factorisation A = L U together
 * with the inverse factors K = L^-1 and S = U^-1, so that A^-1 = S K, for preconditioners
 * that want the direct and the inverse factors at once.  Computed block-recursively as in
 * gen_inv (the factors are kept instead of multiplied out), then put in Crout form.
 *   n     order, 0 <= n <= 65535.
 *   a     device, lda x n column-major, lda >= n.  In: A.  Out: L on and below the
 *         diagonal (non-unit), U strictly above it (its unit diagonal is not stored).
 *   sk    device, ldsk x n column-major, ldsk >= n, not overlapping a.  Out only: K on
 *         and below the diagonal, S strictly above it (unit diagonal not stored).
 *   dtype TRI_F64, TRI_F32 or TRI_F32_MIXED (as gen_inv).
 * Same pivot rule as gen_inv: no pivoting, a zero or non-finite pivot is reported by
 * tri_get_info (its factors are then not meaningful).
 * Errors: TRI_ERR_ARG (bad enum, n < 0, null pointers, small leading dimensions, a == sk),
 *         TRI_ERR_UNSUPPORTED (n > 65535), TRI_ERR_NOMEM, TRI_ERR_CUDA.
 * --------------------------------------------------------------------------------- */
TRI_API tri_status skul(int64_t n, void *a, int64_t lda, void *sk, int64_t ldsk, tri_dtype dtype,
                        void *stream);

/* Bytes of 256-byte aligned device scratch skul_ex needs (the product temporaries of the
 * recursion, the BF16 planes for TRI_F32_MIXED and n elements for the pivots). */
TRI_API size_t skul_workspace_size(int64_t n, tri_dtype dtype);

/* skul with caller scratch (TRI_ERR_NOMEM if too small or misaligned) and an optional
 * per-call status word d_info (as tri_inv_ex). */
TRI_API tri_status skul_ex(int64_t n, void *a, int64_t lda, void *sk, int64_t ldsk, tri_dtype dtype,
                           void *workspace, size_t ws_bytes, int64_t *d_info, void *stream);

/* ---------------------------------------------------------------------------------
 * SQR (Algorithm SQR, Section 5.1): A = Q R (Q orthonormal, R upper with a positive
 * diagonal) together with S = R^-1, so that A^-1 = S Q^T.  No pivoting is needed: any
 * non-singular A whose column blocks are not too ill-conditioned (see below) factors.
 * Built over blocks of columns (recursive block Gram-Schmidt with one
 * re-orthogonalisation, S formed as each block column of R completes; leaves of 64
 * columns, 32 in FP64, by Cholesky QR run twice).
 *   n     order, 0 <= n <= 65535.
 *   a     device, lda x n column-major, lda >= n.  In: A.  Out: Q.
 *   r, s  device, ldr / lds x n column-major (>= n), out only: R and S = R^-1 on and
 *         above the diagonal, zero below.  a, r and s must not overlap.
 *   dtype TRI_F64, TRI_F32 or TRI_F32_MIXED (the block products Q1^T A2, Q1 R12, S11 R12
 *         S22 on the tensor cores with three-term split BF16, where they are large).
 * A column j whose leaf Gram matrix has a pivot that is not positive and finite (A
 * singular, or a leaf block with condition number beyond about u^-1/2) is reported by
 * tri_get_info as index j; the factors are then not meaningful.
 * Errors: TRI_ERR_ARG (bad enum, n < 0, null pointers, small leading dimensions,
 *         overlapping buffers), TRI_ERR_UNSUPPORTED (n > 65535), TRI_ERR_NOMEM,
 *         TRI_ERR_CUDA.
 * --------------------------------------------------------------------------------- */
TRI_API tri_status sqr(int64_t n, void *a, int64_t lda, void *r, int64_t ldr, void *s, int64_t lds,
                       tri_dtype dtype, void *stream);

/* Bytes of 256-byte aligned device scratch sqr_ex needs. */
TRI_API size_t sqr_workspace_size(int64_t n, tri_dtype dtype);

/* sqr with caller scratch (TRI_ERR_NOMEM if too small or misaligned) and an optional
 * per-call status word d_info (as tri_inv_ex). */
TRI_API tri_status sqr_ex(int64_t n, void *a, int64_t lda, void *r, int64_t ldr, void *s, int64_t lds,
                          tri_dtype dtype, void *workspace, size_t ws_bytes, int64_t *d_info, void *stream);

/* General inverse through SQR, in place: A <- A^-1 = S Q^T (Section 5.1, "S Q^t =
 * A^-1").  Same arguments, conditions and errors as gen_inv; scratch (about 3 n^2
 * elements, plus BF16 planes for TRI_F32_MIXED) is allocated on the stream. */
TRI_API tri_status sqr_inv(int64_t n, void *a, int64_t lda, tri_dtype dtype, void *stream);

/* ---------------------------------------------------------------------------------
 * Batched triangular inverses of uneven sizes, in place (block-Jacobi preconditioners):
 * every block is inverted by the recursive split (Section 4.1, block count 2) with CRIT
 * leaves (Section 4.2), entirely in shared memory, inside ONE persistent kernel whose
 * CTAs take blocks from an atomic queue, largest first.
 *   count  number of blocks (>= 0);  sizes: HOST array of count orders (0 <= n_i <= 256
 *          for FP32, <= 128 for FP64, else TRI_ERR_UNSUPPORTED);  ptrs: HOST array of
 *          count DEVICE pointers, block i column-major with leading dimension n_i.
 *   uplo, diag apply to every block; dtype TRI_F32 (TRI_F32_MIXED is the same FP32
 *   path: blocks of at most 256 are far below the size where split products pay) or
 *   TRI_F64.
 * Singular blocks: the smallest index i of a block with a zero or non-finite pivot is
 * recorded and reported by tri_get_info (as the "index").
 *
 * tri_batched_plan_create uploads the descriptors (sorted by size), picks the thread
 * count by timing the candidates on a scratch batch of the same sizes (the caller's data
 * is not touched), and captures {queue reset, persistent kernel} in a CUDA graph.  It
 * allocates device memory and synchronises; call it outside stream capture.
 * tri_batched_exec replays the graph on `stream` (asynchronous; the blocks must not be
 * in use by other work).  tri_batched_plan_destroy frees the plan (after the last
 * tri_batched_exec that uses it has completed).
 * tri_inv_batched = create + exec + synchronise `stream` + destroy.
 * --------------------------------------------------------------------------------- */
typedef struct tri_batched_plan tri_batched_plan;
TRI_API tri_status tri_batched_plan_create(int64_t count, const int64_t *sizes, void *const *ptrs,
                                           tri_uplo uplo, tri_diag diag, tri_dtype dtype,
                                           tri_batched_plan **out);
TRI_API tri_status tri_batched_exec(tri_batched_plan *plan, void *stream);
TRI_API tri_status tri_batched_plan_destroy(tri_batched_plan *plan);
/* Thread count the autotuner chose for the plan's largest size class (diagnostic). */
TRI_API int tri_batched_plan_threads(const tri_batched_plan *plan);

/* The plan's CTA shape per size class (diagnostic): the blocks are split into classes,
 * each its own persistent launch over a largest-first queue, replayed in order:
 *   cls 0: 161..256 rows (FP32) -- 8 x 8 tiles of 32, one CTA per SM, 256 or 512 threads;
 *   cls 1: 129..160 rows (FP32) -- 5 x 5 tiles, two CTAs per SM, 256 or 512 threads;
 *   cls 2: 33..128 rows -- 4 x 4 tiles, several CTAs per SM, 128 or 256 threads;
 *   cls 3: up to 32 rows -- one tile, 32 or 64 threads, many CTAs per SM.
 * The autotuner times each candidate thread count (with the CTAs that fit beside it) on a
 * scratch copy of the class's sizes when the plan is created and keeps the fastest.
 * blocks / threads / ctas (each may be NULL): the class's block count, threads per CTA
 * and persistent CTAs.  Errors: TRI_ERR_ARG (null plan, cls outside 0..3). */
TRI_API tri_status tri_batched_plan_shape(const tri_batched_plan *plan, int cls, int *blocks, int *threads,
                                          int *ctas);

/* The autotuner's choices of this process (keyed by GPU model and SM count, dtype, size
 * class and the histogram of the class's sizes) written to / read from a JSON file, so a
 * later process skips the timing runs for batches it has seen.  Load merges into the
 * process's cache (loaded: entries read; may be NULL).  Errors: TRI_ERR_ARG (null path,
 * file not writable / readable, malformed entry). */
TRI_API tri_status tri_tune_cache_save(const char *path);
TRI_API tri_status tri_tune_cache_load(const char *path, int *loaded);

/* Growth limit of an FP32 plan: an FP64 leaf only for ill-conditioned blocks.  After a
 * block's FP32 inverse, if max|X| * max|T| > tau (a lower bound of its condition number
 * in the max norm) and the block has at most 128 rows, the block (still unchanged in
 * memory) is inverted again in FP64 in shared memory and that result, rounded to FP32, is
 * stored; larger blocks keep the FP32 result.  Default 1e4 for TRI_F32 and TRI_F32_MIXED
 * plans (which run in FP32); tau <= 0 disables.  Synchronous; applies to later
 * tri_batched_exec calls of the plan.
 * Errors: TRI_ERR_ARG (null plan, NaN tau, another device current),
 *         TRI_ERR_UNSUPPORTED (TRI_F64 plan). */
TRI_API tri_status tri_batched_plan_set_growth_limit(tri_batched_plan *plan, double tau);
TRI_API tri_status tri_inv_batched(int64_t count, const int64_t *sizes, void *const *ptrs,
                                   tri_uplo uplo, tri_diag diag, tri_dtype dtype, void *stream);

/* Partition of a batch over the ranks of a multi-GPU job (host only, no CUDA call).
 * The blocks are independent, so each rank inverts its own share with no collective.
 * owner[i] (HOST array of count int32) receives the rank of block i: blocks taken by
 * decreasing order sizes[i], each given to the rank with the smallest sum of m^3 so far
 * (cost of the recursive split, Section 4.1: m^3/3 flops), ties to the lower rank.  Every
 * rank computes the same assignment from the same sizes.  loads (HOST, world doubles, may
 * be NULL) receives each rank's sum of m^3.
 * Errors: TRI_ERR_ARG (count < 0, world < 1, null arrays, a negative size). */
TRI_API tri_status tri_batched_partition(int64_t count, const int64_t *sizes, int world, int32_t *owner,
                                         double *loads);

/* ---------------------------------------------------------------------------------
 * tri_inv_combrit -- the same in-place inverse by Algorithm COMBRIT (Section 4.1) with
 * `beta` diagonal blocks per recursion level (beta = 2, 4, 8 or 16; beta = 2 is the split of
 * tri_inv).  Per level, with the beta diagonal inverses X_ii in place: B_ij = X_ii T_ij
 * (the unit block form T*), the unit block inverse W = B^-1 by the block version of the
 * main Theorem (Section 3), then X_ij = W_ij X_jj.  Leaves (64, FP64: 16) use the CRIT
 * recurrence.  TRI_F32 / TRI_F64 only (CUDA-core products); scratch for the B and W
 * blocks of one level (at most n*n elements) comes from the stream-ordered allocator.
 * Errors: as tri_inv; TRI_ERR_ARG for beta not in {2, 4, 8, 16}; TRI_ERR_UNSUPPORTED for
 * TRI_F32_MIXED.
 * --------------------------------------------------------------------------------- */
TRI_API tri_status tri_inv_combrit(tri_uplo uplo, tri_diag diag, int64_t n, void *a, int64_t lda,
                                   tri_dtype dtype, int beta, void *stream);

/* ---------------------------------------------------------------------------------
 * tri_inv_host -- tri_inv on a matrix in HOST memory (the same in-place operation, the
 * same split, Section 3 / Algorithm COMBRIT with beta = 2): the referenced triangle is
 * copied to the device in 256-column panels (one 2-D copy each, about half of the n x n
 * matrix), inverted with `dtype` on `stream`, and copied back the same way; the other
 * triangle of the host matrix is neither read nor written.  TRI_F32_MIXED sends the
 * triangle instead as the blocks of the recursive split (the 256 x 256 diagonal squares,
 * then each level's off-diagonal blocks), on a copy stream of the library's, in the order
 * the inverse first reads them: the inverse starts on the first blocks while the rest is
 * in flight; for a lower matrix the Newton-Schulz products run in four column groups and
 * each group's columns return as soon as they are final, beside the products of the
 * others (the result is the same either way).  Device memory for the matrix
 * and the workspace comes from the stream-ordered pool and is released before return.
 * Synchronises `stream` before returning (the host matrix holds the result on return).
 * Page-locked host memory gives full link bandwidth; pageable memory also works.
 * *bytes_moved (host pointer, may be NULL): bytes copied in both directions together.
 * Errors: as tri_inv_ex; TRI_ERR_NOMEM if the device allocation fails; TRI_ERR_CUDA for
 * a failed copy.  A zero pivot is reported by tri_get_info, as for tri_inv.
 * --------------------------------------------------------------------------------- */
TRI_API tri_status tri_inv_host(tri_uplo uplo, tri_diag diag, int64_t n, void *a, int64_t lda,
                                tri_dtype dtype, void *stream, int64_t *bytes_moved);

/* ---------------------------------------------------------------------------------
 * Strided batch of equal-order triangular inverses, in place: matrix b starts at
 * a + b * stride (elements, stride >= lda * n), batch <= 65535.  TRI_F32 / TRI_F64 run
 * every split level of all matrices in one launch; TRI_F32_MIXED (n > 256) runs each
 * product of the mixed path (level products, Newton-Schulz residual and update) as one
 * tensor-core launch over the tiles of a chunk of matrices whose BF16 planes fit in
 * 8 GiB (n <= 256: the TRI_F32 levels).  The workspace of the _ex form holds one chunk's
 * planes (tri_inv_strided_batched_workspace_size).  Singular pivots record the matrix
 * index.
 * --------------------------------------------------------------------------------- */
TRI_API tri_status tri_inv_strided_batched(tri_uplo uplo, tri_diag diag, int64_t n, void *a, int64_t lda,
                                           int64_t stride, int64_t batch, tri_dtype dtype, void *stream);
TRI_API size_t tri_inv_strided_batched_workspace_size(int64_t n, int64_t batch, tri_dtype dtype);
/* d_info: optional per-call status word (as tri_inv_ex; it records the matrix index). */
TRI_API tri_status tri_inv_strided_batched_ex(tri_uplo uplo, tri_diag diag, int64_t n, void *a, int64_t lda,
                                              int64_t stride, int64_t batch, tri_dtype dtype, void *workspace,
                                              size_t ws_bytes, int64_t *d_info, void *stream);

/* ---------------------------------------------------------------------------------
 * Adjoint of X = T^-1 (not in the paper; the plain definition from
 * d(T^-1) = -T^-1 dT T^-1): given X (the forward result, `uplo` triangle, unit diagonal
 * implied for TRI_UNIT) and the cotangent G = dL/dX (full n x n, only the `uplo`
 * triangle of G contributes), writes
 *     dT = -P(X^T G X^T)
 * into the `uplo` triangle of dt (the diagonal is set to 0 for TRI_UNIT); the other
 * triangle of dt is not written.  All matrices column-major, device memory; x, g and dt
 * must not overlap.  TRI_F32 / TRI_F64: CUDA-core products; TRI_F32_MIXED: split-BF16
 * tensor-core products (six terms with FP32 promotion, FP32-class accuracy) for n >= 256,
 * one launch per product for a chunk of the batch whose planes fit in 4 GiB.  Scratch: n*n elements per matrix (plus the BF16
 * planes of one chunk for TRI_F32_MIXED), from the stream-ordered allocator or `_ex`.
 * --------------------------------------------------------------------------------- */
TRI_API tri_status tri_inv_backward(tri_uplo uplo, tri_diag diag, int64_t n, const void *x, int64_t ldx,
                                    const void *g, int64_t ldg, void *dt, int64_t lddt, tri_dtype dtype,
                                    void *stream);
TRI_API tri_status tri_inv_backward_strided_batched(tri_uplo uplo, tri_diag diag, int64_t n, const void *x,
                                                    int64_t ldx, int64_t stride_x, const void *g, int64_t ldg,
                                                    int64_t stride_g, void *dt, int64_t lddt, int64_t stride_dt,
                                                    int64_t batch, tri_dtype dtype, void *stream);
TRI_API size_t tri_inv_backward_workspace_size(int64_t n, int64_t batch, tri_dtype dtype);
TRI_API tri_status tri_inv_backward_strided_batched_ex(tri_uplo uplo, tri_diag diag, int64_t n, const void *x,
                                                       int64_t ldx, int64_t stride_x, const void *g, int64_t ldg,
                                                       int64_t stride_g, void *dt, int64_t lddt, int64_t stride_dt,
                                                       int64_t batch, tri_dtype dtype, void *workspace,
                                                       size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------------
 * tri_inv_noalloc -- tri_inv for callers that cannot allocate device memory.
 * The paper has no counterpart; this is an integration entry point.
 *
 * Some callers cannot call cudaMalloc: an application whose own memory manager has
 * already reserved the device's memory (an allocation made inside the library would
 * fail or fragment that pool), or latency-critical code that must neither block in the
 * CUDA allocator nor handle an allocation failure halfway through its work.  This entry
 * point computes exactly what tri_inv computes for TRI_F32 and TRI_F64, but keeps its
 * scratch in a fixed device array of TRI_NOALLOC_SCRATCH_BYTES that the library holds on
 * every GPU that loads it, until the process exits.  It calls no cudaMalloc, cudaFree or
 * other allocating routine.  The caller still passes the matrix (same arguments and
 * layout as tri_inv).
 *   - Sizes whose scratch (tri_inv_workspace_size(n, dtype)) exceeds the array return
 *     TRI_ERR_ARG before anything is queued: TRI_F32 up to n = 4096, TRI_F64 up to
 *     n = 2048.  TRI_F32_MIXED returns TRI_ERR_UNSUPPORTED.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) and caches it; make that first call before any stream
 *     capture begins on that device.  The cached address does not survive
 *     cudaDeviceReset (the library's module is then loaded again elsewhere): do not
 *     call this entry point after resetting a device it was used on.
 *   - The limits above follow from tri_inv_workspace_size (leaves of 64 in FP32 and 16
 *     in FP64, one h x h block per pair of the widest level); a CPU test checks that
 *     both limits fit the array.
 *   - Every call on a device shares the one array, which keeps the previous call's
 *     contents (no call reads scratch it has not written itself).  Calls whose GPU work
 *     can overlap -- on different streams, or from host threads without ordering -- race
 *     on the array and give wrong results: order them on one stream.
 * --------------------------------------------------------------------------------- */
#define TRI_NOALLOC_SCRATCH_BYTES (16u << 20)
TRI_API tri_status tri_inv_noalloc(tri_uplo uplo, tri_diag diag, int64_t n, void *a,
                                   int64_t lda, tri_dtype dtype, void *stream);

/* ---------------------------------------------------------------------------------
 * tri_tc_gemm_bf16 -- the tensor-core product kernel of the mixed path on plain operands,
 * exposed for verification: C = sum_{t < nterms} A_t B_t, the dense "triangular times
 * full" products of the split (Section 4.1, Eq. "ptfm") before any triangular masking.
 *   A_t: m x k BF16, column-major, leading dimension lda (multiple of 8);
 *   B_t: k x n BF16, column-major, leading dimension ldb (multiple of 8);
 *   a_planes / b_planes: HOST arrays of nterms (1..3) device pointers, 16-byte aligned;
 *   C: m x n FP32, column-major, ldc >= m, overwritten.
 * Products are exact in FP32 (BF16 x BF16) and accumulated in FP32 in tensor memory.
 * Errors: TRI_ERR_ARG for bad sizes, alignment or pointers; TRI_ERR_NOMEM if the tile list
 * cannot be allocated (stream-ordered).
 * --------------------------------------------------------------------------------- */
TRI_API tri_status tri_tc_gemm_bf16(int64_t m, int64_t n, int64_t k, int nterms,
                                    const void *const *a_planes, int64_t lda,
                                    const void *const *b_planes, int64_t ldb, float *c,
                                    int64_t ldc, void *stream);

/* ---------------------------------------------------------------------------------
 * tri_mixed_schedule_stats -- host-only inspection of the TRI_F32_MIXED schedule for
 * order n on `ctas` persistent CTAs (no device call).  The mixed path runs the products
 * of every split level (block inverse of the proof of the main Theorem, Section 3:
 * W = B X_A, X21 = -X_C W) and of the Newton-Schulz step (R = I - T X, X += X R) as one
 * launch over a DAG of 128 x 256 output tiles, list-scheduled longest path first.
 * Writes into the host array stats[0..7]: number of tiles, dependency edges, modelled
 * makespan, longest dependency path and total work / ctas (the last three in pipeline
 * slots of one 128 x 256 x 64 product), 1.0 if the per-CTA lists replay to completion
 * (no circular wait), algorithmic flops, CTAs used.
 * Errors: TRI_ERR_ARG for n <= 256 (no tensor-core part), ctas < 1, nstats < 8 or a NULL
 * stats; TRI_ERR_UNSUPPORTED for n > 2^20.
 * --------------------------------------------------------------------------------- */
TRI_API tri_status tri_mixed_schedule_stats(int64_t n, int ctas, double *stats, int nstats);

/* Synchronises `stream`, then reports and clears the device-side status of the calling
 * thread's current device: TRI_ERR_SINGULAR with *first_bad_index set to the smallest
 * bad pivot index recorded since the last call, TRI_ERR_TIMEOUT if a bounded wait ran
 * out, otherwise TRI_OK with *first_bad_index = -1.  first_bad_index is a host pointer
 * and may be NULL. */
TRI_API tri_status tri_get_info(void *stream, int64_t *first_bad_index);

/* Growth limit of the FP64 fallback for ill-conditioned diagonal blocks on the
 * single-matrix paths (tri_inv, tri_inv_ex, the strided batches; FP32 and mixed), process-
 * wide, default 1e4 (the paper is silent on ill-conditioned leaves).  After a diagonal
 * block's FP32 inverse -- a plain-path leaf of 64 rows, or a mixed-path diagonal block of
 * 256 rows -- the growth max|X| max|T| (a lower bound of the block's condition number in
 * the max norm) is compared with tau; above it the block, still unchanged in memory, is
 * inverted again with FP64 arithmetic and that result, rounded to FP32, is kept.  On the
 * mixed path a matrix with such a block also skips the Newton-Schulz step: its residual,
 * computed to FP32 accuracy, would be dominated by rounding once max|X| max|T| is large.
 * tau <= 0 disables the check (results then bit-identical to a run without it on every
 * input); tri_growth_limit returns the current value.
 * Errors: TRI_ERR_ARG (NaN). */
TRI_API tri_status tri_set_growth_limit(double tau);
TRI_API double tri_growth_limit(void);

/* Recipe of TRI_F32_MIXED on the triangular paths (tri_inv[_ex], strided batches) and in
 * gen_inv, process-wide:
 *   TRI_RECIPE_NEWTON_SCHULZ (default)  three-term split-BF16 level products, then one
 *       Newton-Schulz step X <- X + X (I - T X) with a six-term residual and a one-term
 *       update: the result is better than the plain FP32 recursion's.
 *   TRI_RECIPE_DIRECT  the level products take all six split-BF16 terms with FP32
 *       promotion every 64 k (FP32-class products) and there is no Newton-Schulz step:
 *       about the plain FP32 recursion's accuracy, at about 60% of the tensor-core work.
 *       gen_inv follows the same choice (six-term products, no step against A).
 *       Not part of the paper's method or of the spec recipe; an alternative.
 * Errors: TRI_ERR_ARG (unknown recipe). */
#define TRI_RECIPE_NEWTON_SCHULZ 0
#define TRI_RECIPE_DIRECT 1
TRI_API tri_status tri_set_mixed_recipe(int recipe);
TRI_API int tri_mixed_recipe(void);

/* Products of the TRI_F32_MIXED triangular path (single matrices and strided batches,
 * Newton-Schulz recipe) that run on CTA pairs, process-wide: a bit mask of
 *   TRI_PAIR_LEVELS  the level products W = B X_A and X21 = -X_C W at split half-sizes
 *                    whose output tiles are 256 columns wide,
 *   TRI_PAIR_RES     the residual R = I - T X,
 *   TRI_PAIR_UPD     the update X += X R.
 * A pair is a cluster of two CTAs on two SMs that computes each 256 x 256 output tile with
 * one 256-row tensor-core product per k-step (tcgen05.mma.cta_group::2), each CTA staging
 * its own 128 rows of the left operand and half of the right one's tile: the same
 * products, summed in the same order (results are bit-identical to the single-CTA
 * schedule), with a third less operand traffic into each SM.  A schedule choice, not part
 * of the paper's method.  tri_cta_pairs returns the current mask.
 * Errors: TRI_ERR_ARG (bits outside the three). */
#define TRI_PAIR_LEVELS 1
#define TRI_PAIR_RES 2
#define TRI_PAIR_UPD 4
TRI_API tri_status tri_set_cta_pairs(int mask);
TRI_API int tri_cta_pairs(void);
/* CTA pairs of the product kernel that the current device runs at once (the number of
 * tile lists of a pair launch); 0 if the device cannot be queried. */
TRI_API int tri_cta_pair_capacity(void);

/* Measured CUDA-core peak of the current device for dtype TRI_F32 (FFMA) or TRI_F64
 * (DFMA), in TFLOP/s (2 flops per fused multiply-add): every thread of a full grid runs 8
 * independent chains of `iters` dependent FMAs, timed with CUDA events after a warm-up.
 * The denominator of the CUDA-core kernels' rooflines (not part of the method; a
 * measurement aid).  ms (may be NULL) receives the timed launch's duration.  Allocates
 * and synchronises; do not call during stream capture.
 * Errors: TRI_ERR_ARG (dtype, iters < 8, null tflops), TRI_ERR_NOMEM, TRI_ERR_CUDA. */
TRI_API tri_status tri_alu_peak(tri_dtype dtype, int iters, double *tflops, double *ms);

/* Usage of the library's scratch pool on the current device (bytes): in use now, and the
 * high-water mark since the pool was created or last reset (reset_high != 0 resets it
 * after reading).  NULL outputs are skipped.  Creates the pool if it does not exist yet. */
TRI_API tri_status tri_pool_stats(uint64_t *used, uint64_t *used_high, int reset_high);

/* ---------------------------------------------------------------------------------
 * Kernel tracing (host-side bookkeeping, off by default).  While enabled, every kernel
 * the library launches is bracketed by CUDA events on its own stream, and the
 * algorithmic flops / bytes of that launch are recorded.
 *   tri_trace_enable(1) clears earlier records and starts recording; (0) stops.
 *   tri_trace_report() synchronises on the recorded events and writes a JSON object
 *   {"<kernel>": {"launches": L, "ms": T, "flops": F, "bytes": B}, ...} into the host
 *   buffer `buf` of `cap` bytes (NUL-terminated, truncated if too small).  Returns the
 *   length the full report needs (excluding the NUL), or -1 on a CUDA error.
 * --------------------------------------------------------------------------------- */
TRI_API void tri_trace_enable(int on);
TRI_API int64_t tri_trace_report(char *buf, size_t cap);

/* Per-tile device timeline of the last TRI_F32_MIXED tensor-core launch made while tracing
 * was enabled.  Synchronises the device, then copies up to cap_words 64-bit words into the
 * host buffer `buf` (6 words per tile, in each CTA's processing order): [0] = CTA | op << 16
 * | k-blocks << 20 | (row tile) << 32 | (column tile) << 48 with op 0 = W = B X_A,
 * 1 = X21 = -X_C W, 2 = R = I - T X, 3 = X += X R; [1] producer starts waiting for the
 * tile's input regions; [2] first operand load issued; [3] MMA issuer starts the tile;
 * [4] last MMA issued; [5] epilogue done (GPU global timer, ns).  Returns the number of
 * tiles, 0 if no such launch was traced, -1 on a CUDA error.  buf may be NULL. */
TRI_API int64_t tri_trace_timeline(unsigned long long *buf, size_t cap_words);

#ifdef __cplusplus
}
#endif

#endif /* TRIINV_H */
