"""Thin ctypes binding of libtriinv.so (include/triinv.h), plus torch-tensor helpers.

The functions named like the C entry points (``tri_inv``, ``tri_inv_ex``, ...) only
marshal arguments: every step of the computation runs in the library's CUDA kernels.
Loading fails loudly (``RuntimeError``) if the library has not been built; there is no
CPU fallback.

The torch helpers (``inv``, ...) map a row-major torch tensor onto the column-major
ABI: a C-contiguous lower-triangular n x n tensor is, column-major, an upper-triangular
matrix with lda = stride(0), so the helper flips ``uplo`` instead of copying.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(PKG, "_build", "libtriinv.so")

TRI_OK, TRI_ERR_ARG, TRI_ERR_SINGULAR, TRI_ERR_NOMEM, TRI_ERR_CUDA, TRI_ERR_TIMEOUT, \
    TRI_ERR_UNSUPPORTED = range(7)
TRI_LOWER, TRI_UPPER = 0, 1
TRI_NONUNIT, TRI_UNIT = 0, 1
TRI_F64, TRI_F32, TRI_F32_MIXED = 0, 1, 2
MIXED_AVAILABLE = True

_lock = threading.Lock()
_lib = None


class TriError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: {status_string(status)}" if what else status_string(status))


def _declare(lib):
    i64, i32, vp, sz = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
    sigs = {
        "tri_status_string": ([i32], ctypes.c_char_p),
        "tri_version": ([], ctypes.c_char_p),
        "tri_inv": ([i32, i32, i64, vp, i64, i32, vp], i32),
        "tri_inv_workspace_size": ([i64, i32], sz),
        "tri_inv_ex": ([i32, i32, i64, vp, i64, i32, vp, sz, vp, vp], i32),
        "tri_get_info": ([vp, ctypes.POINTER(i64)], i32),
        "tri_inv_noalloc": ([i32, i32, i64, vp, i64, i32, vp], i32),
        "tri_inv_host": ([i32, i32, i64, vp, i64, i32, vp, ctypes.POINTER(i64)], i32),
        "tri_inv_combrit": ([i32, i32, i64, vp, i64, i32, i32, vp], i32),
        "gen_inv": ([i64, vp, i64, i32, vp], i32),
        "tri_inv_strided_batched": ([i32, i32, i64, vp, i64, i64, i64, i32, vp], i32),
        "tri_inv_strided_batched_workspace_size": ([i64, i64, i32], sz),
        "tri_inv_strided_batched_ex": ([i32, i32, i64, vp, i64, i64, i64, i32, vp, sz, vp, vp], i32),
        "tri_inv_backward": ([i32, i32, i64, vp, i64, vp, i64, vp, i64, i32, vp], i32),
        "tri_inv_backward_strided_batched": ([i32, i32, i64, vp, i64, i64, vp, i64, i64, vp, i64, i64, i64,
                                              i32, vp], i32),
        "tri_inv_backward_workspace_size": ([i64, i64, i32], sz),
        "tri_inv_backward_strided_batched_ex": ([i32, i32, i64, vp, i64, i64, vp, i64, i64, vp, i64, i64,
                                                 i64, i32, vp, sz, vp], i32),
        "tri_batched_plan_create": ([i64, ctypes.POINTER(i64), ctypes.POINTER(vp), i32, i32, i32,
                                     ctypes.POINTER(vp)], i32),
        "tri_batched_exec": ([vp, vp], i32),
        "tri_batched_plan_destroy": ([vp], i32),
        "tri_batched_plan_threads": ([vp], i32),
        "tri_batched_plan_shape": ([vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)], i32),
        "tri_tune_cache_save": ([ctypes.c_char_p], i32),
        "tri_tune_cache_load": ([ctypes.c_char_p, ctypes.POINTER(i32)], i32),
        "tri_batched_plan_set_growth_limit": ([vp, ctypes.c_double], i32),
        "tri_inv_batched": ([i64, ctypes.POINTER(i64), ctypes.POINTER(vp), i32, i32, i32, vp], i32),
        "gen_inv_workspace_size": ([i64, i32], sz),
        "gen_inv_ex": ([i64, vp, i64, i32, vp, sz, vp, vp], i32),
        "brsi_inv": ([i64, vp, i64, i32, ctypes.POINTER(i64), i32, vp], i32),
        "brsi_inv_workspace_size": ([i64, i32, i32], sz),
        "brsi_inv_ex": ([i64, vp, i64, i32, ctypes.POINTER(i64), i32, vp, sz, vp, vp], i32),
        "skul": ([i64, vp, i64, vp, i64, i32, vp], i32),
        "skul_workspace_size": ([i64, i32], sz),
        "skul_ex": ([i64, vp, i64, vp, i64, i32, vp, sz, vp, vp], i32),
        "sqr": ([i64, vp, i64, vp, i64, vp, i64, i32, vp], i32),
        "sqr_workspace_size": ([i64, i32], sz),
        "sqr_ex": ([i64, vp, i64, vp, i64, vp, i64, i32, vp, sz, vp, vp], i32),
        "sqr_inv": ([i64, vp, i64, i32, vp], i32),
        "tri_tc_gemm_bf16": ([i64, i64, i64, i32, ctypes.POINTER(vp), i64, ctypes.POINTER(vp), i64,
                              vp, i64, vp], i32),
        "tri_mixed_schedule_stats": ([i64, i32, ctypes.POINTER(ctypes.c_double), i32], i32),
        "tri_batched_partition": ([i64, ctypes.POINTER(i64), i32, ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_double)], i32),
        "tri_set_mixed_recipe": ([i32], i32),
        "tri_mixed_recipe": ([], i32),
        "tri_set_cta_pairs": ([i32], i32),
        "tri_cta_pairs": ([], i32),
        "tri_cta_pair_capacity": ([], i32),
        "tri_set_growth_limit": ([ctypes.c_double], i32),
        "tri_growth_limit": ([], ctypes.c_double),
        "tri_alu_peak": ([i32, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], i32),
        "tri_pool_stats": ([ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), i32], i32),
        "tri_trace_enable": ([i32], None),
        "tri_trace_report": ([ctypes.c_char_p, sz], i64),
        "tri_trace_timeline": ([ctypes.POINTER(ctypes.c_uint64), sz], i64),
    }
    for name, (args, res) in sigs.items():
        if hasattr(lib, name):
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res


def load(path: str | None = None):
    """Load libtriinv.so (once).  Raises RuntimeError if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or SO_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"{p} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(p)
        _declare(lib)
        _lib = lib
        return lib


# ---- C entry points, same names and argument order ------------------------------------

def status_string(status: int) -> str:
    return load().tri_status_string(int(status)).decode()


def tri_version() -> str:
    return load().tri_version().decode()


def tri_inv(uplo, diag, n, ptr, ld, dtype, stream=0) -> int:
    return load().tri_inv(uplo, diag, n, ptr, ld, dtype, stream or None)


def tri_inv_workspace_size(n, dtype) -> int:
    return int(load().tri_inv_workspace_size(n, dtype))


def tri_inv_ex(uplo, diag, n, ptr, ld, dtype, workspace, ws_bytes, stream=0, d_info=0) -> int:
    """d_info: 0 (pivots to the device-wide word of tri_get_info) or the device address of
    an int64 that receives the first bad pivot index or -1 (the C argument before stream)."""
    return load().tri_inv_ex(uplo, diag, n, ptr, ld, dtype, workspace or None, ws_bytes, d_info or None,
                             stream or None)


def gen_inv(n, ptr, ld, dtype, stream=0) -> int:
    return load().gen_inv(n, ptr, ld, dtype, stream or None)


def gen_inv_workspace_size(n, dtype) -> int:
    return int(load().gen_inv_workspace_size(n, dtype))


def gen_inv_ex(n, ptr, ld, dtype, workspace, ws_bytes, stream=0, d_info=0) -> int:
    return load().gen_inv_ex(n, ptr, ld, dtype, workspace or None, ws_bytes, d_info or None, stream or None)


def _perm_arg(perm):
    if perm is None:
        return None
    return (ctypes.c_int64 * max(len(perm), 1))(*[int(p) for p in perm])


def brsi_inv(n, ptr, ld, gamma, dtype, perm=None, stream=0) -> int:
    """BRSI(gamma) general inverse in place; perm: the column permutation P_0 (host list)."""
    return load().brsi_inv(n, ptr, ld, int(gamma), _perm_arg(perm), dtype, stream or None)


def brsi_inv_workspace_size(n, gamma, dtype) -> int:
    return int(load().brsi_inv_workspace_size(n, int(gamma), dtype))


def brsi_inv_ex(n, ptr, ld, gamma, dtype, workspace, ws_bytes, perm=None, stream=0, d_info=0) -> int:
    return load().brsi_inv_ex(n, ptr, ld, int(gamma), _perm_arg(perm), dtype, workspace or None, ws_bytes,
                              d_info or None, stream or None)


def skul(n, a_ptr, lda, sk_ptr, ldsk, dtype, stream=0) -> int:
    return load().skul(n, a_ptr, lda, sk_ptr, ldsk, dtype, stream or None)


def skul_workspace_size(n, dtype) -> int:
    return int(load().skul_workspace_size(n, dtype))


def skul_ex(n, a_ptr, lda, sk_ptr, ldsk, dtype, workspace, ws_bytes, stream=0, d_info=0) -> int:
    return load().skul_ex(n, a_ptr, lda, sk_ptr, ldsk, dtype, workspace or None, ws_bytes, d_info or None,
                          stream or None)


def sqr(n, a_ptr, lda, r_ptr, ldr, s_ptr, lds, dtype, stream=0) -> int:
    return load().sqr(n, a_ptr, lda, r_ptr, ldr, s_ptr, lds, dtype, stream or None)


def sqr_workspace_size(n, dtype) -> int:
    return int(load().sqr_workspace_size(n, dtype))


def sqr_ex(n, a_ptr, lda, r_ptr, ldr, s_ptr, lds, dtype, workspace, ws_bytes, stream=0, d_info=0) -> int:
    return load().sqr_ex(n, a_ptr, lda, r_ptr, ldr, s_ptr, lds, dtype, workspace or None, ws_bytes,
                         d_info or None, stream or None)


def sqr_inv(n, a_ptr, lda, dtype, stream=0) -> int:
    return load().sqr_inv(n, a_ptr, lda, dtype, stream or None)


def _arrays(sizes, ptrs):
    n = len(sizes)
    return (ctypes.c_int64 * n)(*[int(x) for x in sizes]), (ctypes.c_void_p * n)(*[int(p) for p in ptrs])


def tri_batched_plan_create(count, sizes, ptrs, uplo, diag, dtype):
    """Returns (status, plan handle)."""
    sz, pt = _arrays(sizes, ptrs)
    h = ctypes.c_void_p()
    st = load().tri_batched_plan_create(count, sz, pt, uplo, diag, dtype, ctypes.byref(h))
    return st, h


def tri_batched_exec(plan, stream=0) -> int:
    return load().tri_batched_exec(plan, stream or None)


def tri_batched_plan_destroy(plan) -> int:
    return load().tri_batched_plan_destroy(plan)


def tri_batched_plan_threads(plan) -> int:
    return load().tri_batched_plan_threads(plan)


def tri_batched_plan_shape(plan, cls):
    """(blocks, threads, ctas) of size class cls (0: 161..256 rows, 1: 129..160, 2: 33..128, 3: <= 32)."""
    b, t, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    check(load().tri_batched_plan_shape(plan, int(cls), ctypes.byref(b), ctypes.byref(t), ctypes.byref(c)),
          "tri_batched_plan_shape")
    return b.value, t.value, c.value


def tri_tune_cache_save(path: str) -> int:
    return load().tri_tune_cache_save(path.encode())


def tri_tune_cache_load(path: str):
    n = ctypes.c_int(0)
    st = load().tri_tune_cache_load(path.encode(), ctypes.byref(n))
    return st, n.value


def tri_batched_plan_set_growth_limit(plan, tau) -> int:
    return load().tri_batched_plan_set_growth_limit(plan, float(tau))


def tri_inv_batched(count, sizes, ptrs, uplo, diag, dtype, stream=0) -> int:
    sz, pt = _arrays(sizes, ptrs)
    return load().tri_inv_batched(count, sz, pt, uplo, diag, dtype, stream or None)


def tri_batched_partition(sizes, world):
    """(owner, loads): the rank of every block (longest first to the least-loaded rank by
    m^3) and each rank's sum of m^3 -- the multi-GPU split of a batch (no collective)."""
    n = len(sizes)
    sz = (ctypes.c_int64 * max(n, 1))(*[int(k) for k in sizes])
    own = (ctypes.c_int32 * max(n, 1))()
    loads = (ctypes.c_double * max(int(world), 1))()
    check(load().tri_batched_partition(n, sz, int(world), own, loads), "tri_batched_partition")
    return [int(own[i]) for i in range(n)], [float(loads[r]) for r in range(int(world))]


def tri_inv_strided_batched(uplo, diag, n, ptr, ld, stride, batch, dtype, stream=0) -> int:
    return load().tri_inv_strided_batched(uplo, diag, n, ptr, ld, stride, batch, dtype, stream or None)


def tri_inv_strided_batched_workspace_size(n, batch, dtype) -> int:
    return int(load().tri_inv_strided_batched_workspace_size(n, batch, dtype))


def tri_inv_strided_batched_ex(uplo, diag, n, ptr, ld, stride, batch, dtype, workspace, ws_bytes, stream=0,
                               d_info=0) -> int:
    return load().tri_inv_strided_batched_ex(uplo, diag, n, ptr, ld, stride, batch, dtype, workspace or None,
                                             ws_bytes, d_info or None, stream or None)


def tri_inv_backward(uplo, diag, n, x, ldx, g, ldg, dt, lddt, dtype, stream=0) -> int:
    return load().tri_inv_backward(uplo, diag, n, x, ldx, g, ldg, dt, lddt, dtype, stream or None)


def tri_inv_backward_strided_batched(uplo, diag, n, x, ldx, sx, g, ldg, sg, dt, lddt, sd, batch, dtype,
                                     stream=0) -> int:
    return load().tri_inv_backward_strided_batched(uplo, diag, n, x, ldx, sx, g, ldg, sg, dt, lddt, sd, batch,
                                                   dtype, stream or None)


def tri_inv_backward_workspace_size(n, batch, dtype) -> int:
    return int(load().tri_inv_backward_workspace_size(n, batch, dtype))


def tri_inv_backward_strided_batched_ex(uplo, diag, n, x, ldx, sx, g, ldg, sg, dt, lddt, sd, batch, dtype,
                                        workspace, ws_bytes, stream=0) -> int:
    return load().tri_inv_backward_strided_batched_ex(uplo, diag, n, x, ldx, sx, g, ldg, sg, dt, lddt, sd, batch,
                                                      dtype, workspace or None, ws_bytes, stream or None)


TRI_NOALLOC_SCRATCH_BYTES = 16 << 20


def tri_inv_combrit(uplo, diag, n, ptr, ld, dtype, beta, stream=0) -> int:
    """tri_inv by COMBRIT with `beta` (2, 4, 8) diagonal blocks per level."""
    return load().tri_inv_combrit(uplo, diag, n, ptr, ld, dtype, beta, stream or None)


def tri_inv_host(uplo, diag, n, ptr, ld, dtype, stream=0):
    """tri_inv on a matrix in host memory (ptr: host address).  Returns (status,
    bytes copied in both directions); synchronises the stream."""
    moved = ctypes.c_int64(0)
    st = load().tri_inv_host(uplo, diag, n, ptr, ld, dtype, stream or None, ctypes.byref(moved))
    return st, int(moved.value)


def tri_inv_noalloc(uplo, diag, n, ptr, ld, dtype, stream=0) -> int:
    """tri_inv for callers that cannot allocate device memory: the scratch lives in a
    fixed 16 MiB device array held by the library (FP32 up to n = 4096, FP64 up to
    n = 2048).  Calls that overlap on the GPU share that array and race."""
    return load().tri_inv_noalloc(uplo, diag, n, ptr, ld, dtype, stream or None)


def tri_tc_gemm_bf16(m, n, k, a_ptrs, lda, b_ptrs, ldb, c, ldc, stream=0) -> int:
    """C = sum_t A_t B_t on the tensor cores (BF16 planes in, FP32 out); a_ptrs / b_ptrs
    are sequences of device pointers."""
    nt = len(a_ptrs)
    arr_a = (ctypes.c_void_p * nt)(*a_ptrs)
    arr_b = (ctypes.c_void_p * nt)(*b_ptrs)
    return load().tri_tc_gemm_bf16(m, n, k, nt, arr_a, lda, arr_b, ldb, c, ldc, stream or None)


def tri_mixed_schedule_stats(n, ctas) -> dict:
    """Host-only statistics of the mixed path's tensor-core schedule for order n on
    `ctas` CTAs (no GPU needed).  Raises TriError on bad arguments."""
    out = (ctypes.c_double * 8)()
    st = load().tri_mixed_schedule_stats(n, ctas, out, 8)
    if st != TRI_OK:
        raise TriError(st, "tri_mixed_schedule_stats")
    keys = ["tiles", "edges", "makespan", "critical_path", "work_per_cta", "replay_ok", "flops", "ctas"]
    return dict(zip(keys, list(out)))


def tri_get_info(stream=0):
    """Returns (status, first_bad_index)."""
    idx = ctypes.c_int64(-1)
    st = load().tri_get_info(stream or None, ctypes.byref(idx))
    return st, idx.value


TRI_RECIPE_NEWTON_SCHULZ = 0
TRI_RECIPE_DIRECT = 1


def tri_set_mixed_recipe(recipe: int) -> int:
    return load().tri_set_mixed_recipe(int(recipe))


def tri_mixed_recipe() -> int:
    return int(load().tri_mixed_recipe())


TRI_PAIR_LEVELS = 1
TRI_PAIR_RES = 2
TRI_PAIR_UPD = 4
TRI_PAIR_ALL = TRI_PAIR_LEVELS | TRI_PAIR_RES | TRI_PAIR_UPD


def tri_set_cta_pairs(mask: int) -> int:
    return load().tri_set_cta_pairs(int(mask))


def tri_cta_pairs() -> int:
    return int(load().tri_cta_pairs())


def tri_cta_pair_capacity() -> int:
    return int(load().tri_cta_pair_capacity())


def tri_set_growth_limit(tau: float) -> int:
    return load().tri_set_growth_limit(float(tau))


def tri_growth_limit() -> float:
    return float(load().tri_growth_limit())


def tri_alu_peak(dtype, iters: int = 1 << 16):
    """(TFLOP/s, ms): measured FFMA (TRI_F32) or DFMA (TRI_F64) peak of the current device."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    check(load().tri_alu_peak(int(dtype), int(iters), ctypes.byref(tf), ctypes.byref(ms)), "tri_alu_peak")
    return float(tf.value), float(ms.value)


def tri_pool_stats(reset_high: bool = False):
    """(used, used_high) bytes of the library's scratch pool on the current device."""
    used, high = ctypes.c_uint64(0), ctypes.c_uint64(0)
    check(load().tri_pool_stats(ctypes.byref(used), ctypes.byref(high), 1 if reset_high else 0), "tri_pool_stats")
    return int(used.value), int(high.value)


def tri_trace_enable(on: bool):
    load().tri_trace_enable(1 if on else 0)


def tri_trace_report() -> dict:
    import json
    lib = load()
    need = lib.tri_trace_report(None, 0)
    if need < 0:
        raise TriError(TRI_ERR_CUDA, "tri_trace_report")
    buf = ctypes.create_string_buffer(int(need) + 1)
    lib.tri_trace_report(buf, len(buf))
    return json.loads(buf.value.decode())


def tri_trace_timeline():
    """Per-tile timeline of the last traced mixed-path tensor-core launch as a list of
    dicts (cta, op, kblocks, row_tile, col_tile, wait, load, mma, mma_end, done in ns),
    or [] if none was traced."""
    lib = load()
    nt = lib.tri_trace_timeline(None, 0)
    if nt < 0:
        raise TriError(TRI_ERR_CUDA, "tri_trace_timeline")
    if nt == 0:
        return []
    buf = (ctypes.c_uint64 * (6 * nt))()
    if lib.tri_trace_timeline(buf, 6 * nt) < 0:
        raise TriError(TRI_ERR_CUDA, "tri_trace_timeline")
    out = []
    for t in range(nt):
        w = buf[6 * t: 6 * t + 6]
        out.append({"cta": w[0] & 0xFFFF, "op": (w[0] >> 16) & 0xF, "kblocks": (w[0] >> 20) & 0xFFF,
                    "row_tile": (w[0] >> 32) & 0xFFFF, "col_tile": (w[0] >> 48) & 0xFFFF,
                    "wait": w[1], "load": w[2], "mma": w[3], "mma_end": w[4], "done": w[5]})
    return out


def check(status: int, what: str = ""):
    if status != TRI_OK:
        raise TriError(status, what)


# ---- torch helpers ----------------------------------------------------------------

def _stream_handle(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dtype_code(t, mixed: bool) -> int:
    import torch
    if t.dtype == torch.float64:
        if mixed:
            raise ValueError("mixed precision is defined for float32 storage only")
        return TRI_F64
    if t.dtype == torch.float32:
        return TRI_F32_MIXED if mixed else TRI_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _rowmajor_square(t):
    if t.dim() != 2 or t.shape[0] != t.shape[1]:
        raise ValueError("expected a square matrix")
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if t.stride(1) != 1:
        raise ValueError("expected unit stride along the last dimension")


def inv_(t, lower: bool = True, unit: bool = False, mixed: bool = False, stream=None):
    """In place: the ``lower`` (or upper) triangle of the row-major CUDA tensor ``t``
    (n x n, or a batch b x n x n with contiguous matrices) becomes that of t^-1; the other
    triangle is not touched."""
    if t.dim() == 3:
        if not t.is_cuda or not t.is_contiguous() or t.shape[1] != t.shape[2]:
            raise ValueError("expected a contiguous CUDA batch of square matrices")
        b, n = t.shape[0], t.shape[1]
        st = tri_inv_strided_batched(TRI_UPPER if lower else TRI_LOWER, TRI_UNIT if unit else TRI_NONUNIT, n,
                                     t.data_ptr(), max(1, n), n * n, b, _dtype_code(t, mixed),
                                     _stream_handle(stream))
        check(st, "tri_inv_strided_batched")
        return t
    _rowmajor_square(t)
    n = t.shape[0]
    # Row-major lower == column-major upper with lda = stride(0).
    uplo = TRI_UPPER if lower else TRI_LOWER
    st = tri_inv(uplo, TRI_UNIT if unit else TRI_NONUNIT, n, t.data_ptr(), max(1, t.stride(0)),
                 _dtype_code(t, mixed), _stream_handle(stream))
    check(st, "tri_inv")
    return t


def inv_grad(x, g, lower: bool = True, unit: bool = False, mixed: bool = False, stream=None):
    """dL/dT = -P(X^T G X^T) for X = T^-1 (row-major CUDA tensors, n x n or b x n x n).
    The result has zeros outside T's free entries."""
    import torch
    x = x.contiguous()
    g = g.contiguous()
    out = torch.zeros_like(x)
    n = x.shape[-1]
    b = x.shape[0] if x.dim() == 3 else 1
    # Row-major buffers are the column-major transposes: flip the triangle.
    uplo = TRI_UPPER if lower else TRI_LOWER
    st = tri_inv_backward_strided_batched(uplo, TRI_UNIT if unit else TRI_NONUNIT, n, x.data_ptr(), n, n * n,
                                          g.data_ptr(), n, n * n, out.data_ptr(), n, n * n, b,
                                          _dtype_code(x, mixed), _stream_handle(stream))
    check(st, "tri_inv_backward")
    return out


def _tri_inv_function():
    import torch

    class TriInv(torch.autograd.Function):
        """X = T^-1 for a triangular T (n x n or b x n x n CUDA tensor); the backward pass
        is the library's adjoint kernel."""

        @staticmethod
        def forward(ctx, t, lower=True, unit=False, mixed=False):
            x = inv(t, lower=lower, unit=unit, mixed=mixed)
            ctx.save_for_backward(x)
            ctx.flags = (lower, unit, mixed)
            return x

        @staticmethod
        def backward(ctx, g):
            (x,) = ctx.saved_tensors
            lower, unit, mixed = ctx.flags
            return inv_grad(x, g, lower=lower, unit=unit, mixed=mixed), None, None, None

    return TriInv


_TRI_INV_FN = None


def tri_inv_autograd(t, lower: bool = True, unit: bool = False, mixed: bool = False):
    """Differentiable triangular inverse (torch.autograd.Function over the C ABI)."""
    global _TRI_INV_FN
    if _TRI_INV_FN is None:
        _TRI_INV_FN = _tri_inv_function()
    return _TRI_INV_FN.apply(t, lower, unit, mixed)


def general_inv(a, mixed: bool = False, stream=None):
    """Out of place A^-1 of a square CUDA tensor (float32 or float64) by the unpivoted
    block LU of gen_inv.  Row-major A is column-major A^T, and (A^T)^-1 = (A^-1)^T, so the
    column-major call on the row-major buffer returns A^-1 in row-major order."""
    _rowmajor_square(a)
    out = a.contiguous().clone()
    n = out.shape[0]
    st = gen_inv(n, out.data_ptr(), max(1, out.stride(0)), _dtype_code(out, mixed), _stream_handle(stream))
    check(st, "gen_inv")
    return out


def skul_factors(a, mixed: bool = False, stream=None):
    """SKUL (Algorithm SKUL, Section 5.1) of a square CUDA tensor: returns (L, U, S, K)
    with A = L U (L lower, U unit upper, Crout), S = U^-1, K = L^-1 and A^-1 = S K.  The
    C call works on the column-major layout of A, i.e. the row-major buffer of A^T."""
    import torch
    _rowmajor_square(a)
    buf = a.t().contiguous()          # column-major A
    sk = torch.empty_like(buf)
    n = buf.shape[0]
    ld = max(1, n)
    st = skul(n, buf.data_ptr(), ld, sk.data_ptr(), ld, _dtype_code(buf, mixed), _stream_handle(stream))
    check(st, "skul")
    lu, ks = buf.t(), sk.t()          # back to the logical matrices
    eye = torch.eye(n, dtype=a.dtype, device=a.device)
    return torch.tril(lu), torch.triu(lu, 1) + eye, torch.triu(ks, 1) + eye, torch.tril(ks)


def sqr_factors(a, mixed: bool = False, stream=None):
    """SQR (Algorithm SQR, Section 5.1) of a square CUDA tensor: returns (Q, R, S) with
    A = Q R (R upper, positive diagonal) and S = R^-1, so A^-1 = S Q^T."""
    import torch
    _rowmajor_square(a)
    q = a.t().contiguous()            # column-major A
    r = torch.empty_like(q)
    s = torch.empty_like(q)
    n = q.shape[0]
    ld = max(1, n)
    st = sqr(n, q.data_ptr(), ld, r.data_ptr(), ld, s.data_ptr(), ld, _dtype_code(q, mixed),
             _stream_handle(stream))
    check(st, "sqr")
    return q.t(), r.t(), s.t()


def qr_inv(a, mixed: bool = False, stream=None):
    """Out of place A^-1 = S Q^T through SQR (no pivoting needed).  Row-major A is the
    column-major A^T, whose inverse is (A^-1)^T: the row-major result is A^-1."""
    _rowmajor_square(a)
    out = a.contiguous().clone()
    n = out.shape[0]
    st = sqr_inv(n, out.data_ptr(), max(1, out.stride(0)), _dtype_code(out, mixed), _stream_handle(stream))
    check(st, "sqr_inv")
    return out


def inv(t, lower: bool = True, unit: bool = False, mixed: bool = False, stream=None):
    """Out of place: returns the triangular inverse as a clean tril/triu tensor (the
    diagonal is 1 when ``unit``)."""
    import torch
    out = t.contiguous().clone()
    inv_(out, lower=lower, unit=unit, mixed=mixed, stream=stream)
    out = torch.tril(out) if lower else torch.triu(out)
    if unit:
        out.diagonal(dim1=-2, dim2=-1).fill_(1)
    return out
