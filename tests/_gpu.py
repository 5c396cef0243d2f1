"""GPU test helpers: run a C-ABI entry point on a column-major device buffer whose
unreferenced triangle is poisoned with NaN and whose padding rows (lda > n) and tail
guard hold a canary, then check that only the referenced triangle changed."""
import numpy as np

CANARY = -7.25e30


def to_colmajor_buffer(t, lower, ld, dtype, poison=np.nan, guard=64):
    """Flat column-major host buffer of ld*n + guard elements holding the `lower`
    (or upper) triangle of the logical matrix t, poison in the other triangle and the
    canary in the padding rows and the guard tail."""
    n = t.shape[0]
    buf = np.full(ld * n + guard, CANARY, dtype=dtype)
    mat = np.array(t, dtype=np.float64, copy=True)
    mask = np.tril(np.ones((n, n), bool)) if lower else np.triu(np.ones((n, n), bool))
    mat[~mask] = poison
    view = buf[: ld * n].reshape(n, ld)  # row c of view = column c of the matrix
    view[:, :n] = mat.T.astype(dtype)
    return buf


def from_colmajor_buffer(buf, n, ld):
    view = buf[: ld * n].reshape(n, ld)
    return np.array(view[:, :n].T, dtype=np.float64)


def check_untouched(before, after, n, ld, lower, unit=False):
    """The other triangle, the padding rows, the guard tail (and a unit diagonal) must
    be bit-identical."""
    b = before.view(np.uint64 if before.dtype == np.float64 else np.uint32)
    a = after.view(b.dtype)
    bm = b[: ld * n].reshape(n, ld)
    am = a[: ld * n].reshape(n, ld)
    assert np.array_equal(bm[:, n:], am[:, n:]), "padding rows written"
    assert np.array_equal(b[ld * n:], a[ld * n:]), "guard tail written"
    cols = np.arange(n)[:, None]
    rows = np.arange(n)[None, :]
    other = (rows < cols) if lower else (rows > cols)   # [col, row] layout of the view
    if unit:
        other = other | (rows == cols)
    assert np.array_equal(bm[:, :n][other], am[:, :n][other]), "unreferenced triangle written"


def run_tri_inv(lib, torch, t, lower=True, unit=False, dtype="f32", ld_pad=3, stream=None,
                mixed=False, workspace=False, beta=None):
    """Invert the logical matrix t through the C ABI; returns (X, status) where X holds
    the referenced triangle (other triangle zero, unit diagonal set to 1)."""
    n = t.shape[0]
    ld = max(1, n + ld_pad)
    np_dt = np.float64 if dtype == "f64" else np.float32
    code = lib.TRI_F64 if dtype == "f64" else (lib.TRI_F32_MIXED if mixed else lib.TRI_F32)
    host = to_colmajor_buffer(t, lower, ld, np_dt)
    dev = torch.from_numpy(host.copy()).cuda()
    s = stream or torch.cuda.current_stream()
    h = int(s.cuda_stream)
    if beta is not None:
        st = lib.tri_inv_combrit(lib.TRI_LOWER if lower else lib.TRI_UPPER,
                                 lib.TRI_UNIT if unit else lib.TRI_NONUNIT, n, dev.data_ptr(), ld, code, beta, h)
    elif workspace:
        need = lib.tri_inv_workspace_size(n, code)
        ws = torch.empty(max(need, 1) + 256, dtype=torch.uint8, device="cuda")
        ptr = (ws.data_ptr() + 255) // 256 * 256
        st = lib.tri_inv_ex(lib.TRI_LOWER if lower else lib.TRI_UPPER,
                            lib.TRI_UNIT if unit else lib.TRI_NONUNIT, n, dev.data_ptr(), ld,
                            code, ptr, need, h)
    else:
        st = lib.tri_inv(lib.TRI_LOWER if lower else lib.TRI_UPPER,
                         lib.TRI_UNIT if unit else lib.TRI_NONUNIT, n, dev.data_ptr(), ld, code, h)
    s.synchronize()
    out = dev.cpu().numpy()
    check_untouched(host, out, n, ld, lower, unit)
    x = from_colmajor_buffer(out, n, ld)
    x = np.tril(x) if lower else np.triu(x)
    if unit:
        np.fill_diagonal(x, 1.0)
    return x, st


def rel_max_err(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


def normwise_residual(t, x):
    n = t.shape[0]
    r = t @ x - np.eye(n)
    return float(np.linalg.norm(r) / (np.linalg.norm(t) * np.linalg.norm(x)))
