"""GPU tests of tri_inv_host (host-memory matrices): the result equals the device entry
point's bit for bit for TRI_F32 and TRI_F32_MIXED (same kernels on the same values; FP64
products add split-k partial sums atomically, so TRI_F64 agrees to a few units in the last
place), only the referenced triangle of
the host buffer changes (the other triangle holds NaN, padding rows and a tail guard hold
a canary), pinned and pageable host memory both work, and the reported byte count is the
triangle's panels in both directions (the mixed path sends the blocks of the recursive split
instead, in the order the inverse first reads them)."""
import numpy as np
import pytest

from paper_2307_07611_gb300 import inputs
from tests._gpu import check_untouched, from_colmajor_buffer, run_tri_inv, to_colmajor_buffer

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_07611_gb300 import lib as _lib
    _lib.load()
    return _lib


def panel_bytes(n, lower, es):
    total = 0
    for j0 in range(0, n, 256):
        cols = min(256, n - j0)
        rows = (n - j0) if lower else (j0 + cols)
        total += rows * cols * es
    return 2 * total


def block_bytes(n, es):
    """Host-to-device bytes of the mixed path, which sends the matrix in the blocks of the
    recursive split: the 256 x 256 diagonal squares, then every pair's B block (hc x h) of
    every level h = 256, 512, ... < n."""
    total = sum(min(256, n - d0) ** 2 for d0 in range(0, n, 256))
    h = 256
    while h < n:
        q = 0
        while 2 * q * h + h < n:
            c0 = 2 * q * h + h
            total += min(h, n - c0) * h
            q += 1
        h *= 2
    return total * es


@pytest.mark.parametrize("dt", ["f32", "f64", "mixed"])
@pytest.mark.parametrize("lower,unit", [(True, False), (False, False), (True, True)])
@pytest.mark.parametrize("n,pinned", [(300, True), (1000, False), (777, True), (2500, True)])
def test_host_matches_device(lib, dt, lower, unit, n, pinned):
    t = inputs.tri_lower(n, seed=n + 7, law="uniform")
    if not lower:
        t = t.T.copy()
    if dt != "f64":
        t = t.astype(np.float32).astype(np.float64)
    ld = n + 3
    np_dt = np.float64 if dt == "f64" else np.float32
    code = {"f64": lib.TRI_F64, "f32": lib.TRI_F32, "mixed": lib.TRI_F32_MIXED}[dt]
    host0 = to_colmajor_buffer(t, lower, ld, np_dt)
    buf = torch.from_numpy(host0.copy())
    if pinned:
        buf = buf.pin_memory()
    st, moved = lib.tri_inv_host(lib.TRI_LOWER if lower else lib.TRI_UPPER,
                                 lib.TRI_UNIT if unit else lib.TRI_NONUNIT, n, buf.data_ptr(), ld, code,
                                 int(torch.cuda.current_stream().cuda_stream))
    assert st == lib.TRI_OK and lib.tri_get_info()[0] == lib.TRI_OK
    out = buf.numpy()
    check_untouched(host0, out, n, ld, lower, unit)
    if dt == "mixed":   # blocks in, panels out
        assert moved == block_bytes(n, 4) + panel_bytes(n, lower, 4) // 2
    else:
        assert moved == panel_bytes(n, lower, np_dt().itemsize)
    x = from_colmajor_buffer(out, n, ld)
    x = np.tril(x) if lower else np.triu(x)
    if unit:
        np.fill_diagonal(x, 1.0)
    want, st2 = run_tri_inv(lib, torch, t, lower=lower, unit=unit, dtype="f64" if dt == "f64" else "f32",
                            mixed=(dt == "mixed"), ld_pad=3)
    assert st2 == lib.TRI_OK
    if dt == "f64":
        assert np.abs(x - want).max() <= 1e-14 * np.abs(want).max()
    else:
        assert np.array_equal(x, want)


def test_host_singular_and_arguments(lib):
    n = 400
    t = inputs.tri_lower(n, seed=5)
    t[123, 123] = 0.0
    host = torch.from_numpy(to_colmajor_buffer(t, True, n, np.float32)).pin_memory()
    st, _ = lib.tri_inv_host(lib.TRI_LOWER, lib.TRI_NONUNIT, n, host.data_ptr(), n, lib.TRI_F32, 0)
    assert st == lib.TRI_OK
    assert lib.tri_get_info() == (lib.TRI_ERR_SINGULAR, 123)
    assert lib.tri_inv_host(lib.TRI_LOWER, lib.TRI_NONUNIT, n, host.data_ptr(), n - 1, lib.TRI_F32, 0)[0] == \
        lib.TRI_ERR_ARG
    assert lib.tri_inv_host(lib.TRI_LOWER, lib.TRI_NONUNIT, 0, 0, 1, lib.TRI_F32, 0)[0] == lib.TRI_OK
