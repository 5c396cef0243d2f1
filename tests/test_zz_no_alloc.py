"""tri_inv_noalloc: the entry point for callers that cannot allocate device memory
(an application whose memory manager already owns the GPU's memory, or code that must
not block in or handle failures of the CUDA allocator mid-work).  Its scratch is a fixed
16 MiB device array inside the library instead of an allocation from the library's
stream-ordered pool; the test also checks that the pool does not grow during the call.

The test calls it through the C ABI and compares it with tri_inv on the same inputs,
twice in a row (the second call finds the first call's leftovers in the shared array),
with the tolerance of the other parity tests.  This file is collected last on purpose,
and it must pass on its own in a fresh process as well as after the other tests."""
import numpy as np
import pytest

from paper_2307_07611_gb300 import inputs
from tests._gpu import to_colmajor_buffer, from_colmajor_buffer, check_untouched

torch = pytest.importorskip("torch")

U = {"f32": 2.0 ** -24, "f64": 2.0 ** -53}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_07611_gb300 import lib as _lib
    _lib.load()
    return _lib


def _run(lib, fn, t, lower, dt, ld, unit=False):
    n = t.shape[0]
    np_dt = np.float64 if dt == "f64" else np.float32
    code = lib.TRI_F64 if dt == "f64" else lib.TRI_F32
    host = to_colmajor_buffer(t, lower, ld, np_dt)
    dev = torch.from_numpy(host.copy()).cuda()
    s = torch.cuda.current_stream()
    st = fn(lib.TRI_LOWER if lower else lib.TRI_UPPER, lib.TRI_UNIT if unit else lib.TRI_NONUNIT, n,
            dev.data_ptr(), ld, code, int(s.cuda_stream))
    s.synchronize()
    out = dev.cpu().numpy()
    check_untouched(host, out, n, ld, lower, unit)
    x = from_colmajor_buffer(out, n, ld)
    x = np.tril(x) if lower else np.triu(x)
    if unit:
        np.fill_diagonal(x, 1.0)
    return x, st


@pytest.mark.gpu
@pytest.mark.parametrize("dt,n,lower,unit", [("f32", 4096, True, False), ("f32", 1500, False, False),
                                             ("f64", 2048, True, False), ("f64", 333, False, False),
                                             ("f32", 1000, True, True)])
def test_noalloc_matches_tri_inv_two_calls(lib, dt, n, lower, unit):
    tol = 40.0 * np.sqrt(n) * U[dt]
    for call, seed in enumerate((11, 12)):
        t = inputs.tri_lower(n, seed=seed + n, law="normal")
        if not lower:
            t = t.T.copy()
        if dt == "f32":
            t = t.astype(np.float32).astype(np.float64)
        # The library's own scratch pool must not grow during the no-allocation call:
        # its high-water mark is reset first (nothing of the library is in use between
        # calls) and read again after the call has completed.
        used0, _ = lib.tri_pool_stats(reset_high=True)
        x_na, st_na = _run(lib, lib.tri_inv_noalloc, t, lower, dt, n + 3, unit)
        used1, high1 = lib.tri_pool_stats()
        assert used0 == 0 and used1 == 0 and high1 == 0, (used0, used1, high1)
        x_ref, st_ref = _run(lib, lib.tri_inv, t, lower, dt, n + 3, unit)
        assert st_na == lib.TRI_OK and st_ref == lib.TRI_OK, (call, st_na, st_ref)
        assert lib.tri_get_info()[0] == lib.TRI_OK
        err = np.abs(x_na - x_ref).max() / np.abs(x_ref).max()
        assert err <= tol, (call, err)


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    s = int(torch.cuda.current_stream().cuda_stream)
    buf = torch.zeros(16, device="cuda")
    p = buf.data_ptr()
    assert lib.tri_inv_noalloc(0, 0, 4097, p, 4097, lib.TRI_F32, s) == lib.TRI_ERR_ARG
    assert lib.tri_inv_noalloc(0, 0, 2049, p, 2049, lib.TRI_F64, s) == lib.TRI_ERR_ARG
    assert lib.tri_inv_noalloc(0, 0, 100, p, 100, lib.TRI_F32_MIXED, s) == lib.TRI_ERR_UNSUPPORTED
    assert lib.tri_inv_noalloc(0, 0, 0, p, 1, lib.TRI_F32, s) == lib.TRI_OK
