"""GPU parity of skul (Algorithm SKUL, Section 5.1: Crout A = L U with K = L^-1 and
S = U^-1 formed alongside) against the FP64 oracle, which runs the algorithm as printed.

Each factor F in {L, U, S, K} is compared as max |F - F_oracle| / max |F_oracle| with the
tolerances of gen_inv (the same block recursion): 40 sqrt(n) u for FP64, FP32 and mixed
(six-term split-BF16 products with FP32 promotion, u = 2^-24).  Independently of the
oracle: ||L U - A||_F / ||A||_F and the normwise residual of S K as an inverse.
"""
import numpy as np
import pytest

import oracle
from paper_2307_07611_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = {"f32": 2.0 ** -24, "f64": 2.0 ** -53}
CANARY = -3.5e30


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_07611_gb300 import lib as _lib
    _lib.load()
    return _lib


def code_of(lib, dt):
    return {"f64": lib.TRI_F64, "f32": lib.TRI_F32, "mixed": lib.TRI_F32_MIXED}[dt]


def tol(n, dt):
    return 40.0 * np.sqrt(max(n, 1)) * U["f64" if dt == "f64" else "f32"]


def run_skul(lib, a, dt, pad_a=3, pad_sk=5, workspace=False):
    """skul through the C ABI on column-major buffers whose padding rows hold a canary.
    Returns (L, U, S, K) as dense FP64 matrices and the status."""
    n = a.shape[0]
    np_dt = np.float64 if dt == "f64" else np.float32
    ha = np.full((n, n + pad_a), CANARY, dtype=np_dt)       # row c = column c
    ha[:, :n] = a.T.astype(np_dt)
    hs = np.full((n, n + pad_sk), CANARY, dtype=np_dt)
    da = torch.from_numpy(ha.copy()).cuda()
    ds = torch.from_numpy(hs.copy()).cuda()
    s = int(torch.cuda.current_stream().cuda_stream)
    if workspace:
        need = lib.skul_workspace_size(n, code_of(lib, dt))
        ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        ptr = (ws.data_ptr() + 255) // 256 * 256
        st = lib.skul_ex(n, da.data_ptr(), n + pad_a, ds.data_ptr(), n + pad_sk, code_of(lib, dt), ptr, need, s)
    else:
        st = lib.skul(n, da.data_ptr(), n + pad_a, ds.data_ptr(), n + pad_sk, code_of(lib, dt), s)
    torch.cuda.synchronize()
    oa, osk = da.cpu().numpy(), ds.cpu().numpy()
    assert np.array_equal(oa[:, n:], ha[:, n:]), "padding rows of a written"
    assert np.array_equal(osk[:, n:], hs[:, n:]), "padding rows of sk written"
    lu = oa[:, :n].T.astype(np.float64)
    ks = osk[:, :n].T.astype(np.float64)
    eye = np.eye(n)
    return (np.tril(lu), np.triu(lu, 1) + eye, np.triu(ks, 1) + eye, np.tril(ks)), st


def residual(a, x):
    r = a @ x - np.eye(a.shape[0])
    return np.linalg.norm(r) / (np.linalg.norm(a) * np.linalg.norm(x))


@pytest.mark.parametrize("dt", ["f64", "f32", "mixed"])
@pytest.mark.parametrize("n", [1, 5, 100, 128, 129, 300, 700, 1024, 1500])
def test_skul_parity(lib, dt, n):
    a = inputs.general(n, seed=n + 7, dtype=np.float64 if dt == "f64" else np.float32).astype(np.float64)
    got, st = run_skul(lib, a, dt, workspace=(n == 300))
    assert st == lib.TRI_OK
    assert lib.tri_get_info()[0] == lib.TRI_OK
    want = oracle.skul(a)
    for name, g, w in zip("LUSK", got, want):
        err = np.abs(g - w).max() / np.abs(w).max()
        assert err <= tol(n, dt), (name, err)
    lo, up, s, k = got
    assert np.linalg.norm(lo @ up - a) / np.linalg.norm(a) <= (1e-14 if dt == "f64" else 2e-6)
    assert residual(a, s @ k) <= (1e-13 if dt == "f64" else 5e-6)


@pytest.mark.parametrize("dt", ["f64", "f32", "mixed"])
def test_skul_paper_example(lib, dt):
    from tests._golden import matrices
    g = matrices("skul_sqr_5x5.txt")
    got, st = run_skul(lib, g["A"], dt)
    assert st == lib.TRI_OK
    for name, f in zip("LUSK", got):
        assert np.abs(f - g[name]).max() < 1.5e-4, name


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_skul_zero_pivot_reported(lib, dt):
    n = 300
    a = inputs.general(n, seed=4, dtype=np.float64)
    a[0, 0] = 0.0
    run_skul(lib, a, dt)
    st, bad = lib.tri_get_info()
    assert st == lib.TRI_ERR_SINGULAR and bad == 0


def test_skul_torch_wrapper_rowmajor(lib):
    n = 257
    a = inputs.general(n, seed=9, dtype=np.float32)
    lo, up, s, k = lib.skul_factors(torch.from_numpy(a).cuda())
    want = oracle.skul(a.astype(np.float64))
    for name, g, w in zip("LUSK", (lo, up, s, k), want):
        err = np.abs(g.double().cpu().numpy() - w).max() / np.abs(w).max()
        assert err <= tol(n, "f32"), (name, err)
