"""GPU parity of gen_inv (A^-1 = U^-1 L^-1 from an unpivoted block LU) against the FP64
oracle (Crout LU in SKUL's order, two triangular inverses, their product).

Tolerances (max |X - X_oracle| / max |X_oracle|), on A = N(0,1)/sqrt(n) + 2I (kappa ~ 5,
growth ~ 1): 40 sqrt(n) u for FP64, FP32 and mixed alike (u = 2^-24 for the FP32 storage
of mixed), as for the triangular path: the mixed path's three-term products are followed
by a Newton-Schulz step against A with a six-term residual (n >= 512; smaller orders run
every product on CUDA cores).  Independently of the oracle: normwise residual
||AX - I||_F / (||A||_F ||X||_F) <= 1e-13 (FP64) and <= 5e-6 (FP32, mixed), and the mixed
residual at most twice the plain FP32 one on the same input ("equal residual").
"""
import numpy as np
import pytest

import oracle
from paper_2307_07611_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = {"f32": 2.0 ** -24, "f64": 2.0 ** -53}


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


def run_gen(lib, a, dt, ld_pad=3, workspace=False):
    """gen_inv through the C ABI on a column-major buffer with padding rows holding a canary."""
    n = a.shape[0]
    ld = n + ld_pad
    np_dt = np.float64 if dt == "f64" else np.float32
    host = np.full((n, ld), -3.5e30, dtype=np_dt)           # row c = column c
    host[:, :n] = a.T.astype(np_dt)
    dev = torch.from_numpy(host.copy()).cuda()
    s = int(torch.cuda.current_stream().cuda_stream)
    if workspace:
        need = lib.gen_inv_workspace_size(n, code_of(lib, dt))
        ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        ptr = (ws.data_ptr() + 255) // 256 * 256
        st = lib.gen_inv_ex(n, dev.data_ptr(), ld, code_of(lib, dt), ptr, need, s)
    else:
        st = lib.gen_inv(n, dev.data_ptr(), ld, code_of(lib, dt), s)
    torch.cuda.synchronize()
    out = dev.cpu().numpy()
    assert np.array_equal(out[:, n:], host[:, n:]), "padding rows written"
    return out[:, :n].T.astype(np.float64), st


def residual(a, x):
    r = a @ x - np.eye(a.shape[0])
    return np.linalg.norm(r) / (np.linalg.norm(a) * np.linalg.norm(x))


@pytest.mark.parametrize("dt", ["f64", "f32", "mixed"])
@pytest.mark.parametrize("n", [1, 5, 100, 128, 129, 300, 700, 1024, 2000])
def test_gen_inv_parity(lib, dt, n):
    a = inputs.general(n, seed=n, dtype=np.float64 if dt == "f64" else np.float32).astype(np.float64)
    x, st = run_gen(lib, a, dt, workspace=(n == 300))
    assert st == lib.TRI_OK
    assert lib.tri_get_info()[0] == lib.TRI_OK
    want = oracle.gen_inv(a)
    err = np.abs(x - want).max() / np.abs(want).max()
    assert err <= tol(n, dt), err
    assert residual(a, x) <= (1e-13 if dt == "f64" else 5e-6)


@pytest.mark.parametrize("n", [512, 700, 1024, 2000, 3000])
def test_gen_inv_mixed_equal_residual(lib, n):
    """Mixed residual at most twice the plain FP32 residual on the same input."""
    a = inputs.general(n, seed=100 + n, dtype=np.float32).astype(np.float64)
    xm, st = run_gen(lib, a, "mixed")
    assert st == lib.TRI_OK
    xp, st = run_gen(lib, a, "f32")
    assert st == lib.TRI_OK
    rm, rp = residual(a, xm), residual(a, xp)
    assert rm <= 2.0 * rp, (rm, rp)


@pytest.mark.parametrize("dt", ["f64", "f32", "mixed"])
def test_gen_inv_paper_example(lib, dt):
    from tests._golden import matrices
    g = matrices("skul_sqr_5x5.txt")
    x, st = run_gen(lib, g["A"], dt)
    assert st == lib.TRI_OK
    assert np.abs(x - g["S"] @ g["K"]).max() < 2e-4        # printed inverse factors
    assert np.abs(x - oracle.gen_inv(g["A"])).max() <= tol(5, dt) * np.abs(x).max()


@pytest.mark.parametrize("dt", ["f64", "f32", "mixed"])
def test_gen_inv_zero_pivot_reported(lib, dt):
    n = 400
    a = inputs.general(n, seed=2, dtype=np.float64)
    a[0, 0] = 0.0
    run_gen(lib, a, dt)
    st, bad = lib.tri_get_info()
    assert st == lib.TRI_ERR_SINGULAR and bad == 0


def test_gen_inv_argument_errors(lib):
    assert lib.gen_inv(-1, 0, 1, lib.TRI_F32) == lib.TRI_ERR_ARG
    assert lib.gen_inv(0, 0, 1, lib.TRI_F32) == lib.TRI_OK
    assert lib.gen_inv(10, 0, 10, lib.TRI_F32) == lib.TRI_ERR_ARG
    assert lib.gen_inv(10, 4096, 9, lib.TRI_F32) == lib.TRI_ERR_ARG


_N16K = {}


def _oracle_cols_16384(cols):
    """64 FP64 oracle columns of A^-1 for the n = 16384 workload (seed 0), computed once
    per test session (one LU of A on the host's cores)."""
    if "x" not in _N16K:
        a = inputs.general(16384, seed=0, dtype=np.float32)
        _N16K["a"] = a
        _N16K["x"] = oracle.inverse_columns(a.astype(np.float64), cols)
    return _N16K["a"], _N16K["x"]


@pytest.mark.slow
@pytest.mark.parametrize("dt", ["mixed", "f32"])
def test_gen_inv_full_size_n16384_sampled(lib, dt):
    """The general FP32 n = 16384 workload: 64 columns of X element-wise against the FP64
    oracle (FP32-class tolerance), and per column the normwise residual of A X - I."""
    n = 16384
    cols = sorted(set([0, 1, 4095, 8191, 8192, 12000, 16383] +
                      list(np.random.default_rng(7).choice(n, 57, replace=False))))[:64]
    a, want = _oracle_cols_16384(cols)
    dev = torch.from_numpy(np.ascontiguousarray(a.T)).cuda()
    st = lib.gen_inv(n, dev.data_ptr(), n, code_of(lib, dt), int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == lib.TRI_OK and lib.tri_get_info()[0] == lib.TRI_OK
    x = dev[cols, :].double().cpu().numpy().T        # columns of X
    del dev
    err = np.abs(x - want).max() / np.abs(want).max()
    assert err <= tol(n, dt), err
    a64 = a.astype(np.float64)
    r = a64 @ x
    r[cols, range(len(cols))] -= 1.0
    anorm = np.linalg.norm(a64)
    for c in range(len(cols)):
        assert np.linalg.norm(r[:, c]) / (anorm * np.linalg.norm(x[:, c])) <= 5e-6
