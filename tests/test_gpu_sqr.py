"""GPU parity of sqr (Algorithm SQR, Section 5.1: A = Q R with S = R^-1 formed alongside)
and of sqr_inv (A^-1 = S Q^T) against the FP64 oracle, which runs the printed modified
Gram-Schmidt algorithm one column at a time.  The GPU builds the same factors over
column blocks; the QR with a positive diagonal is unique, so the factors compare entry by
entry.

Tolerances.  On A = N(0,1)/sqrt(n) + 2I (kappa ~ 5) the forward error of a backward
stable QR is about kappa times the backward error, so each factor F in {Q, R, S} is held
to max |F - F_oracle| / max |F_oracle| <= 8 tol(n), tol as for the triangular path
(FP64 / FP32 40 sqrt(n) u; mixed 0.25 sqrt(n) 2^-16).  Independently of the oracle:
orthogonality max |Q^T Q - I| <= 100 u sqrt(n) (mixed: 2^-16 sqrt(n)), ||Q R - A||_F /
||A||_F, and the residual of S Q^T as an inverse.
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
    if dt == "mixed":
        return 0.25 * np.sqrt(n) * 2.0 ** -16
    return 40.0 * np.sqrt(max(n, 1)) * U[dt]


def orth_tol(n, dt):
    return (2.0 ** -16 if dt == "mixed" else 100.0 * U[dt]) * np.sqrt(max(n, 1))


def _dev(host):
    return torch.from_numpy(host.copy()).cuda()


def run_sqr(lib, a, dt, pads=(3, 2, 5), workspace=False):
    """sqr through the C ABI on column-major buffers with canary padding rows."""
    n = a.shape[0]
    np_dt = np.float64 if dt == "f64" else np.float32
    hosts = []
    for k, pad in enumerate(pads):
        h = np.full((n, n + pad), CANARY, dtype=np_dt)   # row c = column c
        if k == 0:
            h[:, :n] = a.T.astype(np_dt)
        hosts.append(h)
    da, dr, ds = (_dev(h) for h in hosts)
    s = int(torch.cuda.current_stream().cuda_stream)
    args = (n, da.data_ptr(), n + pads[0], dr.data_ptr(), n + pads[1], ds.data_ptr(), n + pads[2], code_of(lib, dt))
    if workspace:
        need = lib.sqr_workspace_size(n, code_of(lib, dt))
        ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        st = lib.sqr_ex(*args, (ws.data_ptr() + 255) // 256 * 256, need, s)
    else:
        st = lib.sqr(*args, s)
    torch.cuda.synchronize()
    outs = []
    for d, h in zip((da, dr, ds), hosts):
        o = d.cpu().numpy()
        assert np.array_equal(o[:, n:], h[:, n:]), "padding rows written"
        outs.append(o[:, :n].T.astype(np.float64))
    return outs, st


def residual(a, x):
    r = a @ x - np.eye(a.shape[0])
    return np.linalg.norm(r) / (np.linalg.norm(a) * np.linalg.norm(x))


@pytest.mark.parametrize("dt", ["f64", "f32", "mixed"])
@pytest.mark.parametrize("n", [1, 5, 31, 32, 33, 63, 64, 65, 100, 129, 300, 700, 1024])
def test_sqr_parity(lib, dt, n):
    a = inputs.general(n, seed=n + 3, dtype=np.float64 if dt == "f64" else np.float32).astype(np.float64)
    (q, r, s), st = run_sqr(lib, a, dt, workspace=(n == 300))
    assert st == lib.TRI_OK
    assert lib.tri_get_info()[0] == lib.TRI_OK
    assert not np.any(np.tril(r, -1)) and not np.any(np.tril(s, -1))
    want = oracle.sqr(a)
    for name, g, w in zip("QRS", (q, r, s), want):
        err = np.abs(g - w).max() / np.abs(w).max()
        assert err <= 8 * tol(n, dt), (name, err)
    assert np.abs(q.T @ q - np.eye(n)).max() <= orth_tol(n, dt)
    assert np.linalg.norm(q @ r - a) / np.linalg.norm(a) <= (1e-14 if dt == "f64" else 2e-6)
    assert residual(a, s @ q.T) <= (1e-13 if dt == "f64" else 5e-6)


@pytest.mark.parametrize("n", [2048, 2500])
def test_sqr_mixed_split_k_parity(lib, n):
    """Sizes at which the mixed path runs Q1^T A2 on the tensor cores as k slices (two
    slices at the top split, including the ragged 2500 = 1280 + 1220 columns)."""
    a = inputs.general(n, seed=n + 11, dtype=np.float32).astype(np.float64)
    (q, r, s), st = run_sqr(lib, a, "mixed")
    assert st == lib.TRI_OK and lib.tri_get_info()[0] == lib.TRI_OK
    want = oracle.sqr(a)
    for name, g, w in zip("QRS", (q, r, s), want):
        err = np.abs(g - w).max() / np.abs(w).max()
        assert err <= 8 * tol(n, "mixed"), (name, err)
    assert np.abs(q.T @ q - np.eye(n)).max() <= orth_tol(n, "mixed")
    assert residual(a, s @ q.T) <= 5e-6


@pytest.mark.parametrize("dt", ["f64", "f32", "mixed"])
def test_sqr_paper_example(lib, dt):
    from tests._golden import matrices
    g = matrices("skul_sqr_5x5.txt")
    (q, r, s), st = run_sqr(lib, g["A"], dt)
    assert st == lib.TRI_OK
    assert np.abs(q - g["Q"]).max() < 1.5e-4
    assert np.abs(r - g["R"]).max() < 2e-4
    assert np.abs(s - g["S_R"]).max() < 1.5e-4


@pytest.mark.parametrize("dt", ["f64", "f32", "mixed"])
@pytest.mark.parametrize("n", [64, 257, 1000])
def test_sqr_inv_parity(lib, dt, n):
    a = inputs.general(n, seed=n, dtype=np.float64 if dt == "f64" else np.float32).astype(np.float64)
    np_dt = np.float64 if dt == "f64" else np.float32
    dev = torch.from_numpy(np.ascontiguousarray(a.T).astype(np_dt)).cuda()
    st = lib.sqr_inv(n, dev.data_ptr(), n, code_of(lib, dt), int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == lib.TRI_OK and lib.tri_get_info()[0] == lib.TRI_OK
    x = dev.cpu().numpy().T.astype(np.float64)
    q, r, s = oracle.sqr(a)
    want = s @ q.T
    assert np.abs(x - want).max() / np.abs(want).max() <= 8 * tol(n, dt)
    assert residual(a, x) <= (1e-13 if dt == "f64" else 5e-6)


def test_sqr_inv_mixed_tensor_core_product(lib):
    """n = 2048: the final S Q^T (upper S, transposed Q) has enough output tiles to run on
    the tensor cores directly."""
    n = 2048
    a = inputs.general(n, seed=21, dtype=np.float32).astype(np.float64)
    dev = torch.from_numpy(np.ascontiguousarray(a.T).astype(np.float32)).cuda()
    st = lib.sqr_inv(n, dev.data_ptr(), n, lib.TRI_F32_MIXED, int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == lib.TRI_OK and lib.tri_get_info()[0] == lib.TRI_OK
    x = dev.cpu().numpy().T.astype(np.float64)
    q, r, s = oracle.sqr(a)
    want = s @ q.T
    assert np.abs(x - want).max() / np.abs(want).max() <= 8 * tol(n, "mixed")
    assert residual(a, x) <= 5e-6


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_sqr_inv_needs_no_pivoting(lib, dt):
    """A zero leading entry stops the unpivoted LU of gen_inv; the QR route inverts it."""
    n = 300
    a = inputs.general(n, seed=5, dtype=np.float64)
    a[0, 0] = 0.0
    np_dt = np.float64 if dt == "f64" else np.float32
    dev = torch.from_numpy(np.ascontiguousarray(a.T).astype(np_dt)).cuda()
    st = lib.sqr_inv(n, dev.data_ptr(), n, code_of(lib, dt), int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == lib.TRI_OK and lib.tri_get_info()[0] == lib.TRI_OK
    x = dev.cpu().numpy().T.astype(np.float64)
    assert residual(a, x) <= (1e-13 if dt == "f64" else 5e-6)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_sqr_zero_column_reported(lib, dt):
    n = 200
    a = inputs.general(n, seed=6, dtype=np.float64)
    a[:, 70] = 0.0
    run_sqr(lib, a, dt)
    st, bad = lib.tri_get_info()
    assert st == lib.TRI_ERR_SINGULAR and bad == 70


def test_sqr_torch_wrappers(lib):
    n = 190
    a = inputs.general(n, seed=8, dtype=np.float32)
    q, r, s = lib.sqr_factors(torch.from_numpy(a).cuda())
    want = oracle.sqr(a.astype(np.float64))
    for name, g, w in zip("QRS", (q, r, s), want):
        err = np.abs(g.double().cpu().numpy() - w).max() / np.abs(w).max()
        assert err <= 8 * tol(n, "f32"), (name, err)
    x = lib.qr_inv(torch.from_numpy(a).cuda()).double().cpu().numpy()
    assert residual(a.astype(np.float64), x) <= 5e-6
