"""GPU parity of brsi_inv (BRSI with gamma blocks, Section 5.2) against the FP64 oracle
that runs the paper's steps (oracle.brsi: A_{l+1} = I + M_l^-1 N_l, A P_0 = M_0 ... L).

Tolerances as for gen_inv (max |X - X_oracle| / max |X_oracle|): 40 sqrt(n) u for FP64,
FP32 and mixed (u = 2^-24 for FP32 storage; the mixed products are followed by a
Newton-Schulz step against A for n >= 512).  Inputs: A = N(0,1)/sqrt(n) + 2I (the general
law), whose diagonal blocks are non-singular for every split; a matrix with singular
diagonal blocks is inverted once the column permutation P_0 of Step 1 swaps its block
columns, and without it the zero pivot is reported."""
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


def run_brsi(lib, a, gamma, dt, perm=None, ld_pad=3, workspace=False):
    n = a.shape[0]
    ld = n + ld_pad
    np_dt = np.float64 if dt == "f64" else np.float32
    host = np.full((n, ld), -3.5e30, dtype=np_dt)          # row c = column c
    host[:, :n] = a.T.astype(np_dt)
    dev = torch.from_numpy(host.copy()).cuda()
    s = int(torch.cuda.current_stream().cuda_stream)
    if workspace:
        need = lib.brsi_inv_workspace_size(n, gamma, code_of(lib, dt))
        ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        ptr = (ws.data_ptr() + 255) // 256 * 256
        st = lib.brsi_inv_ex(n, dev.data_ptr(), ld, gamma, code_of(lib, dt), ptr, need, perm=perm, stream=s)
    else:
        st = lib.brsi_inv(n, dev.data_ptr(), ld, gamma, code_of(lib, dt), perm=perm, stream=s)
    torch.cuda.synchronize()
    out = dev.cpu().numpy()
    assert np.array_equal(out[:, n:], host[:, n:]), "padding rows written"
    return out[:, :n].T.astype(np.float64), st


def residual(a, x):
    r = a @ x - np.eye(a.shape[0])
    return np.linalg.norm(r) / (np.linalg.norm(a) * np.linalg.norm(x))


_ORACLE = {}


def _case(n, gamma):
    """FP32-representable input (shared by all three precisions) and its oracle inverse,
    computed once; the oracle inverts blocks of at most 32 rows directly."""
    if (n, gamma) not in _ORACLE:
        a = inputs.general(n, seed=n + gamma, dtype=np.float32).astype(np.float64)
        _ORACLE[(n, gamma)] = (a, oracle.brsi(a, gamma, leaf=32))
    return _ORACLE[(n, gamma)]


@pytest.mark.parametrize("dt", ["f64", "f32", "mixed"])
@pytest.mark.parametrize("n,gamma", [(1, 2), (7, 3), (100, 2), (129, 3), (300, 4), (513, 5), (700, 8),
                                     (1024, 4), (1500, 16)])
def test_brsi_parity(lib, dt, n, gamma):
    a, want = _case(n, gamma)
    x, st = run_brsi(lib, a, gamma, dt, workspace=(n == 300))
    assert st == lib.TRI_OK
    assert lib.tri_get_info()[0] == lib.TRI_OK
    err = np.abs(x - want).max() / np.abs(want).max()
    assert err <= tol(n, dt), err
    assert residual(a, x) <= (1e-13 if dt == "f64" else 5e-6)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_brsi_column_permutation(lib, dt):
    """Singular diagonal blocks: zero without P_0 (reported), inverted with it."""
    n = 600
    rng = np.random.default_rng(5)
    a = np.zeros((n, n))
    h = n // 2
    a[:h, h:] = np.eye(h) * 2.0 + rng.standard_normal((h, h)) / np.sqrt(n)
    a[h:, :h] = np.eye(h) * 2.0 + rng.standard_normal((h, h)) / np.sqrt(n)
    a = a.astype(np.float32).astype(np.float64)
    perm = list(range(h, n)) + list(range(h))
    x, st = run_brsi(lib, a, 2, dt, perm=perm)
    assert st == lib.TRI_OK and lib.tri_get_info()[0] == lib.TRI_OK
    want = oracle.brsi(a, 2, perm=perm)
    assert np.abs(x - want).max() / np.abs(want).max() <= tol(n, dt)
    _, st = run_brsi(lib, a, 2, dt)
    assert st == lib.TRI_OK
    info, bad = lib.tri_get_info()
    assert info == lib.TRI_ERR_SINGULAR and bad == 0


def test_brsi_paper_example(lib):
    from tests._golden import matrices
    g = matrices("skul_sqr_5x5.txt")
    for gamma in (2, 3, 5):
        x, st = run_brsi(lib, g["A"], gamma, "f64")
        assert st == lib.TRI_OK
        assert np.abs(x - g["S"] @ g["K"]).max() < 2e-4        # printed inverse factors


def test_brsi_argument_errors(lib):
    A = lib.TRI_ERR_ARG
    buf = torch.zeros(16, device="cuda")
    p = buf.data_ptr()
    assert lib.brsi_inv(4, p, 4, 1, lib.TRI_F32) == A                     # gamma < 2
    assert lib.brsi_inv(4, p, 4, 17, lib.TRI_F32) == A                    # gamma > 16
    assert lib.brsi_inv(4, p, 4, 2, lib.TRI_F32, perm=[0, 1, 1, 3]) == A  # not a permutation
    assert lib.brsi_inv(4, p, 4, 2, lib.TRI_F32, perm=[0, 1, 2, 4]) == A
    assert lib.brsi_inv(4, p, 3, 2, lib.TRI_F32) == A                     # lda < n
    assert lib.brsi_inv(0, p, 1, 2, lib.TRI_F32) == lib.TRI_OK
