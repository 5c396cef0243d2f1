"""GPU tests of the adjoint dT = -P(X^T G X^T) (tri_inv_backward, strided batches and the
torch.autograd.Function), against FP64 central finite differences and the FP64 oracle
gradient, plus the strided-batched forward.

Tolerances: FP64 finite differences agree to 1e-7 normwise (h = 1e-6 max(1, |t_ij|));
against the oracle gradient, max |dT - dT_oracle| / max |dT_oracle| <= c sqrt(n) u with
c = 80 for FP32 / FP64 / mixed (two products, each bounded as in the forward tests; the
mixed products take six split-BF16 terms with FP32 promotion, u = 2^-24).
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

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


def code(lib, dt):
    return {"f64": lib.TRI_F64, "f32": lib.TRI_F32, "mixed": lib.TRI_F32_MIXED}[dt]


def gtol(n, dt):
    return 80.0 * np.sqrt(n) * U["f64" if dt == "f64" else "f32"]


def colmajor(m, dtype):
    """Device buffer holding the logical matrix m column-major (row-major of m^T)."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(m).T)).to(dtype).cuda()


def backward_c(lib, x, g, lower, unit, dt):
    n = x.shape[0]
    tdt = torch.float64 if dt == "f64" else torch.float32
    xd, gd = colmajor(x, tdt), colmajor(g, tdt)
    out = torch.full((n, n + 2), float("nan"), dtype=tdt, device="cuda")   # ld = n + 2, canary
    st = lib.tri_inv_backward(lib.TRI_LOWER if lower else lib.TRI_UPPER,
                              lib.TRI_UNIT if unit else lib.TRI_NONUNIT, n, xd.data_ptr(), n, gd.data_ptr(), n,
                              out.data_ptr(), n + 2, code(lib, dt), int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == lib.TRI_OK
    o = out.double().cpu().numpy()
    assert np.isnan(o[:, n:]).all(), "padding written"
    d = o[:, :n].T
    mask = np.tril(np.ones((n, n), bool)) if lower else np.triu(np.ones((n, n), bool))
    if unit:
        assert np.all(np.diag(d) == 0.0)
    assert np.isnan(d[~mask]).all(), "other triangle written"
    return np.where(mask, d, 0.0)


def loss(t, w, lower, unit):
    x = sla.solve_triangular(t, np.eye(t.shape[0]), lower=lower, unit_diagonal=unit)
    return float(np.sum(w * x))


@pytest.mark.parametrize("lower,unit", [(True, False), (False, False), (True, True)])
def test_adjoint_fp64_central_differences(lib, lower, unit):
    n = 32
    t = inputs.tri_lower(n, seed=21, law="uniform")
    if not lower:
        t = t.T.copy()
    w = np.random.default_rng(22).standard_normal((n, n))
    x = sla.solve_triangular(t, np.eye(n), lower=lower, unit_diagonal=unit)
    got = backward_c(lib, x, w, lower, unit, "f64")
    fd = np.zeros((n, n))
    for i, j in itertools.product(range(n), range(n)):
        free = (i >= j) if lower else (i <= j)
        if unit and i == j:
            free = False
        if not free:
            continue
        h = 1e-6 * max(1.0, abs(t[i, j]))
        tp, tm = t.copy(), t.copy()
        tp[i, j] += h
        tm[i, j] -= h
        fd[i, j] = (loss(tp, w, lower, unit) - loss(tm, w, lower, unit)) / (2 * h)
    assert np.linalg.norm(got - fd) <= 1e-7 * np.linalg.norm(fd)


@pytest.mark.parametrize("dt", ["f64", "f32", "mixed"])
@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("n", [70, 300, 1024])
def test_adjoint_matches_oracle_gradient(lib, dt, lower, n):
    t = inputs.tri_lower(n, seed=n + 1, law="uniform")
    if not lower:
        t = t.T.copy()
    x = oracle.tri_inv(t, lower=lower)
    if dt != "f64":
        x = x.astype(np.float32).astype(np.float64)
    g = np.random.default_rng(n).standard_normal((n, n))
    if dt != "f64":
        g = g.astype(np.float32).astype(np.float64)
    want = oracle.tri_grad(x, g, lower=lower)
    got = backward_c(lib, x, g, lower, False, dt)
    assert np.abs(got - want).max() <= gtol(n, dt) * np.abs(want).max()


def test_adjoint_only_referenced_triangle_of_g(lib):
    n = 300
    t = inputs.tri_lower(n, seed=3)
    x = oracle.tri_inv(t).astype(np.float32).astype(np.float64)
    g = np.random.default_rng(4).standard_normal((n, n)).astype(np.float32).astype(np.float64)
    g2 = g.copy()
    g2[np.triu_indices(n, 1)] = np.nan
    a = backward_c(lib, x, g, True, False, "f32")
    b = backward_c(lib, x, g2, True, False, "f32")
    assert np.array_equal(a, b)


@pytest.mark.parametrize("dt", ["f32", "f64", "mixed"])
def test_strided_batched_forward(lib, dt):
    b, n = 6, 300
    tdt = torch.float64 if dt == "f64" else torch.float32
    ts = np.stack([inputs.tri_lower(n, seed=50 + i, law="uniform") for i in range(b)])
    if dt != "f64":
        ts = ts.astype(np.float32).astype(np.float64)
    dev = torch.from_numpy(np.ascontiguousarray(np.transpose(ts, (0, 2, 1)))).to(tdt).cuda()
    st = lib.tri_inv_strided_batched(lib.TRI_LOWER, lib.TRI_NONUNIT, n, dev.data_ptr(), n, n * n, b,
                                     code(lib, dt), int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == lib.TRI_OK and lib.tri_get_info()[0] == lib.TRI_OK
    xs = np.transpose(dev.double().cpu().numpy(), (0, 2, 1))
    u = U["f64" if dt == "f64" else "f32"]
    for i in range(b):
        want = oracle.tri_inv(ts[i])
        assert np.abs(np.tril(xs[i]) - want).max() <= 40 * np.sqrt(n) * u * np.abs(want).max()


@pytest.mark.parametrize("mixed", [False, True])
def test_autograd_function_batch(lib, mixed):
    """loss = sum(W * T^-1) over a batch of 4 lower FP32 n = 1024 matrices (uniform law),
    W ~ N(0,1): T.grad against the FP64 oracle gradient."""
    from paper_2307_07611_gb300 import lib as L
    b, n = 4, 1024
    ts, ws = inputs.adjoint_batch(b, n, seed=0)
    t = torch.from_numpy(ts).cuda().requires_grad_(True)
    w = torch.from_numpy(ws).cuda()
    x = L.tri_inv_autograd(t, lower=True, mixed=mixed)
    (w * x).sum().backward()
    grad = t.grad.double().cpu().numpy()
    dt = "mixed" if mixed else "f32"
    for i in range(b):
        xo = oracle.tri_inv(ts[i].astype(np.float64))
        want = oracle.tri_grad(xo, ws[i].astype(np.float64))
        assert np.abs(grad[i] - want).max() <= 2 * gtol(n, dt) * np.abs(want).max()
        assert not np.any(np.triu(grad[i], 1))
