"""GPU parity of tri_inv / tri_inv_ex (plain FP32 and FP64 paths) against the FP64
oracle, through the C ABI.

Tolerance (floating point): every entry of X comes out of at most log2(n/64)+1 levels
of dot products of length <= n.  With random-sign rounding errors the forward error of
an entry is about kappa * sqrt(n) * u * max|X|; the value laws used here have
kappa(T) <= 5.  The tests allow 8x headroom over that estimate:
    max|X - X_oracle| <= 40 * sqrt(n) * u * max|X_oracle|,   u = 2^-24 or 2^-53,
and, independently of the oracle, the normwise residual
||T X - I||_F / (||T||_F ||X||_F) <= 5e-6 (FP32) or 1e-13 (FP64).
Integer families whose inverses are small integers must match bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2307_07611_gb300 import inputs
from tests._gpu import normwise_residual, rel_max_err, run_tri_inv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = {"f32": 2.0 ** -24, "f64": 2.0 ** -53}
RESID = {"f32": 5e-6, "f64": 1e-13}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_07611_gb300 import lib as _lib
    _lib.load()
    return _lib


def tol(n, dt):
    return 40.0 * np.sqrt(max(n, 1)) * U[dt]


def logical(n, seed, law, lower):
    t = inputs.tri_lower(n, seed=seed, law=law)
    return t if lower else t.T.copy()


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("n", [1, 2, 3, 17, 63, 64, 65, 127, 128, 129, 200, 511, 1000])
def test_lower_nonunit_parity(lib, dt, n):
    t = logical(n, n, "normal", True)
    if dt == "f32":
        t = t.astype(np.float32).astype(np.float64)
    x, st = run_tri_inv(lib, torch, t, lower=True, dtype=dt)
    assert st == lib.TRI_OK
    assert lib.tri_get_info()[0] == lib.TRI_OK
    want = oracle.tri_inv(t)
    assert rel_max_err(x, want) <= tol(n, dt)
    assert normwise_residual(t, x) <= RESID[dt]
    if dt == "f32":
        d = np.diag(t).astype(np.float32)
        assert np.array_equal(np.diag(x).astype(np.float32), np.float32(1) / d)


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("unit", [False, True])
@pytest.mark.parametrize("n", [70, 300, 1500])
def test_uplo_diag_parity(lib, dt, lower, unit, n):
    t = logical(n, 7 * n + lower + 2 * unit, "uniform", lower)
    if dt == "f32":
        t = t.astype(np.float32).astype(np.float64)
    x, st = run_tri_inv(lib, torch, t, lower=lower, unit=unit, dtype=dt, ld_pad=5,
                        workspace=(n == 300))
    assert st == lib.TRI_OK
    want = oracle.tri_inv(t, lower=lower, unit=unit)
    assert rel_max_err(x, want) <= tol(n, dt)
    tu = t.copy()
    if unit:
        np.fill_diagonal(tu, 1.0)
    assert normwise_residual(tu, x) <= RESID[dt]


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("lower", [True, False])
def test_integer_families_bit_exact(lib, dt, lower):
    cases = [inputs.ones_unit_lower(300),
             inputs.bidiagonal_unit_lower(1000, seed=1)[0],
             inputs.level_nilpotent_unit_lower(777, 64, seed=2)[0],
             inputs.level_nilpotent_unit_lower(1024, 256, seed=3)[0]]
    t1, _ = inputs.level_nilpotent_unit_lower(520, 64, seed=4, lo=-1, hi=1)
    t2, _ = inputs.level_nilpotent_unit_lower(520, 128, seed=5, lo=-1, hi=1)
    cases.append(t1 @ t2)
    for t in cases:
        if not lower:
            t = t.T.copy()
        want = oracle.tri_inv(t, lower=lower, unit=True)
        assert np.array_equal(want, np.round(want))
        for unit in (True, False):
            x, st = run_tri_inv(lib, torch, t, lower=lower, unit=unit, dtype=dt)
            assert st == lib.TRI_OK
            assert np.array_equal(x, want), (t.shape, unit)


def test_paper_worked_example_exact(lib):
    from tests._golden import matrices
    g = matrices("theorem_example_4x4.txt")
    for dt in ("f32", "f64"):
        x, _ = run_tri_inv(lib, torch, g["T"], lower=False, unit=True, dtype=dt)
        assert np.array_equal(x, g["Tinv"])
        x, _ = run_tri_inv(lib, torch, g["T"].T.copy(), lower=True, unit=False, dtype=dt)
        assert np.array_equal(x, g["Tinv"].T)


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_singular_pivot_reported(lib, dt):
    n = 333
    t = inputs.tri_lower(n, seed=3)
    t[200, 200] = 0.0
    t[250, 250] = np.inf
    _, st = run_tri_inv(lib, torch, t, lower=True, dtype=dt)
    assert st == lib.TRI_OK  # queued fine
    st, bad = lib.tri_get_info()
    assert st == lib.TRI_ERR_SINGULAR and bad == 200
    assert lib.tri_get_info() == (lib.TRI_OK, -1)  # cleared
    # unit diagonal: the stored zero is never read
    _, st = run_tri_inv(lib, torch, t, lower=True, unit=True, dtype=dt)
    assert lib.tri_get_info() == (lib.TRI_OK, -1)


def test_config_single_f64_n512(lib):
    # single lower FP64, n = 512, seed 0, uniform law, leaf 64 (3 split levels)
    t = inputs.tri_lower(512, seed=0, law="uniform")
    x, st = run_tri_inv(lib, torch, t, lower=True, dtype="f64", ld_pad=0)
    want = oracle.tri_inv(t)
    assert rel_max_err(x, want) <= tol(512, "f64")
    assert normwise_residual(t, x) <= 1e-13


def test_deterministic_and_stream(lib):
    n = 900
    t = inputs.tri_lower(n, seed=8, law="normal").astype(np.float32).astype(np.float64)
    s = torch.cuda.Stream()
    x1, _ = run_tri_inv(lib, torch, t, dtype="f32", stream=s)
    x2, _ = run_tri_inv(lib, torch, t, dtype="f32")
    assert np.array_equal(x1, x2)


def test_torch_helper_rowmajor(lib):
    n = 257
    t = inputs.tri_lower(n, seed=5, law="normal")
    for lower in (True, False):
        tt = t if lower else t.T.copy()
        dev = torch.tensor(tt, dtype=torch.float64, device="cuda")
        x = lib.inv(dev, lower=lower).cpu().numpy()
        want = oracle.tri_inv(tt, lower=lower)
        assert rel_max_err(x, want) <= tol(n, "f64")


@pytest.mark.slow
@pytest.mark.parametrize("lower", [True, False])
def test_full_size_f32_n8192_sampled(lib, lower):
    """The FP32 n = 8192 workload (normal law): every element against the FP64 oracle
    (all 8192 columns) and the normwise residual of the whole result."""
    n = 8192
    t = inputs.tri_lower(n, seed=0, law="normal", dtype=np.float32).astype(np.float64)
    tt = t if lower else t.T.copy()
    x, st = run_tri_inv(lib, torch, tt, lower=lower, dtype="f32", ld_pad=0)
    assert st == lib.TRI_OK
    want = oracle.tri_inv(tt, lower=lower)
    assert rel_max_err(x, want) <= tol(n, "f32")
    assert normwise_residual(tt, x) <= 5e-6
