"""GPU parity of tri_inv_combrit (Algorithm COMBRIT, Section 4.1, with beta = 2, 4, 8, 16
diagonal blocks per level) against the FP64 oracle.  Same tolerances as the plain path
(40 sqrt(n) u max|X| against the oracle, normwise residual 5e-6 / 1e-13); integer families
whose inverses are small integers are exact; only the referenced triangle is written
(checked by run_tri_inv: NaN in the other triangle, canaries in the padding)."""
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


@pytest.mark.parametrize("beta", [2, 4, 8, 16])
@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("n", [1, 17, 64, 200, 1000, 1537, 2048])
def test_combrit_lower_parity(lib, beta, dt, n):
    t = inputs.tri_lower(n, seed=n + beta, law="uniform")
    if dt == "f32":
        t = t.astype(np.float32).astype(np.float64)
    x, st = run_tri_inv(lib, torch, t, lower=True, dtype=dt, beta=beta)
    assert st == lib.TRI_OK and lib.tri_get_info()[0] == lib.TRI_OK
    want = oracle.tri_inv(t)
    assert rel_max_err(x, want) <= 40 * np.sqrt(n) * U[dt]
    assert normwise_residual(t, x) <= RESID[dt]


@pytest.mark.parametrize("beta", [4, 8, 16])
@pytest.mark.parametrize("lower,unit", [(False, False), (True, True), (False, True)])
def test_combrit_uplo_diag(lib, beta, lower, unit):
    n = 777
    t = inputs.tri_lower(n, seed=beta + 10 * lower + 100 * unit, law="normal")
    if not lower:
        t = t.T.copy()
    x, st = run_tri_inv(lib, torch, t, lower=lower, unit=unit, dtype="f64", beta=beta)
    assert st == lib.TRI_OK
    want = oracle.tri_inv(t, lower=lower, unit=unit)
    assert rel_max_err(x, want) <= 40 * np.sqrt(n) * U["f64"]


@pytest.mark.parametrize("beta", [2, 4, 8, 16])
def test_combrit_integer_families_bit_exact(lib, beta):
    for t in (inputs.ones_unit_lower(600), inputs.bidiagonal_unit_lower(1100, seed=1)[0],
              inputs.level_nilpotent_unit_lower(1024, 256, seed=2)[0]):
        want = oracle.tri_inv(t, lower=True, unit=True)
        for dt in ("f32", "f64"):
            x, st = run_tri_inv(lib, torch, t, lower=True, unit=True, dtype=dt, beta=beta)
            assert st == lib.TRI_OK
            assert np.array_equal(x, want)


def test_combrit_singular_reported(lib):
    n = 900
    t = inputs.tri_lower(n, seed=3)
    t[433, 433] = 0.0
    run_tri_inv(lib, torch, t, lower=True, dtype="f32", beta=4)
    assert lib.tri_get_info() == (lib.TRI_ERR_SINGULAR, 433)
