"""The direct recipe of the mixed triangular path (tri_set_mixed_recipe(TRI_RECIPE_DIRECT)):
the level products take all six split-BF16 terms with FP32 promotion and there is no
Newton-Schulz step.  Parity against the FP64 oracle at the FP32 tolerance of the plain
path (40 sqrt(n) 2^-24, max |X - X_oracle| / max |X_oracle|), uplo / unit handling, and the
equal-residual criterion (normwise residual at most twice the plain FP32 one, and
<= 5e-6) up to the n = 8192 workload.  The recipe is process-wide; every test restores the
default."""
import numpy as np
import pytest

import oracle
from paper_2307_07611_gb300 import inputs
from tests._gpu import normwise_residual, rel_max_err, run_tri_inv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_07611_gb300 import lib as _lib
    _lib.load()
    assert _lib.tri_set_mixed_recipe(_lib.TRI_RECIPE_DIRECT) == _lib.TRI_OK
    yield _lib
    _lib.tri_set_mixed_recipe(_lib.TRI_RECIPE_NEWTON_SCHULZ)


def tol(n):
    return 40.0 * np.sqrt(n) * 2.0 ** -24


@pytest.mark.parametrize("n", [257, 700, 1000, 2048, 3000])
@pytest.mark.parametrize("lower,unit", [(True, False), (False, False), (True, True)])
def test_direct_parity(lib, n, lower, unit):
    t = inputs.tri_lower(n, seed=n, law="normal", dtype=np.float32).astype(np.float64)
    if not lower:
        t = t.T.copy()
    x, st = run_tri_inv(lib, torch, t, lower=lower, unit=unit, dtype="f32", mixed=True)
    assert st == lib.TRI_OK and lib.tri_get_info()[0] == lib.TRI_OK
    want = oracle.tri_inv(t, lower=lower, unit=unit)
    assert rel_max_err(x, want) <= tol(n)


@pytest.mark.parametrize("n", [1000, 3000, 8192])
def test_direct_equal_residual(lib, n):
    t = inputs.tri_lower(n, seed=0, law="normal", dtype=np.float32).astype(np.float64)
    x, st = run_tri_inv(lib, torch, t, lower=True, dtype="f32", mixed=True, ld_pad=0)
    assert st == lib.TRI_OK
    xp, _ = run_tri_inv(lib, torch, t, lower=True, dtype="f32", ld_pad=0)
    r_direct, r_plain = normwise_residual(t, x), normwise_residual(t, xp)
    assert r_direct <= 5e-6 and r_direct <= 2.0 * r_plain, (r_direct, r_plain)
    if n == 8192:
        assert rel_max_err(x, oracle.tri_inv(t)) <= tol(n)


def test_recipe_setting(lib):
    assert lib.tri_set_mixed_recipe(7) == lib.TRI_ERR_ARG
    assert lib.tri_mixed_recipe() == lib.TRI_RECIPE_DIRECT


@pytest.mark.parametrize("n", [600, 2000])
def test_direct_gen_inv(lib, n):
    """gen_inv under the direct recipe: six-term products, no Newton-Schulz step; FP32
    tolerance against the oracle and equal residual against plain FP32."""
    a = inputs.general(n, seed=n, dtype=np.float32).astype(np.float64)

    def run(code):
        dev = torch.from_numpy(np.ascontiguousarray(a.T).astype(np.float32)).cuda()
        assert lib.gen_inv(n, dev.data_ptr(), n, code, int(torch.cuda.current_stream().cuda_stream)) == lib.TRI_OK
        torch.cuda.synchronize()
        return dev.cpu().numpy().T.astype(np.float64)

    xd, xp = run(lib.TRI_F32_MIXED), run(lib.TRI_F32)
    want = oracle.gen_inv(a)
    assert np.abs(xd - want).max() / np.abs(want).max() <= tol(n)
    res = lambda x: np.linalg.norm(a @ x - np.eye(n)) / (np.linalg.norm(a) * np.linalg.norm(x))
    assert res(xd) <= 2.0 * res(xp), (res(xd), res(xp))
