"""The FP64 fallback for ill-conditioned diagonal blocks on the single-matrix paths
(tri_set_growth_limit; the paper is silent on ill-conditioned leaves).

An n = 2048 lower matrix of the FP32 law (normal, sqrt(n) scaling) carries two
ill-conditioned diagonal blocks: a unit block with N(0,1) * s strict lower part (growth
max|X| max|T| 3.4e7 for 64 rows, s = 1; 1.2e6 for 96 rows, s = 0.6) and the subdiagonal -2 block (x_ij = 2^(i-j), exact in FP32).  On
the plain path they sit in 64-row leaves, on the mixed path inside 256-row diagonal
blocks.  The diagonal blocks of T^-1 are the inverses of T's diagonal blocks (block lower
triangular), so the oracle inverts each block on its own.  With the default limit every
entry of those blocks is within 2^-23 (relative) of the FP64 oracle; with the limit
disabled the FP32 recurrence is measurably worse; well-conditioned inputs give
bit-identical results with the limit on and off."""
import numpy as np
import pytest

import oracle
from paper_2307_07611_gb300 import inputs
from tests._gpu import run_tri_inv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_07611_gb300 import lib as _lib
    _lib.load()
    yield _lib
    _lib.tri_set_growth_limit(1.0e4)


def _ill(n, scale, seed):
    g = np.random.default_rng(seed)
    return np.eye(n) + np.tril(g.standard_normal((n, n)), -1) * scale


def _embedded(n, blocks, seed=0):
    """The FP32-law matrix with the given (row0, block) pairs placed on its diagonal (their
    rows to the left of the block zeroed, so each stays a diagonal block)."""
    t = inputs.tri_lower(n, seed=seed, law="normal", dtype=np.float32).astype(np.float64)
    for r0, b in blocks:
        m = b.shape[0]
        t[r0:r0 + m, :r0 + m] = 0.0
        t[r0:r0 + m, r0:r0 + m] = b
    return t.astype(np.float32).astype(np.float64)


def _entry_rel_err(x, want):
    m = want != 0
    return float(np.max(np.abs(x[m] - want[m]) / np.abs(want[m])))


def _run(lib, t, mixed, tau):
    assert lib.tri_set_growth_limit(tau) == lib.TRI_OK
    x, st = run_tri_inv(lib, torch, t, lower=True, dtype="f32", mixed=mixed, ld_pad=0)
    assert st == lib.TRI_OK
    assert lib.tri_get_info()[0] == lib.TRI_OK
    return x


@pytest.mark.parametrize("kind", ["ill", "pow2"])
@pytest.mark.parametrize("mixed", [False, True])
def test_ill_conditioned_diagonal_blocks_fp64(lib, mixed, kind):
    n = 2048
    if kind == "ill":
        b = _ill(96, 0.6, 3) if mixed else _ill(64, 1.0, 4)   # growth 1.2e6 / 3.4e7
    else:
        b = np.eye(64) - 2.0 * np.eye(64, k=-1)
    # plain: the 64-row leaf at row 320; mixed: inside the 256-row diagonal block [512, 768)
    r0 = 600 if mixed else 320
    t = _embedded(n, [(r0, b)])
    on = _run(lib, t, mixed, 1.0e4)
    off = _run(lib, t, mixed, 0.0)
    m = b.shape[0]
    want = oracle.tri_inv(t[r0:r0 + m, r0:r0 + m])
    e_on = _entry_rel_err(on[r0:r0 + m, r0:r0 + m], want)
    assert e_on <= 2.0 ** -23, e_on
    if kind == "ill":
        e_off = _entry_rel_err(off[r0:r0 + m, r0:r0 + m], want)
        assert e_off > 10 * e_on, (e_off, e_on)
    else:
        assert np.array_equal(on[r0:r0 + m, r0:r0 + m], want)   # x_ij = 2^(i-j): exact


@pytest.mark.parametrize("mixed", [False, True])
def test_growth_limit_leaves_well_conditioned_inputs_alone(lib, mixed):
    t = inputs.tri_lower(2048, seed=5, law="normal", dtype=np.float32).astype(np.float64)
    on = _run(lib, t, mixed, 1.0e4)
    off = _run(lib, t, mixed, 0.0)
    assert np.array_equal(on, off)


def test_growth_limit_setting(lib):
    assert lib.tri_set_growth_limit(float("nan")) == lib.TRI_ERR_ARG
    assert lib.tri_set_growth_limit(123.0) == lib.TRI_OK
    assert lib.tri_growth_limit() == pytest.approx(123.0)
    assert lib.tri_set_growth_limit(-1.0) == lib.TRI_OK
    assert lib.tri_growth_limit() == 0.0
    assert lib.tri_set_growth_limit(1.0e4) == lib.TRI_OK
