"""CTA-pair schedule of the mixed triangular path (tri_set_cta_pairs): the full-width level
products W = B X_A and X21 = -X_C W (block inverse, proof of the main Theorem, Section 3),
the residual R = I - T X and the update X += X R of the Newton-Schulz step, each computed by
clusters of two CTAs (256-row output tiles, one tcgen05.mma.cta_group::2 per k-step).

The pair schedule runs the same products and sums them in the same order as the
single-CTA schedule (the extra k-blocks of a 256-row tile multiply zeros), so its results
must be bit-identical; on top of that: parity against the FP64 oracle at the mixed path's
tolerance 40 sqrt(n) 2^-24, every product on its own, upper / unit views, ragged orders,
strided batches and the n = 8192 workload.  The setting is process-wide; every test
restores it."""
import numpy as np
import pytest

import oracle
from paper_2307_07611_gb300 import inputs
from tests._gpu import normwise_residual, rel_max_err, run_tri_inv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_07611_gb300 import lib as _lib
    _lib.load()
    before = _lib.tri_cta_pairs()
    yield _lib
    _lib.tri_set_cta_pairs(before)


def tol(n):
    return 40.0 * np.sqrt(n) * U32


def _run(lib, t, mask, **kw):
    assert lib.tri_set_cta_pairs(mask) == lib.TRI_OK
    try:
        x, st = run_tri_inv(lib, torch, t, dtype="f32", mixed=True, **kw)
    finally:
        lib.tri_set_cta_pairs(0)
    assert st == lib.TRI_OK
    assert lib.tri_get_info()[0] == lib.TRI_OK
    return x


def test_pairs_small_update_only(lib):
    """Smallest case first: one product (the update) on pairs, n = 1000 (ragged 256-row
    tiles), bit-identical to the single-CTA schedule."""
    n = 1000
    t = inputs.tri_lower(n, seed=11, law="normal", dtype=np.float32).astype(np.float64)
    ref = _run(lib, t, 0)
    got = _run(lib, t, lib.TRI_PAIR_UPD)
    assert np.array_equal(got, ref), np.abs(got - ref).max()


@pytest.mark.parametrize("mask", [1, 2, 4, 7])
@pytest.mark.parametrize("n", [700, 2048, 4500])
def test_pairs_bit_identical(lib, n, mask):
    t = inputs.tri_lower(n, seed=n + mask, law="normal", dtype=np.float32).astype(np.float64)
    ref = _run(lib, t, 0)
    got = _run(lib, t, mask)
    assert np.array_equal(got, ref), (mask, np.abs(got - ref).max())


@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("unit", [False, True])
def test_pairs_uplo_diag_parity(lib, lower, unit):
    n = 2300
    t = inputs.tri_lower(n, seed=5 + 2 * lower + unit, law="uniform")
    if not lower:
        t = t.T.copy()
    t = t.astype(np.float32).astype(np.float64)
    got = _run(lib, t, lib.TRI_PAIR_ALL, lower=lower, unit=unit, ld_pad=9)
    ref = _run(lib, t, 0, lower=lower, unit=unit, ld_pad=9)
    assert np.array_equal(got, ref)
    assert rel_max_err(got, oracle.tri_inv(t, lower=lower, unit=unit)) <= tol(n)


@pytest.mark.parametrize("n", [1537, 3000])
def test_pairs_oracle_parity_and_residual(lib, n):
    t = inputs.tri_lower(n, seed=n, law="normal", dtype=np.float32).astype(np.float64)
    x = _run(lib, t, lib.TRI_PAIR_ALL)
    assert rel_max_err(x, oracle.tri_inv(t)) <= tol(n)
    xp, _ = run_tri_inv(lib, torch, t, lower=True, dtype="f32")
    r_mixed, r_plain = normwise_residual(t, x), normwise_residual(t, xp)
    assert r_mixed <= 5e-6 and r_mixed <= 2.0 * r_plain, (r_mixed, r_plain)


def test_pairs_integer_family_bit_exact(lib):
    t = inputs.level_nilpotent_unit_lower(2048, 512, seed=3)[0]
    want = oracle.tri_inv(t, lower=True, unit=True)
    x = _run(lib, t, lib.TRI_PAIR_ALL, unit=True)
    assert np.array_equal(x, want)


def test_pairs_strided_batch(lib):
    """Three matrices of order 1300 in one strided batch: the pair tiles of all three in one
    schedule per product, bit-identical to the single-CTA schedule."""
    n, batch, ld = 1300, 3, 1304
    stride = ld * n + 64
    mats = [inputs.tri_lower(n, seed=40 + b, law="normal", dtype=np.float32) for b in range(batch)]
    host = np.zeros(stride * batch, dtype=np.float32)
    for b, m in enumerate(mats):
        host[b * stride: b * stride + ld * n].reshape(n, ld)[:, :n] = m.T

    def run(mask):
        assert lib.tri_set_cta_pairs(mask) == lib.TRI_OK
        dev = torch.from_numpy(host.copy()).cuda()
        st = lib.tri_inv_strided_batched(lib.TRI_LOWER, lib.TRI_NONUNIT, n, dev.data_ptr(), ld, stride, batch,
                                         lib.TRI_F32_MIXED, int(torch.cuda.current_stream().cuda_stream))
        torch.cuda.synchronize()
        lib.tri_set_cta_pairs(0)
        assert st == lib.TRI_OK
        return dev.cpu().numpy()

    got, ref = run(lib.TRI_PAIR_ALL), run(0)
    assert np.array_equal(got, ref)
    b = 1
    x = np.tril(got[b * stride: b * stride + ld * n].reshape(n, ld)[:, :n].T.astype(np.float64))
    assert rel_max_err(x, oracle.tri_inv(mats[b].astype(np.float64))) <= tol(n)


def test_pairs_setting(lib):
    assert lib.tri_set_cta_pairs(8) == lib.TRI_ERR_ARG
    assert lib.tri_set_cta_pairs(-1) == lib.TRI_ERR_ARG
    assert lib.tri_set_cta_pairs(lib.TRI_PAIR_RES) == lib.TRI_OK
    assert lib.tri_cta_pairs() == lib.TRI_PAIR_RES
    assert lib.tri_set_cta_pairs(0) == lib.TRI_OK


@pytest.mark.slow
def test_pairs_full_size_n8192(lib):
    """The n = 8192 workload: bit-identical to the single-CTA schedule, every element
    against the FP64 oracle, equal residual against plain FP32."""
    n = 8192
    t = inputs.tri_lower(n, seed=0, law="normal", dtype=np.float32).astype(np.float64)
    x = _run(lib, t, lib.TRI_PAIR_ALL, ld_pad=0)
    ref = _run(lib, t, 0, ld_pad=0)
    assert np.array_equal(x, ref)
    assert rel_max_err(x, oracle.tri_inv(t)) <= tol(n)
    xp, _ = run_tri_inv(lib, torch, t, lower=True, dtype="f32", ld_pad=0)
    r_mixed, r_plain = normwise_residual(t, x), normwise_residual(t, xp)
    assert r_mixed <= 5e-6 and r_mixed <= 2.0 * r_plain, (r_mixed, r_plain)
