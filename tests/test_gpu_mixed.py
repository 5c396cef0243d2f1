"""GPU tests of the mixed-precision path (TRI_F32_MIXED): the tcgen05 product kernel on
its own, then the whole inverse against the FP64 oracle.

Product kernel: BF16 x BF16 products are exact in FP32, so C differs from the exact
sum only by FP32 accumulation: |C - C_exact| <= k * 2^-23 * (|A| |B|)_ij is a loose
bound; the test asserts 8 * sqrt(k) * 2^-24 * (|A| |B|)_ij + tiny (random-sign rounding).

Mixed inverse: after the Newton-Schulz step the result must reach the plain FP32
accuracy class: the same oracle tolerance as the plain path (40 sqrt(n) u32 max|X|), a
normwise residual <= 5e-6 and <= 2x the plain FP32 path's residual on the same input.
Integer families whose inverses stay below 2^8 in magnitude are exact in one BF16
piece, so the mixed path must reproduce them bit for bit (R = 0 exactly, the update is
a no-op).
"""
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
    return _lib


def colmajor_bf16(x, ld):
    """x (rows x cols) -> device BF16 tensor, column-major with leading dimension ld; the
    padding rows hold NaN, which must never reach a stored result."""
    rows, cols = x.shape
    buf = torch.full((cols, ld), float("nan"), dtype=torch.bfloat16)
    buf[:, :rows] = torch.from_numpy(np.ascontiguousarray(x.T)).to(torch.bfloat16)
    return buf.cuda()


@pytest.mark.parametrize("m,n,k,nt", [(128, 256, 64, 1), (128, 256, 16, 1), (300, 520, 200, 2),
                                      (1024, 768, 1000, 3), (64, 40, 8, 1), (1500, 300, 2048, 2)])
def test_tc_product_kernel(lib, m, n, k, nt):
    rng = np.random.default_rng(m + n + k)
    lda = (m + 7) // 8 * 8 + 8
    ldb = (k + 7) // 8 * 8
    As, Bs, ad, bd = [], [], [], []
    for _ in range(nt):
        a = rng.standard_normal((m, k)).astype(np.float32)
        b = rng.standard_normal((k, n)).astype(np.float32)
        da, db = colmajor_bf16(a, lda), colmajor_bf16(b, ldb)
        ad.append(da)
        bd.append(db)
        As.append(da.float().cpu().numpy()[:, :m].T.astype(np.float64))
        Bs.append(db.float().cpu().numpy()[:, :k].T.astype(np.float64))
    ldc = m + 5
    c = torch.full((n, ldc), float("nan"), dtype=torch.float32, device="cuda")
    st = lib.tri_tc_gemm_bf16(m, n, k, [x.data_ptr() for x in ad], lda, [x.data_ptr() for x in bd],
                              ldb, c.data_ptr(), ldc, int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == lib.TRI_OK
    got = c.cpu().numpy()
    assert np.isnan(got[:, m:]).all(), "wrote past m rows"
    got = got[:, :m].T.astype(np.float64)
    want = sum(a @ b for a, b in zip(As, Bs))
    scale = sum(np.abs(a) @ np.abs(b) for a, b in zip(As, Bs))
    err = np.abs(got - want)
    assert (err <= 8 * np.sqrt(k) * U32 * scale + 1e-30).all(), float((err / (scale + 1e-30)).max())


def tol(n):
    return 40.0 * np.sqrt(n) * U32


@pytest.mark.parametrize("n", [257, 300, 511, 512, 700, 1000, 1537, 2048, 3000])
def test_mixed_lower_parity(lib, n):
    t = inputs.tri_lower(n, seed=n, law="normal").astype(np.float32).astype(np.float64)
    x, st = run_tri_inv(lib, torch, t, lower=True, dtype="f32", mixed=True)
    assert st == lib.TRI_OK
    assert lib.tri_get_info()[0] == lib.TRI_OK
    want = oracle.tri_inv(t)
    assert rel_max_err(x, want) <= tol(n)
    xp, _ = run_tri_inv(lib, torch, t, lower=True, dtype="f32")
    r_mixed, r_plain = normwise_residual(t, x), normwise_residual(t, xp)
    assert r_mixed <= 5e-6
    assert r_mixed <= 2.0 * r_plain, (r_mixed, r_plain)


@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("unit", [False, True])
@pytest.mark.parametrize("n", [600, 1300])
def test_mixed_uplo_diag_parity(lib, lower, unit, n):
    t = inputs.tri_lower(n, seed=3 * n + lower + 2 * unit, law="uniform")
    if not lower:
        t = t.T.copy()
    t = t.astype(np.float32).astype(np.float64)
    x, st = run_tri_inv(lib, torch, t, lower=lower, unit=unit, dtype="f32", mixed=True, ld_pad=9,
                        workspace=(n == 600))
    assert st == lib.TRI_OK
    want = oracle.tri_inv(t, lower=lower, unit=unit)
    assert rel_max_err(x, want) <= tol(n)
    tu = t.copy()
    if unit:
        np.fill_diagonal(tu, 1.0)
    assert normwise_residual(tu, x) <= 5e-6


@pytest.mark.parametrize("lower", [True, False])
def test_mixed_integer_families_bit_exact(lib, lower):
    cases = [inputs.ones_unit_lower(1000),
             inputs.bidiagonal_unit_lower(1500, seed=1)[0],
             inputs.level_nilpotent_unit_lower(1100, 256, seed=2)[0],
             inputs.level_nilpotent_unit_lower(2048, 512, seed=3)[0],
             inputs.level_nilpotent_unit_lower(700, 64, seed=6)[0]]
    t1, _ = inputs.level_nilpotent_unit_lower(1024, 256, seed=4, lo=-1, hi=1)
    t2, _ = inputs.level_nilpotent_unit_lower(1024, 512, seed=5, lo=-1, hi=1)
    cases.append(t1 @ t2)
    for t in cases:
        if not lower:
            t = t.T.copy()
        want = oracle.tri_inv(t, lower=lower, unit=True)
        assert np.abs(want).max() < 256
        for unit in (True, False):
            x, st = run_tri_inv(lib, torch, t, lower=lower, unit=unit, dtype="f32", mixed=True)
            assert st == lib.TRI_OK
            assert np.array_equal(x, want), (t.shape, unit, np.abs(x - want).max())


def test_mixed_singular_reported(lib):
    n = 900
    t = inputs.tri_lower(n, seed=3)
    t[700, 700] = 0.0
    run_tri_inv(lib, torch, t, lower=True, dtype="f32", mixed=True)
    st, bad = lib.tri_get_info()
    assert st == lib.TRI_ERR_SINGULAR and bad == 700


def test_mixed_small_sizes_fall_back_to_fp32_levels(lib):
    for n in (1, 5, 64, 200, 256):
        t = inputs.tri_lower(n, seed=n, law="normal").astype(np.float32).astype(np.float64)
        x, st = run_tri_inv(lib, torch, t, lower=True, dtype="f32", mixed=True)
        assert st == lib.TRI_OK
        assert rel_max_err(x, oracle.tri_inv(t)) <= tol(n)


@pytest.mark.slow
def test_mixed_full_size_n8192(lib):
    """The FP32 n = 8192 workload on the mixed path: every element against the FP64
    oracle (all 8192 columns, threaded over the host's cores), the normwise residual, and
    the equal-residual criterion against the plain path."""
    n = 8192
    t = inputs.tri_lower(n, seed=0, law="normal", dtype=np.float32).astype(np.float64)
    x, st = run_tri_inv(lib, torch, t, lower=True, dtype="f32", mixed=True, ld_pad=0)
    assert st == lib.TRI_OK
    want = oracle.tri_inv(t)
    assert rel_max_err(x, want) <= tol(n)
    xp, _ = run_tri_inv(lib, torch, t, lower=True, dtype="f32", ld_pad=0)
    r_mixed, r_plain = normwise_residual(t, x), normwise_residual(t, xp)
    assert r_mixed <= 5e-6 and r_mixed <= 2.0 * r_plain, (r_mixed, r_plain)


def test_mixed_graph_schedule_same_results(lib):
    """The single-launch dependency-driven schedule (TRI_MIXED_SCHEDULE=graph, read once
    per process) runs the same products in another order: the parity, uplo / diag and
    bit-exact tests above must pass under it too (run in a child process)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, TRI_MIXED_SCHEDULE="graph")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu",
                        os.path.join(root, "tests", "test_gpu_mixed.py"),
                        "-k", "lower_parity or uplo_diag or integer_families or singular"],
                       cwd=root, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout


def test_mixed_merged_levels_bit_identical_to_per_level_launches(lib, tmp_path):
    """Every split level runs by default in launches of its own; TRI_MIXED_SCHEDULE=merged
    (read once per process) runs the low levels (h = 256 .. 1024) as one launch whose
    tiles wait on the dependency counters of the pairs they read.  Both run the same
    products in the same order, so the inverses must be bit-identical: the merged result
    is computed in a child process and compared."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cases = [(700, 1, True, False), (1537, 2, True, False), (2048, 3, False, True), (3000, 4, True, False)]
    child = (
        "import sys, numpy as np, torch\n"
        "sys.path.insert(0, %r)\n"
        "from paper_2307_07611_gb300 import inputs, lib\n"
        "from tests._gpu import run_tri_inv\n"
        "lib.load()\n"
        "for n, seed, lower, unit in %r:\n"
        "    t = inputs.tri_lower(n, seed=seed, law='normal', dtype=np.float32).astype(np.float64)\n"
        "    t = t if lower else t.T.copy()\n"
        "    x, st = run_tri_inv(lib, torch, t, lower=lower, unit=unit, dtype='f32', mixed=True)\n"
        "    assert st == lib.TRI_OK\n"
        "    np.save(%r + '/x%%d.npy' %% n, x)\n" % (root, cases, str(tmp_path)))
    env = dict(os.environ, TRI_MIXED_SCHEDULE="merged")
    r = subprocess.run([sys.executable, "-c", child], cwd=root, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    for n, seed, lower, unit in cases:
        t = inputs.tri_lower(n, seed=seed, law="normal", dtype=np.float32).astype(np.float64)
        t = t if lower else t.T.copy()
        x, st = run_tri_inv(lib, torch, t, lower=lower, unit=unit, dtype="f32", mixed=True)
        assert st == lib.TRI_OK and lib.tri_get_info()[0] == lib.TRI_OK
        assert np.array_equal(x, np.load(str(tmp_path / ("x%d.npy" % n)))), n
        assert rel_max_err(x, oracle.tri_inv(t, lower=lower, unit=unit)) <= tol(n)
