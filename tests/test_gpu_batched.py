"""GPU parity of the batched entry points (tri_inv_batched and the plan API: one
persistent, graph-captured launch) against the FP64 oracle, block by block.

Tolerance per block as for tri_inv: max |X - X_oracle| <= 40 sqrt(n) u max |X_oracle|.
Each block lives in its own device buffer padded with canary values, and its upper
triangle holds NaN: neither may change.
"""
import numpy as np
import pytest

import oracle
from paper_2307_07611_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = {"f32": 2.0 ** -24, "f64": 2.0 ** -53}
CANARY = -9.5e30


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_07611_gb300 import lib as _lib
    _lib.load()
    return _lib


def tol(n, dt):
    return 40.0 * np.sqrt(max(n, 1)) * U[dt]


class Batch:
    """Blocks stored column-major (ld = n) in one device buffer with canary gaps."""

    def __init__(self, blocks, lower, dt):
        self.np_dt = np.float64 if dt == "f64" else np.float32
        self.lower = lower
        self.sizes = [b.shape[0] for b in blocks]
        self.offs, off = [], 64
        for n in self.sizes:
            self.offs.append(off)
            off += n * n + 64
        host = np.full(off, CANARY, dtype=self.np_dt)
        for b, o in zip(blocks, self.offs):
            n = b.shape[0]
            m = np.array(b, dtype=np.float64)
            mask = np.tril(np.ones((n, n), bool)) if lower else np.triu(np.ones((n, n), bool))
            m[~mask] = np.nan
            host[o:o + n * n] = m.T.reshape(-1).astype(self.np_dt)
        self.host = host
        self.dev = torch.from_numpy(host.copy()).cuda()
        es = 8 if dt == "f64" else 4
        self.ptrs = [self.dev.data_ptr() + o * es for o in self.offs]

    def reset(self):
        self.dev.copy_(torch.from_numpy(self.host))

    def result(self, unit):
        out = self.dev.cpu().numpy()
        # canaries and the other triangle untouched
        bits = lambda a: a.view(np.uint64 if a.dtype == np.float64 else np.uint32)
        keep = np.ones(out.shape, bool)
        xs = []
        for n, o in zip(self.sizes, self.offs):
            x = out[o:o + n * n].reshape(n, n).T.astype(np.float64)
            tri = np.tril(np.ones((n, n), bool)) if self.lower else np.triu(np.ones((n, n), bool))
            if unit:
                tri &= ~np.eye(n, dtype=bool)
            keep[o:o + n * n] = ~tri.T.reshape(-1)
            x = np.where(tri, x, 0.0)
            if unit:
                np.fill_diagonal(x, 1.0)
            xs.append(x)
        assert np.array_equal(bits(out)[keep], bits(self.host)[keep]), "wrote outside the blocks' triangles"
        return xs


def check_blocks(xs, blocks, lower, unit, dt, exact=False):
    for x, t in zip(xs, blocks):
        want = oracle.tri_inv(t, lower=lower, unit=unit)
        if exact:
            assert np.array_equal(x, want)
        else:
            assert np.abs(x - want).max() <= tol(t.shape[0], dt) * max(np.abs(want).max(), 1e-300)


EDGE = [1, 2, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 200, 255, 256]


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("unit", [False, True])
def test_batched_edge_sizes(lib, dt, lower, unit):
    sizes = [s for s in EDGE if dt == "f32" or s <= 128]
    rng = np.random.default_rng(len(sizes) + lower + 2 * unit)
    blocks = []
    for n in sizes:
        t = inputs.tri_lower(n, law="uniform", rng=rng)
        if dt == "f32":
            t = t.astype(np.float32).astype(np.float64)
        blocks.append(t if lower else t.T.copy())
    b = Batch(blocks, lower, dt)
    code = lib.TRI_F64 if dt == "f64" else lib.TRI_F32
    st = lib.tri_inv_batched(len(sizes), sizes, b.ptrs, lib.TRI_LOWER if lower else lib.TRI_UPPER,
                             lib.TRI_UNIT if unit else lib.TRI_NONUNIT, code,
                             int(torch.cuda.current_stream().cuda_stream))
    assert st == lib.TRI_OK
    assert lib.tri_get_info()[0] == lib.TRI_OK
    check_blocks(b.result(unit), blocks, lower, unit, dt)


def test_batched_integer_blocks_bit_exact(lib):
    blocks = [inputs.ones_unit_lower(n) for n in (1, 17, 64, 256)]
    blocks += [inputs.bidiagonal_unit_lower(n, seed=n)[0] for n in (5, 130, 255)]
    blocks += [inputs.level_nilpotent_unit_lower(n, 32, seed=n)[0] for n in (96, 250)]
    b = Batch(blocks, True, "f32")
    st = lib.tri_inv_batched(len(blocks), [x.shape[0] for x in blocks], b.ptrs, lib.TRI_LOWER,
                             lib.TRI_NONUNIT, lib.TRI_F32, 0)
    assert st == lib.TRI_OK
    check_blocks(b.result(False), blocks, True, False, "f32", exact=True)


def test_batched_plan_graph_replay_config_batch(lib):
    """The batched workload: 4096 lower FP32 blocks, sizes uniform in {16..256}, uniform
    law with sqrt(n_b) scaling; plan (sorted queue, autotuned threads, captured graph)
    replayed twice; every block checked by its residual, a sample against the oracle."""
    sizes, blocks = inputs.batched_blocks(4096, seed=0, dtype=np.float32)
    blocks = [t.astype(np.float64) for t in blocks]
    b = Batch(blocks, True, "f32")
    st, plan = lib.tri_batched_plan_create(len(blocks), sizes, b.ptrs, lib.TRI_LOWER, lib.TRI_NONUNIT,
                                           lib.TRI_F32)
    assert st == lib.TRI_OK
    assert lib.tri_batched_plan_threads(plan) in (256, 512)
    assert [lib.tri_batched_plan_shape(plan, c)[0] for c in range(4)] == [
        int(np.sum(sizes > 160)), int(np.sum((sizes > 128) & (sizes <= 160))),
        int(np.sum((sizes > 32) & (sizes <= 128))), int(np.sum(sizes <= 32))]
    s = int(torch.cuda.current_stream().cuda_stream)
    for rep in range(2):
        b.reset()
        assert lib.tri_batched_exec(plan, s) == lib.TRI_OK
        torch.cuda.synchronize()
        xs = b.result(False)
    assert lib.tri_batched_plan_destroy(plan) == lib.TRI_OK
    assert lib.tri_get_info()[0] == lib.TRI_OK
    for x, t in zip(xs, blocks):
        r = t @ x - np.eye(t.shape[0])
        assert np.linalg.norm(r) / (np.linalg.norm(t) * np.linalg.norm(x)) <= 5e-6
    order = np.argsort(sizes)
    sample = list(order[:8]) + list(order[-8:]) + list(range(0, 4096, 257))
    check_blocks([xs[i] for i in sample], [blocks[i] for i in sample], True, False, "f32")


def test_batched_size_classes_and_tune_cache(lib, tmp_path):
    """Blocks of every size class in one plan (161..256 rows, 129..160, 33..128, up to 32): each class
    runs with the CTA shape the autotuner picked; the results match the oracle; the tuner's
    choices round-trip through the JSON tune cache."""
    import json
    sizes = [256, 200, 129, 128, 77, 33, 32, 20, 1] * 3
    rng = np.random.default_rng(11)
    blocks = [inputs.tri_lower(n, law="uniform", rng=rng).astype(np.float32).astype(np.float64) for n in sizes]
    b = Batch(blocks, True, "f32")
    st, plan = lib.tri_batched_plan_create(len(blocks), sizes, b.ptrs, lib.TRI_LOWER, lib.TRI_NONUNIT,
                                           lib.TRI_F32)
    assert st == lib.TRI_OK
    shapes = [lib.tri_batched_plan_shape(plan, c) for c in range(4)]
    assert [sh[0] for sh in shapes] == [6, 3, 9, 9]
    assert shapes[0][1] in (256, 512) and shapes[1][1] in (256, 512) and shapes[2][1] in (128, 256)
    assert shapes[3][1] in (32, 64)
    assert all(sh[2] >= 1 for sh in shapes)
    assert lib.tri_batched_exec(plan, int(torch.cuda.current_stream().cuda_stream)) == lib.TRI_OK
    torch.cuda.synchronize()
    check_blocks(b.result(False), blocks, True, False, "f32")
    assert lib.tri_batched_plan_destroy(plan) == lib.TRI_OK
    path = str(tmp_path / "tune.json")
    assert lib.tri_tune_cache_save(path) == lib.TRI_OK
    doc = json.load(open(path))
    assert doc["version"] == 1 and len(doc["entries"]) >= 4
    assert all(e["threads"] in (32, 64, 128, 256, 512) for e in doc["entries"])
    st, n = lib.tri_tune_cache_load(path)
    assert st == lib.TRI_OK and n == len(doc["entries"])


def test_batched_singular_block_reported(lib):
    blocks = [inputs.tri_lower(n, seed=n) for n in (40, 90, 150)]
    blocks[1][33, 33] = 0.0
    blocks[2][7, 7] = 0.0
    b = Batch(blocks, True, "f32")
    lib.tri_inv_batched(3, [40, 90, 150], b.ptrs, lib.TRI_LOWER, lib.TRI_NONUNIT, lib.TRI_F32, 0)
    st, bad = lib.tri_get_info()
    assert st == lib.TRI_ERR_SINGULAR and bad == 1


def test_batched_rejects_large_blocks(lib):
    buf = torch.zeros(300 * 300, device="cuda")
    assert lib.tri_inv_batched(1, [300], [buf.data_ptr()], 0, 0, lib.TRI_F32, 0) == lib.TRI_ERR_UNSUPPORTED
    assert lib.tri_inv_batched(1, [129], [buf.data_ptr()], 0, 0, lib.TRI_F64, 0) == lib.TRI_ERR_UNSUPPORTED
    assert lib.tri_inv_batched(0, [], [], 0, 0, lib.TRI_F32, 0) == lib.TRI_OK


def _ill_block(n, scale, seed):
    """Unit-diagonal lower block with strict lower entries N(0,1) * scale: growth
    max|X| max|T| far above 1e4 at the sizes used (measured on the host: n = 96,
    scale 0.6 gives 1.2e6), while a plain FP32 recurrence loses digits in the small
    entries of X."""
    g = np.random.default_rng(seed)
    return np.eye(n) + np.tril(g.standard_normal((n, n)), -1) * scale


def _run_plan(lib, blocks, tau, unit):
    b = Batch(blocks, True, "f32")
    sizes = [t.shape[0] for t in blocks]
    st, plan = lib.tri_batched_plan_create(len(blocks), sizes, b.ptrs, lib.TRI_LOWER,
                                           lib.TRI_UNIT if unit else lib.TRI_NONUNIT, lib.TRI_F32)
    assert st == lib.TRI_OK
    if tau is not None:
        assert lib.tri_batched_plan_set_growth_limit(plan, tau) == lib.TRI_OK
    assert lib.tri_batched_exec(plan, int(torch.cuda.current_stream().cuda_stream)) == lib.TRI_OK
    torch.cuda.synchronize()
    assert lib.tri_batched_plan_destroy(plan) == lib.TRI_OK
    return b.result(unit)


def _entry_rel_err(x, t):
    want = oracle.tri_inv(t.astype(np.float32).astype(np.float64), lower=True, unit=True)
    m = np.tril(np.ones(t.shape, bool), -1) & (want != 0)
    return np.max(np.abs(x[m] - want[m]) / np.abs(want[m]))


def test_batched_growth_limit_fp64_leaf(lib):
    """An FP64 leaf only for ill-conditioned blocks: with the default limit (1e4) a block of
    order <= 128 whose FP32 inverse shows growth above it is inverted again in FP64, so every
    entry is within one FP32 rounding of the FP64 oracle (2^-24 relative, plus FP64 error);
    with the limit disabled the FP32 recurrence is measurably worse on the same block."""
    blocks = [_ill_block(96, 0.6, 3), _ill_block(64, 1.0, 4)]
    on = _run_plan(lib, blocks, None, True)
    off = _run_plan(lib, blocks, 0.0, True)
    for x_on, x_off, t in zip(on, off, blocks):
        e_on, e_off = _entry_rel_err(x_on, t), _entry_rel_err(x_off, t)
        assert e_on <= 2.0 ** -23, e_on
        assert e_off > 10 * e_on, (e_off, e_on)
    assert lib.tri_get_info()[0] == lib.TRI_OK


def test_batched_growth_limit_power_of_two_block(lib):
    """Subdiagonal -2 (x_ij = 2^(i-j), growth 2^(n-1)): the FP64 leaf runs and the result is
    exact."""
    n = 64
    t = np.eye(n) - 2.0 * np.eye(n, k=-1)
    (x,) = _run_plan(lib, [t], None, False)
    want = np.tril(2.0 ** (np.arange(n)[:, None] - np.arange(n)[None, :]))
    assert np.array_equal(x, want)


def test_batched_growth_limit_leaves_the_rest_alone(lib):
    """Well-conditioned blocks (the batched law), up to 256 rows, keep the FP32 result:
    bit-identical with the limit on and off."""
    blocks = [inputs.tri_lower(n, seed=n).astype(np.float64) for n in (40, 128, 200, 256)]
    on = _run_plan(lib, blocks, None, False)
    off = _run_plan(lib, blocks, 0.0, False)
    for a, b in zip(on, off):
        assert np.array_equal(a, b)


def test_batched_growth_limit_large_blocks(lib):
    """Ill-conditioned blocks of 129..256 rows (their FP64 tiles do not fit in shared
    memory) are inverted again by the FP64 column recurrence from the unchanged source:
    entrywise within 2^-23 of the FP64 oracle, against far worse without the limit; the
    well-conditioned block beside them is untouched."""
    blocks = [_ill_block(200, 0.5, 7), _ill_block(256, 0.45, 8), inputs.tri_lower(180, seed=9).astype(np.float64)]
    on = _run_plan(lib, blocks, None, True)
    off = _run_plan(lib, blocks, 0.0, True)
    for x_on, x_off, t in zip(on[:2], off[:2], blocks[:2]):
        e_on, e_off = _entry_rel_err(x_on, t), _entry_rel_err(x_off, t)
        assert e_on <= 2.0 ** -23, e_on
        assert e_off > 10 * e_on, (e_off, e_on)
    assert np.array_equal(on[2], off[2])
    assert lib.tri_get_info()[0] == lib.TRI_OK


def test_batched_growth_limit_errors(lib):
    buf = torch.zeros(64 * 64, dtype=torch.float64, device="cuda")
    st, plan = lib.tri_batched_plan_create(1, [64], [buf.data_ptr()], lib.TRI_LOWER, lib.TRI_UNIT, lib.TRI_F64)
    assert st == lib.TRI_OK
    assert lib.tri_batched_plan_set_growth_limit(plan, 10.0) == lib.TRI_ERR_UNSUPPORTED
    assert lib.tri_batched_plan_set_growth_limit(plan, float("nan")) == lib.TRI_ERR_ARG
    assert lib.tri_batched_plan_destroy(plan) == lib.TRI_OK
