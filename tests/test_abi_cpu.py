"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/triinv.h declares, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

from paper_2307_07611_gb300 import build as cuda_build
from paper_2307_07611_gb300 import lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libtri():
    cuda_build.build()
    return lib.load()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^TRI_API\s+[^;(]*?\b(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ["tri_inv", "tri_inv_ex", "tri_inv_workspace_size", "tri_get_info",
                 "tri_status_string"]:
        assert must in names


def test_every_declared_symbol_is_exported(libtri):
    missing = [n for n in declared_functions() if not hasattr(libtri, n)]
    assert not missing, missing


def test_binding_names_match_abi():
    for n in declared_functions():
        if n == "tri_status_string":
            continue
        assert hasattr(lib, n), f"python binding lacks {n}"


def test_status_strings(libtri):
    for s in range(7):
        assert lib.status_string(s).startswith("TRI_")
    assert "unknown" in lib.status_string(99)


def test_argument_errors_need_no_gpu(libtri):
    A = lib.TRI_ERR_ARG
    assert lib.tri_inv(0, 0, -1, 0, 1, lib.TRI_F32) == A           # n < 0
    assert lib.tri_inv(0, 0, 0, 0, 1, lib.TRI_F32) == lib.TRI_OK   # n == 0: no-op
    assert lib.tri_inv(0, 0, 5, 0, 5, lib.TRI_F32) == A            # NULL
    assert lib.tri_inv(0, 0, 5, 4096, 4, lib.TRI_F32) == A         # lda < n
    assert lib.tri_inv(0, 0, 5, 4096, 5, 9) == A                   # dtype
    assert lib.tri_inv(2, 0, 5, 4096, 5, lib.TRI_F32) == A         # uplo
    assert lib.tri_inv(0, 3, 5, 4096, 5, lib.TRI_F32) == A         # diag


def test_workspace_checks_need_no_gpu(libtri):
    n = 1000
    need = lib.tri_inv_workspace_size(n, lib.TRI_F32)
    assert need > 0
    assert lib.tri_inv_ex(0, 0, n, 4096, n, lib.TRI_F32, 0, 0) == lib.TRI_ERR_NOMEM
    assert lib.tri_inv_ex(0, 0, n, 4096, n, lib.TRI_F32, 256, need - 1) == lib.TRI_ERR_NOMEM
    assert lib.tri_inv_ex(0, 0, n, 4096, n, lib.TRI_F32, 256 + 8, need) == lib.TRI_ERR_NOMEM
    assert lib.tri_inv_workspace_size(0, lib.TRI_F32) == 0
    assert lib.tri_inv_workspace_size(64, lib.TRI_F32) == 0   # a single leaf


def test_noalloc_limits_fit_its_scratch(libtri):
    """The documented limits of tri_inv_noalloc (FP32 n <= 4096, FP64 n <= 2048) follow from
    tri_inv_workspace_size and the array size declared in the header."""
    import re
    hdr = open(os.path.join(ROOT, "include", "triinv.h")).read()
    m = re.search(r"#define TRI_NOALLOC_SCRATCH_BYTES \((\d+)u << (\d+)\)", hdr)
    cap = int(m.group(1)) << int(m.group(2))
    assert cap == lib.TRI_NOALLOC_SCRATCH_BYTES
    assert lib.tri_inv_workspace_size(4096, lib.TRI_F32) <= cap < lib.tri_inv_workspace_size(4097, lib.TRI_F32)
    assert lib.tri_inv_workspace_size(2048, lib.TRI_F64) <= cap < lib.tri_inv_workspace_size(2049, lib.TRI_F64)


def test_plain_workspace_formula(libtri):
    # one h x h block per active pair at the widest level, leaf 64
    for n, es, dt in [(8192, 4, lib.TRI_F32), (512, 8, lib.TRI_F64), (1000, 4, lib.TRI_F32)]:
        best, h = 0, 64
        while h < n:
            pairs = (n - h + 2 * h - 1) // (2 * h)
            best = max(best, pairs * h * h * es)
            h *= 2
        assert lib.tri_inv_workspace_size(n, dt) == best


def _tiles_expected(n):
    """128 x 256 output tiles of the mixed path's products: per split level h >= 256,
    W = B X_A (h/256 column tiles x ceil(hc/128) row tiles per pair) and X21 (the same
    count), then R and the update (one tile per 128 x 256 block meeting the lower
    triangle)."""
    cd = lambda a, b: -(-a // b)
    total = 0
    h = 256
    while h < n:
        q = 0
        while 2 * q * h + h < n:
            hc = min(h, n - (2 * q * h + h))
            total += 2 * (h // 256) * cd(hc, 128)
            q += 1
        h *= 2
    ns = sum(cd(min((tm + 1) * 128, n), 256) for tm in range(cd(n, 128)))
    return total + 2 * ns


@pytest.mark.parametrize("n", [257, 300, 512, 777, 1000, 1024, 2048, 3000, 4096, 8192])
def test_mixed_schedule_is_complete_and_deadlock_free(libtri, n):
    """The host schedule of the mixed path: every tile once, lists that replay to
    completion in order (no circular wait), makespan no shorter than either lower bound,
    flops = the algorithmic count (3 terms per level product, 6 + 1 for Newton-Schulz)."""
    s = lib.tri_mixed_schedule_stats(n, 152)
    assert s["tiles"] == _tiles_expected(n)
    assert s["replay_ok"] == 1.0
    assert s["makespan"] >= s["critical_path"] - 1e-9
    assert s["makespan"] >= s["work_per_cta"] - 1e-9
    fl = 0.0
    h = 256
    while h < n:
        q = 0
        while 2 * q * h + h < n:
            hc = min(h, n - (2 * q * h + h))
            fl += 3.0 * hc * h * (h + 1) + 3.0 * h * hc * (hc + 1)
            q += 1
        h *= 2
    fl += 7.0 * n * (n + 1) * (n + 2) / 3.0
    assert s["flops"] == pytest.approx(fl, rel=1e-12)
    assert s["ctas"] == min(152, s["tiles"])


def test_mixed_schedule_small_grids_and_errors(libtri):
    for ctas in (1, 2, 7):
        s = lib.tri_mixed_schedule_stats(2048, ctas)
        assert s["replay_ok"] == 1.0 and s["ctas"] == ctas
    with pytest.raises(lib.TriError):
        lib.tri_mixed_schedule_stats(256, 152)      # no tensor-core part
    with pytest.raises(lib.TriError):
        lib.tri_mixed_schedule_stats(4096, 0)


def test_combrit_argument_errors_need_no_gpu(libtri):
    A = lib.TRI_ERR_ARG
    assert lib.tri_inv_combrit(0, 0, 16, 4096, 16, lib.TRI_F32, 3) == A          # beta not 2/4/8/16
    assert lib.tri_inv_combrit(0, 0, 16, 4096, 16, lib.TRI_F32, 32) == A
    assert lib.tri_inv_combrit(0, 0, -1, 4096, 16, lib.TRI_F32, 4) == A
    assert lib.tri_inv_combrit(0, 0, 16, 4096, 16, lib.TRI_F32_MIXED, 4) == lib.TRI_ERR_UNSUPPORTED
    assert lib.tri_inv_combrit(0, 0, 0, 0, 1, lib.TRI_F64, 8) == lib.TRI_OK       # n == 0: no-op
    assert lib.tri_inv_combrit(0, 0, 16, 0, 16, lib.TRI_F32, 2) == A             # NULL
    assert lib.tri_inv_combrit(0, 0, 16, 4096, 15, lib.TRI_F32, 2) == A          # lda < n


def test_skul_argument_errors_need_no_gpu(libtri):
    A = lib.TRI_ERR_ARG
    assert lib.skul(-1, 4096, 1, 8192, 1, lib.TRI_F32) == A
    assert lib.skul(0, 0, 1, 0, 1, lib.TRI_F32) == lib.TRI_OK                # n == 0: no-op
    assert lib.skul(8, 0, 8, 8192, 8, lib.TRI_F32) == A                      # NULL a
    assert lib.skul(8, 4096, 8, 0, 8, lib.TRI_F32) == A                      # NULL sk
    assert lib.skul(8, 4096, 8, 4096, 8, lib.TRI_F32) == A                   # a == sk
    assert lib.skul(8, 4096, 7, 8192, 8, lib.TRI_F32) == A                   # lda < n
    assert lib.skul(8, 4096, 8, 8192, 7, lib.TRI_F64) == A                   # ldsk < n
    assert lib.skul(8, 4096, 8, 8192, 8, 9) == A                             # dtype
    assert lib.skul(70000, 4096, 70000, 8192, 70000, lib.TRI_F32) == lib.TRI_ERR_UNSUPPORTED
    need = lib.skul_workspace_size(1000, lib.TRI_F32)
    assert need > 0 and lib.skul_workspace_size(0, lib.TRI_F32) == 0
    # the K\S buffer is the caller's: less scratch than gen_inv by about n^2 elements
    assert need < lib.gen_inv_workspace_size(1000, lib.TRI_F32)
    assert lib.skul_ex(1000, 4096, 1000, 8192, 1000, lib.TRI_F32, 256, need - 1) == lib.TRI_ERR_NOMEM
    assert lib.skul_ex(1000, 4096, 1000, 8192, 1000, lib.TRI_F32, 264, need) == lib.TRI_ERR_NOMEM


def test_sqr_argument_errors_need_no_gpu(libtri):
    A = lib.TRI_ERR_ARG
    n = 8
    assert lib.sqr(-1, 4096, 1, 8192, 1, 16384, 1, lib.TRI_F32) == A
    assert lib.sqr(0, 0, 1, 0, 1, 0, 1, lib.TRI_F32) == lib.TRI_OK                 # n == 0: no-op
    assert lib.sqr(n, 0, n, 8192, n, 16384, n, lib.TRI_F32) == A                   # NULL a
    assert lib.sqr(n, 4096, n, 8192, n, 0, n, lib.TRI_F32) == A                    # NULL s
    assert lib.sqr(n, 4096, n - 1, 8192, n, 16384, n, lib.TRI_F32) == A            # lda < n
    assert lib.sqr(n, 4096, n, 8192, n, 16384, n, 9) == A                          # dtype
    # overlapping outputs (r starts inside a's n x n footprint)
    assert lib.sqr_ex(n, 4096, n, 4096 + 64, n, 16384, n, lib.TRI_F32, 256, 1 << 20) == A
    assert lib.sqr_ex(n, 4096, n, 8192, n, 8192, n, lib.TRI_F64, 256, 1 << 20) == A  # r == s
    assert lib.sqr(70000, 4096, 70000, 8192, 70000, 16384, 70000, lib.TRI_F32) == lib.TRI_ERR_UNSUPPORTED
    need = lib.sqr_workspace_size(1000, lib.TRI_F32)
    assert need > 0 and lib.sqr_workspace_size(0, lib.TRI_F32) == 0
    assert lib.sqr_ex(1000, 4096, 1000, 1 << 24, 1000, 1 << 25, 1000, lib.TRI_F32, 256, need - 1) \
        == lib.TRI_ERR_NOMEM
    assert lib.sqr_inv(-1, 4096, 1, lib.TRI_F32) == A
    assert lib.sqr_inv(0, 0, 1, lib.TRI_F32) == lib.TRI_OK
    assert lib.sqr_inv(4, 0, 4, lib.TRI_F32) == A


def test_batched_growth_limit_null_plan_needs_no_gpu(libtri):
    assert lib.tri_batched_plan_set_growth_limit(None, 1e4) == lib.TRI_ERR_ARG


def test_brsi_argument_errors_need_no_gpu(libtri):
    A = lib.TRI_ERR_ARG
    assert lib.brsi_inv(-1, 4096, 1, 2, lib.TRI_F32) == A
    assert lib.brsi_inv(5, 4096, 5, 1, lib.TRI_F32) == A
    assert lib.brsi_inv(5, 4096, 5, 17, lib.TRI_F32) == A
    assert lib.brsi_inv(5, 0, 5, 2, lib.TRI_F32) == A
    assert lib.brsi_inv(5, 4096, 5, 2, lib.TRI_F32, perm=[0, 0, 1, 2, 3]) == A
    assert lib.brsi_inv(5, 4096, 5, 2, 9) == A
    assert lib.brsi_inv_workspace_size(100, 1, lib.TRI_F32) == 0
    need = lib.brsi_inv_workspace_size(100, 4, lib.TRI_F32)
    assert need >= 4 * 100 * 100 * 4
    assert lib.brsi_inv_ex(100, 4096, 100, 4, lib.TRI_F32, 256, need - 1) == lib.TRI_ERR_NOMEM


def test_tune_cache_file_errors_need_no_gpu(libtri, tmp_path):
    assert lib.tri_tune_cache_load(str(tmp_path / "missing.json"))[0] == lib.TRI_ERR_ARG
    bad = tmp_path / "bad.json"
    bad.write_text('{"version": 1, "entries": [{"key": "x", "threads": 7}]}')
    assert lib.tri_tune_cache_load(str(bad))[0] == lib.TRI_ERR_ARG
    good = tmp_path / "good.json"
    good.write_text('{"version": 1, "entries": [{"key": "cpu-test:1:c2:0,", "threads": 32}]}')
    assert lib.tri_tune_cache_load(str(good)) == (lib.TRI_OK, 1)
    out = tmp_path / "out.json"
    assert lib.tri_tune_cache_save(str(out)) == lib.TRI_OK
    import json
    assert any(e["key"] == "cpu-test:1:c2:0," for e in json.load(open(out))["entries"])



def test_process_settings_need_no_gpu(libtri):
    """The process-wide settings (growth limit, mixed recipe, CTA-pair products) validate
    their argument and round-trip without a device."""
    assert lib.tri_set_cta_pairs(8) == lib.TRI_ERR_ARG
    assert lib.tri_set_cta_pairs(lib.TRI_PAIR_LEVELS | lib.TRI_PAIR_UPD) == lib.TRI_OK
    assert lib.tri_cta_pairs() == lib.TRI_PAIR_LEVELS | lib.TRI_PAIR_UPD
    assert lib.tri_set_cta_pairs(0) == lib.TRI_OK
    assert lib.tri_set_mixed_recipe(5) == lib.TRI_ERR_ARG
    assert lib.tri_mixed_recipe() == lib.TRI_RECIPE_NEWTON_SCHULZ
