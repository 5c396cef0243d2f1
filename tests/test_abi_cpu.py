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


def test_plain_workspace_formula(libtri):
    # one h x h block per active pair at the widest level, leaf 64
    for n, es, dt in [(8192, 4, lib.TRI_F32), (512, 8, lib.TRI_F64), (1000, 4, lib.TRI_F32)]:
        best, h = 0, 64
        while h < n:
            pairs = (n - h + 2 * h - 1) // (2 * h)
            best = max(best, pairs * h * h * es)
            h *= 2
        assert lib.tri_inv_workspace_size(n, dt) == best
