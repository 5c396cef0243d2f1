"""Per-call status words (`d_info` of the `_ex` entry points): each call records its own
first bad pivot (or -1) in the caller's device word, so calls on different streams do not
see each other's singular pivots, and the device-wide word of tri_get_info is untouched.
A zero pivot is the paper's stop condition for the inverse (Section 4.2, CRIT divides by
t_ii; Section 5.1, SKUL divides by the pivot)."""
import numpy as np
import pytest

from paper_2307_07611_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_07611_gb300 import lib as _lib
    _lib.load()
    return _lib


def _ws(lib, need):
    buf = torch.empty(max(need, 1) + 256, dtype=torch.uint8, device="cuda")
    return buf, (buf.data_ptr() + 255) // 256 * 256


@pytest.mark.parametrize("dt", ["f64", "f32", "mixed"])
def test_tri_inv_ex_info_per_stream(lib, dt):
    n, bad = 700, 123
    code = {"f64": lib.TRI_F64, "f32": lib.TRI_F32, "mixed": lib.TRI_F32_MIXED}[dt]
    tdt = torch.float64 if dt == "f64" else torch.float32
    t_bad = inputs.tri_lower(n, seed=5, law="normal")
    t_bad[bad, bad] = 0.0
    t_ok = inputs.tri_lower(n, seed=6, law="normal")
    src1 = torch.from_numpy(np.ascontiguousarray(t_bad.T)).to(tdt).cuda()
    src2 = torch.from_numpy(np.ascontiguousarray(t_ok.T)).to(tdt).cuda()
    a1, a2 = torch.empty_like(src1), torch.empty_like(src2)
    need = lib.tri_inv_workspace_size(n, code)
    w1, p1 = _ws(lib, need)
    w2, p2 = _ws(lib, need)
    info = torch.full((2,), 777, dtype=torch.int64, device="cuda")
    assert lib.tri_get_info()[0] == lib.TRI_OK          # clears the device-wide word
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    for rep in range(2):                                 # the word is reset by every call
        a1.copy_(src1)                                   # in place: restore the inputs
        a2.copy_(src2)
        torch.cuda.synchronize()
        st1 = lib.tri_inv_ex(0, 0, n, a1.data_ptr(), n, code, p1, need, int(s1.cuda_stream),
                             d_info=info.data_ptr())
        st2 = lib.tri_inv_ex(0, 0, n, a2.data_ptr(), n, code, p2, need, int(s2.cuda_stream),
                             d_info=info.data_ptr() + 8)
        assert st1 == lib.TRI_OK and st2 == lib.TRI_OK
        torch.cuda.synchronize()
        assert info.cpu().tolist() == [bad, -1], rep
    assert lib.tri_get_info() == (lib.TRI_OK, -1)        # nothing went to the device-wide word


def test_gen_inv_ex_and_batched_info(lib):
    n = 600
    a = inputs.general(n, seed=3, dtype=np.float32)
    a[0, 0] = 0.0
    da = torch.from_numpy(np.ascontiguousarray(a.T)).cuda()
    need = lib.gen_inv_workspace_size(n, lib.TRI_F32_MIXED)
    w, p = _ws(lib, need)
    info = torch.full((3,), 5, dtype=torch.int64, device="cuda")
    s = int(torch.cuda.current_stream().cuda_stream)
    assert lib.gen_inv_ex(n, da.data_ptr(), n, lib.TRI_F32_MIXED, p, need, s, d_info=info.data_ptr()) == lib.TRI_OK
    # strided batch of 4 lower matrices, matrix 2 singular: the matrix index is recorded
    m, b = 300, 4
    ts = [inputs.tri_lower(m, seed=40 + i, law="normal") for i in range(b)]
    ts[2][17, 17] = 0.0
    host = np.stack([np.ascontiguousarray(x.T) for x in ts]).astype(np.float32)
    db = torch.from_numpy(host).cuda()
    needb = lib.tri_inv_strided_batched_workspace_size(m, b, lib.TRI_F32)
    wb, pb = _ws(lib, needb)
    assert lib.tri_inv_strided_batched_ex(0, 0, m, db.data_ptr(), m, m * m, b, lib.TRI_F32, pb, needb, s,
                                          d_info=info.data_ptr() + 8) == lib.TRI_OK
    ok = torch.from_numpy(np.ascontiguousarray(inputs.general(n, seed=4, dtype=np.float32).T)).cuda()
    assert lib.gen_inv_ex(n, ok.data_ptr(), n, lib.TRI_F32, p, need, s, d_info=info.data_ptr() + 16) == lib.TRI_OK
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 2, -1]
    assert lib.tri_get_info() == (lib.TRI_OK, -1)
