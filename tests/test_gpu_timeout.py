"""Failure detection without a GPU fault: the single-launch tensor-core schedule of the
mixed path waits on ready counters with a bounded deadline.  With one counter withheld
(TRI_DEBUG_WITHHOLD, a flag that nothing sets) and a 50 ms deadline
(TRI_DEBUG_WAIT_LIMIT_US), the launch must end by itself, tri_get_info must report
TRI_ERR_TIMEOUT, and the context must stay usable: a tensor-core product and a plain
inverse run correctly afterwards in the same process."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, time
import numpy as np, torch
import oracle
from paper_2307_07611_gb300 import inputs, lib
lib.load()
n = 1024
t = inputs.tri_lower(n, seed=3, law="normal").astype(np.float32)
dev = torch.from_numpy(np.ascontiguousarray(t.T)).cuda()
s = int(torch.cuda.current_stream().cuda_stream)
t0 = time.time()
st = lib.tri_inv(lib.TRI_LOWER, lib.TRI_NONUNIT, n, dev.data_ptr(), n, lib.TRI_F32_MIXED, s)
info = lib.tri_get_info(s)
elapsed = time.time() - t0
# the same context afterwards: a tensor-core product (allocates tensor memory again)
a = torch.randn(256, 128, dtype=torch.float32).to(torch.bfloat16)
b = torch.randn(128, 256, dtype=torch.float32).to(torch.bfloat16)
ad = a.t().contiguous().cuda(); bd = b.t().contiguous().cuda()
c = torch.zeros(256, 256, dtype=torch.float32, device="cuda")
st_tc = lib.tri_tc_gemm_bf16(256, 256, 128, [ad.data_ptr()], 256, [bd.data_ptr()], 128, c.data_ptr(), 256, s)
torch.cuda.synchronize()
want = a.double() @ b.double()
tc_err = float((c.t().double().cpu() - want).abs().max() / want.abs().max())
# and a plain FP32 inverse
d2 = torch.from_numpy(np.ascontiguousarray(t.T)).cuda()
st2 = lib.tri_inv(lib.TRI_LOWER, lib.TRI_NONUNIT, n, d2.data_ptr(), n, lib.TRI_F32, s)
info2 = lib.tri_get_info(s)
x = np.tril(d2.cpu().numpy().T.astype(np.float64))
want_x = oracle.tri_inv(t.astype(np.float64))
err = float(np.abs(x - want_x).max() / np.abs(want_x).max())
print(json.dumps({"st": st, "info": info[0], "elapsed": elapsed, "st_tc": st_tc, "tc_err": tc_err,
                  "st2": st2, "info2": info2[0], "err": err}))
"""


def test_withheld_counter_times_out_and_context_survives():
    from paper_2307_07611_gb300 import lib
    env = dict(os.environ, TRI_MIXED_SCHEDULE="graph", TRI_DEBUG_WAIT_LIMIT_US="50000",
               # n = 1024: the ready counter of X region (rows 256..383, columns 0..255),
               # written by the first X21 tile of level h = 256 and read by level h = 512
               TRI_DEBUG_WITHHOLD="8", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["st"] == lib.TRI_OK                     # the launch itself is fine
    assert out["info"] == lib.TRI_ERR_TIMEOUT          # the bounded wait ran out
    assert out["elapsed"] < 10.0
    assert out["st_tc"] == lib.TRI_OK and out["tc_err"] < 1e-5
    assert out["st2"] == lib.TRI_OK and out["info2"] == lib.TRI_OK
    assert out["err"] < 40 * 32 * 2.0 ** -24
