"""The debug build's device-side index checks (-DIDW_DEBUG_CHECKS).

compute-sanitizer is not available here, so the kernels of the local and
k-NN forms carry their own bounds checks in a debug build: a failed check
records its site in a device word and skips the access.  A child process
loads the debug library (IDW_DEBUG_CHECKS=1), runs both forms over inputs
chosen to stress the index arithmetic, checks parity with the oracle, and
reads the word, which must stay zero.  The release library refuses the
query (its checks are compiled out).
"""
import json
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes, json
import numpy as np
import torch
import oracle, synthetic
import paper_1402_4986_gb300 as idw
from paper_1402_4986_gb300 import _lib

def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()

rng = np.random.default_rng(81)
cases = []
u = synthetic.uniform_problem(3001, 1500, seed=82, exact_hits=5)
cases.append(("uniform", u["data"], u["queries"]))
c = synthetic.config_local(seed=83, n=8000, m=1500, clustered=True)
cases.append(("clustered", c["data"], c["queries"]))
line = u["data"].copy(); line[:, 0] = 0.25
cases.append(("line", line, u["queries"]))
far = np.concatenate([u["queries"], [[-5, 0.5], [0.5, 9], [1e6, -1e6], [np.nan, 0.1]]]).astype(np.float32)
nf = u["data"].copy(); nf[::7, 1] = np.inf
cases.append(("far and non-finite", nf, far))
cases.append(("n < k", u["data"][:5], u["queries"][:300]))
worst = 0.0
for name, data, q in cases:
    d, qq = dev(data), dev(q)
    Z, cnt = idw.interpolate_local(d, qq, 2.0, 0.03, counts=True)
    Zo, _, co = oracle.idw_local(data, q, 2.0, 0.03)
    assert np.array_equal(cnt.cpu().numpy(), co), name
    _, cm = idw.interpolate_modified(d, qq, 2.0, 0.03, counts=True)
    assert np.array_equal(cm.cpu().numpy(), co), name
    ho = idw.Handle(torch.cuda.current_device())  # the caller's query order
    idw.set_option("local_query_order", 1, handle=ho)
    _, cnt_o = idw.interpolate_local(d, qq, 2.0, 0.03, counts=True, handle=ho)
    assert np.array_equal(cnt_o.cpu().numpy(), co), name
    _, nbr_o = idw.interpolate_knn(d, qq, 2.0, 9, neighbours=True, handle=ho)
    assert np.array_equal(nbr_o.cpu().numpy(), oracle.idw_knn(data, q, 2.0, 9)["nbr"]), name
    ho.close()
    gl = torch.linspace(-1.0, 1.0, q.shape[0], device="cuda")
    gzl = idw.local_backward(d, qq, 2.0, 0.03, gl)[0].cpu().numpy()
    Gl = oracle.idw_local_grad(data, q, 2.0, 0.03, gl.cpu().numpy())["grad_z"]
    assert np.max(np.abs(gzl - Gl)) <= 1e-4 * max(np.max(np.abs(Gl)), 1e-30), name
    _, cnt_ix = idw.LocalIndex(d, radius=0.03).interpolate(qq, 2.0, 0.02, counts=True)
    assert np.array_equal(cnt_ix.cpu().numpy(), oracle.idw_local(data, q, 2.0, 0.02)[2]), name
    gzk = idw.knn_backward(d, qq, 2.0, 9, gl)[0].cpu().numpy()
    Gk = oracle.idw_knn_grad(data, q, 2.0, 9, gl.cpu().numpy())["grad_z"]
    assert np.max(np.abs(gzk - Gk)) <= 1e-4 * max(np.max(np.abs(Gk)), 1e-30), name
    kix = idw.LocalIndex(d, k=9)
    for k in (1, 9, 33):
        Zk, nbr = idw.interpolate_knn(d, qq, 2.0, k, neighbours=True)
        r = oracle.idw_knn(data, q, 2.0, k)
        assert np.array_equal(nbr.cpu().numpy(), r["nbr"]), (name, k)
        _, nbr_ix = kix.knn(qq, 2.0, k, neighbours=True)
        assert np.array_equal(nbr_ix.cpu().numpy(), r["nbr"]), (name, k, "index")
        ok = ~np.isnan(r["Z"])
        if ok.any():
            worst = max(worst, float(np.max(np.abs(Zk.cpu().numpy()[ok] - r["Z"][ok]))))
torch.cuda.synchronize()
sites = ctypes.c_uint32(0)
st = _lib.load().idw_debug_check_failures(torch.cuda.current_device(), ctypes.byref(sites))
print(json.dumps({"status": st, "sites": sites.value, "worst": worst,
                  "lib": _lib.library_path()}))
"""


@pytest.fixture(scope="module")
def idw():
    from paper_1402_4986_gb300 import build
    build.build()
    build.build(debug=True)
    import paper_1402_4986_gb300 as m
    return m


def test_release_build_has_no_checks(idw):
    import ctypes
    from paper_1402_4986_gb300 import _lib
    sites = ctypes.c_uint32(123)
    st = _lib.load().idw_debug_check_failures(torch.cuda.current_device(), ctypes.byref(sites))
    assert st == 6 and sites.value == 0  # IDW_ERR_UNSUPPORTED


def test_debug_build_index_checks_stay_clean(idw):
    env = dict(os.environ, IDW_DEBUG_CHECKS="1")
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    out = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    assert res["lib"].endswith("_debug.so")
    assert res["status"] == 0, res
    assert res["sites"] == 0, f"index checks failed at sites {res['sites']:#x}"
    assert res["worst"] <= 1e-5
