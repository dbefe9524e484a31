"""The bounds-checked build on the device: its probe catches an index
outside its range without touching memory (and the context stays usable),
and screens on every path (single target: Gram and direct; 16 targets:
multi-target Gram and the tensor-core kernel; FP64; a batched screen) run
through the checks without a violation and with the same lists, scores and
counts as the normal build.  Runs in a child process that loads
libdse_checked.so."""
import json
import os
import subprocess
import sys

import pytest

import __graft_entry__ as ge

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
import torch
from paper_2602_06986_gb300 import dse, workloads as W
assert dse.LIB_PATH.endswith("libdse_checked.so")
out = {"probe_in": dse.bounds_probe(2, 3), "probe_out": dse.bounds_probe(3, 3), "probe_neg": dse.bounds_probe(-1, 3)}
def run(w, Y, **kw):
    sp = dse.Space(torch.from_numpy(w["X"]).cuda(), w["units"], w["op_mask"], w["max_rung"],
                   unit_check_addsub=w["unit_check_addsub"], explog_dimensionless=w["explog_dimensionless"])
    r = sp.screen(torch.from_numpy(np.ascontiguousarray(Y)).cuda(), 100, **kw)
    lists = [[int(i) for i in r.fetch(l)[0]] + [float(s) for s in r.fetch(l)[1]] for l in range(r.n_lists)]
    st = r.stats()
    r.free(); sp.free()
    return {"lists": lists, "reasons": st["reasons"], "path": st["binary_path"]}
w = W.medium(1)
out["medium_gram"] = run(w, w["Y"])
out["medium_direct"] = run(w, w["Y"], flags=dse.FLAG_DIRECT)
out["medium_fp64"] = run(w, w["Y"], precision=dse.PREC_FP64)
wl = W.large(0, n_targets=16)
wl = dict(wl, X=np.ascontiguousarray(wl["X"][:, :700]))
Yl = np.ascontiguousarray(wl["Y"][:, :700])
out["large_gmt"] = run(wl, Yl, precision=dse.PREC_AUTO)
out["large_tc"] = run(wl, Yl, precision=dse.PREC_AUTO, flags=dse.FLAG_DIRECT)
print("RESULT" + json.dumps(out))
'''


def _run(variant):
    env = dict(os.environ)
    if variant:
        env["DSE_LIB_VARIANT"] = variant
    else:
        env.pop("DSE_LIB_VARIANT", None)
    code = CHILD if variant else CHILD.replace('assert dse.LIB_PATH.endswith("libdse_checked.so")', "")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT")][-1]
    return json.loads(line[len("RESULT"):])


def test_checked_build_on_device():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ge.build()
    from paper_2602_06986_gb300 import _build, dse

    _build.build(checked=True)
    chk = _run("checked")
    assert chk["probe_in"] == dse.OK
    assert chk["probe_out"] == dse.EBOUNDS and chk["probe_neg"] == dse.EBOUNDS
    ref = _run(None)
    assert ref["probe_in"] == dse.EINVAL  # (normal build: no checks)
    for key in ("medium_gram", "medium_direct", "medium_fp64", "large_gmt", "large_tc"):
        assert chk[key] == ref[key], key
    assert chk["medium_gram"]["path"] == dse.PATH_GRAM and chk["large_gmt"]["path"] == dse.PATH_GRAM_MT
    assert chk["large_tc"]["path"] == dse.PATH_TENSOR
