"""The debug build (library compiled with -DTRSGD_DEBUG): index checks of the
drawn slice indices and fiber columns.

Nothing here makes an access leave its buffer. The debug build must give
the product build's results bit for bit while every index is valid; the
reporting path is exercised by lowering the bound of the check on one core
(trsgd_debug_index_bound) below I_k, so that valid draws are reported as
violations: the next synchronising call returns TRSGD_EBADINDEX, and the
cores stay finite. Each debug run is a child process with TRSGD_DEBUG=1
(the library loader picks the debug build from the environment).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2303_16492_gb300 import _abi
from paper_2303_16492_gb300 import build as _build
from tests.gpu_helpers import cuda

pytestmark = [pytest.mark.gpu, cuda]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# cluster path: FP32 pieces on the tensor cores; whole-GPU path: BF16 operands
SHAPES = {
    "cluster": dict(dims=[30, 40, 50], ranks=[3, 4, 2], J=64, prec=_abi.FP32, path=_abi.PATH_CLUSTER, x=_abi.DTYPE_F32),
    "grid": dict(dims=[200, 70, 60], ranks=[8, 6, 5], J=300, prec=_abi.BF16_MIXED, path=_abi.PATH_GRID,
                 x=_abi.DTYPE_BF16),
}

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, {root!r})
from paper_2303_16492_gb300 import api, _abi
spec = json.loads({spec!r})
def problem():
    g = torch.Generator().manual_seed(11)
    d, r = spec["dims"], spec["ranks"]
    N = len(d)
    cores = [(torch.randn(d[k], r[k] * r[(k + 1) % N], generator=g) * 0.3).cuda() for k in range(N)]
    X = api.reconstruct([c.clone() for c in cores], d, r)
    X = X + 0.01 * torch.randn(X.shape, generator=g).cuda()
    if spec["x"] == _abi.DTYPE_BF16:
        X = X.to(torch.bfloat16)
    init = [(c + 0.05 * torch.randn(c.shape, generator=g).cuda()).contiguous() for c in cores]
    pc = api.ProblemConfig(dims=d, ranks=r, J=spec["J"], prec=spec["prec"], alpha=0.02, seed=7,
                           path=spec["path"], x_dtype=spec["x"])
    return pc, X, init
pc, X, init = problem()
s = api.Solver([pc], [X], [init])
s.run(0, 6)
torch.cuda.synchronize()
out = {{"cores": [c.cpu().numpy().tolist() for c in init]}}
if spec.get("bound_core") is not None:
    k = spec["bound_core"]
    s.debug_index_bound(k, max(1, spec["dims"][k] // 2))
    try:   # several modes: core k's indices are drawn whenever n != k; run synchronises
        s.run(6, 6)
        out["status"] = 0
    except _abi.TrsgdError as e:
        out["status"] = e.status
    torch.cuda.synchronize()
    out["finite"] = all(bool(torch.isfinite(c).all()) for c in init)
s.close()
print("RESULT " + json.dumps(out))
"""


def _child(spec, debug):
    env = dict(os.environ)
    if debug:
        env["TRSGD_DEBUG"] = "1"
    else:
        env.pop("TRSGD_DEBUG", None)
    code = CHILD.format(root=ROOT, spec=json.dumps(spec))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


@pytest.fixture(scope="module")
def debug_lib():
    return _build.build(debug=True)


@pytest.mark.parametrize("path", sorted(SHAPES))
def test_debug_build_matches_product_build(debug_lib, path):
    spec = dict(SHAPES[path])
    prod = _child(spec, debug=False)
    dbg = _child(spec, debug=True)
    for a, b in zip(prod["cores"], dbg["cores"]):
        np.testing.assert_array_equal(np.asarray(a), np.asarray(b))


@pytest.mark.parametrize("path", sorted(SHAPES))
def test_debug_build_reports_out_of_range_indices(debug_lib, path):
    spec = dict(SHAPES[path], bound_core=1)
    out = _child(spec, debug=True)
    assert out["status"] == _abi.EBADINDEX
    assert out["finite"]


def test_product_build_has_no_checks():
    spec = dict(SHAPES["cluster"], bound_core=1)
    env = dict(os.environ)
    env.pop("TRSGD_DEBUG", None)
    code = CHILD.format(root=ROOT, spec=json.dumps(spec))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode != 0 and "unsupported configuration" in r.stderr
