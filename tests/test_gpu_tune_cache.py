"""A shared tuning cache (LQCD_TUNE_CACHE) makes solves reproducible across processes: the
second process loads the launch shapes the first one tuned, so every reduction sums in the
same order and the mixed-precision CG takes the same iterations to the same solution."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys, hashlib
sys.path.insert(0, %r)
import torch
import paper_1309_0551_gb300 as lq
import synth
ctx = lq.Context(0)
dims, mass = (8, 8, 8, 8), 0.01
U = torch.from_numpy(synth.gauge_field(dims, "haar", seed=4)).cuda()
b = torch.from_numpy(synth.fermion_field(dims, 2, seed=5)).cuda()
hi = lq.lq_gauge_pack(ctx, dims, U, "f64", 18)
lo = lq.lq_gauge_pack(ctx, dims, U, "bf16", 12)
x = torch.empty_like(b)
st = lq.cg_solve(ctx, hi, lo, mass, b, x, 2, tol=1e-10, maxiter=40000)
print(json.dumps({"iters": [s["iters"] for s in st],
                  "x": hashlib.sha256(x.cpu().numpy().tobytes()).hexdigest(),
                  "keys": ctx.tune_report().count("\n")}))
"""


def _run(cache):
    env = dict(os.environ, LQCD_TUNE_CACHE=str(cache))
    p = subprocess.run([sys.executable, "-c", SCRIPT % ROOT], env=env, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_two_processes_with_a_shared_cache_agree(tmp_path):
    cache = tmp_path / "tune.txt"
    first = _run(cache)
    assert cache.exists() and first["keys"] > 0
    lines = cache.read_text().splitlines()
    assert len(lines) == first["keys"] and all(l.count("\t") == 2 for l in lines)
    second = _run(cache)
    assert second["iters"] == first["iters"]
    assert second["x"] == first["x"]        # bitwise the same solution
