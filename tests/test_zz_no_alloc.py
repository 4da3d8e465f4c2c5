"""cg_solve_noalloc: the solver for callers that cannot allocate GPU memory when they solve
(a host framework or plugin that forbids cudaMalloc/cudaFree on its threads, or a loop
under a fixed memory budget).  It must give what cg_solve gives, call after call, although
its scratch lives in one fixed device array that every call reuses.

This file is named to be collected last: if it fails, a run stopping at the first failure
has already run every other test.
"""
import numpy as np
import pytest

import synth
from oracle import dslash as odslash
from helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    import paper_1309_0551_gb300 as lq
    return lq


@pytest.fixture(scope="module")
def ctx(lq):
    return lq.Context(0)


@pytest.mark.parametrize("inner", [None, "f32"])
def test_noalloc_matches_cg_solve_on_consecutive_calls(lq, ctx, inner):
    import torch
    dims, mass, nrhs = (8, 8, 8, 8), 0.1, 2
    U = synth.gauge_field(dims, "haar", seed=91)
    b = synth.fermion_field(dims, nrhs, seed=92)
    Ud = torch.from_numpy(U).cuda()
    hi = lq.lq_gauge_pack(ctx, dims, Ud, "f64", 18)
    lo = lq.lq_gauge_pack(ctx, dims, Ud, inner, 12) if inner else None
    bd = torch.from_numpy(b).cuda()
    x_ref = torch.empty_like(bd)
    lq.cg_solve(ctx, hi, lo, mass, bd, x_ref, nrhs, tol=1e-10)
    ref = x_ref.cpu().numpy()
    for call in range(2):
        x = torch.full_like(bd, float("nan"))   # the entry point must overwrite all of x
        st = lq.cg_solve_noalloc(ctx, hi, lo, mass, bd, x, nrhs, tol=1e-10)
        got = x.cpu().numpy()
        for k in range(nrhs):
            assert st[k]["true_rel_resid"] <= 1e-10, (call, k, st[k])
            assert rel_l2(got[k], ref[k]) < 1e-8, (call, k)
            r = b[k] - odslash.normal_op(U, got[k], mass, dims)
            assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1.05e-10


def test_noalloc_rejects_problems_beyond_its_array(lq, ctx):
    import torch
    dims = (32, 32, 32, 16)   # 262144 sites per parity: far beyond the fixed scratch
    Ud = torch.from_numpy(synth.gauge_field(dims, "unit")).cuda()
    hi = lq.lq_gauge_pack(ctx, dims, Ud, "f64", 18)
    b = torch.ones((1, synth.volume(dims) // 2, 3), dtype=torch.complex128, device="cuda")
    x = torch.empty_like(b)
    with pytest.raises(lq.LQError, match="INVALID_ARG.*scratch"):
        lq.cg_solve_noalloc(ctx, hi, None, 0.1, b, x, 1)
