"""Batched CG over lattices of uneven sizes (one persistent launch per phase): every system
must match its own single-lattice solve and the oracle's operator."""
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


def _setup(lq, ctx, dims_list, nrhs, inner, seed, eps=0.2):
    import torch
    out = []
    for i, dims in enumerate(dims_list):
        U = synth.gauge_field(dims, "near_identity", seed=seed + i, eps=eps)
        b = synth.fermion_field(dims, nrhs, seed=seed + 100 + i)
        Ud = torch.from_numpy(U).cuda()
        hi = lq.lq_gauge_pack(ctx, dims, Ud, "f64", 18)
        lo = lq.lq_gauge_pack(ctx, dims, Ud, inner, 12) if inner else None
        out.append((dims, U, b, hi, lo, torch.from_numpy(b).cuda()))
    return out


@pytest.mark.parametrize("inner", [None, "f32", "bf16"])
def test_batched_matches_single_and_oracle(lq, ctx, inner):
    import torch
    lats = _setup(lq, ctx, [(4, 4, 4, 4), (6, 6, 6, 6), (4, 4, 2, 8), (8, 8, 8, 8)], 3, inner, 101)
    masses = [0.1, 0.2, 0.15, 0.1]
    xs = [torch.empty_like(l[5]) for l in lats]
    st = lq.cg_solve_batched(ctx, [l[3] for l in lats], None if inner is None else [l[4] for l in lats],
                             masses, [l[5] for l in lats], xs, 3, tol=1e-10, maxiter=20000)
    for (dims, U, b, hi, lo, bd), x, m, s in zip(lats, xs, masses, st):
        xn = x.cpu().numpy()
        xs1 = torch.empty_like(bd)
        lq.cg_solve(ctx, hi, lo, m, bd, xs1, 3, tol=1e-10, maxiter=20000)
        for k in range(3):
            assert s[k]["true_rel_resid"] <= 1e-10
            r = b[k] - odslash.normal_op(U, xn[k], m, dims)
            assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1.05e-10
            assert rel_l2(xn[k], xs1[k].cpu().numpy()) < 1e-8


def test_batched_uneven_config_8_12_16_24(lq, ctx):
    """Lattices 8^4, 12^4, 16^4, 24^4, 8 right-hand sides each, links exp(i 0.2 H), FP32
    inner iteration, tol 1e-8; two sampled systems per lattice verified with the oracle."""
    import torch
    dims_list = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16), (24, 24, 24, 24)]
    lats = _setup(lq, ctx, dims_list, 8, "f32", 5)
    xs = [torch.empty_like(l[5]) for l in lats]
    st = lq.cg_solve_batched(ctx, [l[3] for l in lats], [l[4] for l in lats], [0.1] * 4,
                             [l[5] for l in lats], xs, 8, tol=1e-8, maxiter=20000)
    for (dims, U, b, hi, lo, bd), x, s in zip(lats, xs, st):
        assert all(si["true_rel_resid"] <= 1e-8 for si in s)
        xn = x.cpu().numpy()
        for k in (0, 7):
            r = b[k] - odslash.normal_op(U, xn[k], 0.1, dims)
            assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1.05e-8


def test_batched_rejects_mixed_formats(lq, ctx):
    import torch
    lats = _setup(lq, ctx, [(4, 4, 4, 4), (4, 4, 4, 6)], 1, "f32", 7)
    lo2 = lq.lq_gauge_pack(ctx, (4, 4, 4, 6), torch.from_numpy(lats[1][1]).cuda(), "bf16", 12)
    xs = [torch.empty_like(l[5]) for l in lats]
    with pytest.raises(lq.LQError, match="INVALID_ARG"):
        lq.cg_solve_batched(ctx, [l[3] for l in lats], [lats[0][4], lo2], [0.1, 0.1],
                            [l[5] for l in lats], xs, 1)


@pytest.mark.parametrize("shape", ["64,2,8", "128,2,8", "64,4,8"])
def test_batched_rhs_warp_shapes(lq, shape, monkeypatch):
    """The batched mixed solve with the multi-lattice rhs-per-warp kernel forced (its fused
    <p,Ap> and residual-norm reductions, the w1 epilogue and the skipping of converged
    systems), against the single-lattice solves and the oracle's operator."""
    import torch
    monkeypatch.setenv("LQCD_DSLASH_SHAPE", shape)
    ctx = lq.Context(0)
    lats = _setup(lq, ctx, [(4, 4, 4, 4), (6, 6, 6, 6), (4, 4, 2, 8), (8, 8, 8, 8)], 5, "f32", 111)
    masses = [0.1, 0.2, 0.15, 0.1]
    xs = [torch.empty_like(l[5]) for l in lats]
    st = lq.cg_solve_batched(ctx, [l[3] for l in lats], [l[4] for l in lats], masses, [l[5] for l in lats], xs, 5,
                             tol=1e-10, maxiter=20000)
    for (dims, U, b, hi, lo, bd), x, m, s in zip(lats, xs, masses, st):
        xn = x.cpu().numpy()
        for k in range(5):
            assert s[k]["true_rel_resid"] <= 1e-10
            r = b[k] - odslash.normal_op(U, xn[k], m, dims)
            assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1.05e-10
