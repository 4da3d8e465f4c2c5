"""CG on M = m^2 - D_eo D_oe: FP64 and mixed precision against the oracle (dense solve,
FP64 CG, true residual with the oracle's operator), several right-hand sides, failure
statuses."""
import numpy as np
import pytest

import synth
from oracle import cg as ocg, dslash as odslash
from helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    import paper_1309_0551_gb300 as lq
    return lq


@pytest.fixture(scope="module")
def ctx(lq):
    return lq.Context(0)


def _gauges(lq, ctx, U, dims, lo=None, recon=12):
    import torch
    Ud = torch.from_numpy(U).cuda()
    hi = lq.lq_gauge_pack(ctx, dims, Ud, "f64", 18)
    low = lq.lq_gauge_pack(ctx, dims, Ud, lo, recon) if lo else None
    return hi, low


def _true_resid(U, b, x, mass, dims):
    r = b - odslash.normal_op(U, x, mass, dims)
    return np.linalg.norm(r) / np.linalg.norm(b)


@pytest.mark.parametrize("inner", [None, "f32", "bf16", "f16"])
def test_cg_4444_against_dense_solve(lq, ctx, inner):
    import torch
    dims, mass = (4, 4, 4, 4), 0.1
    U = synth.gauge_field(dims, "haar", seed=81)
    b = synth.fermion_field(dims, 1, seed=82)
    hi, lo = _gauges(lq, ctx, U, dims, inner)
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    st = lq.cg_solve(ctx, hi, lo, mass, bd, xd, 1, tol=1e-10, maxiter=5000)
    x = xd.cpu().numpy()
    M = odslash.dense_normal(U, mass, dims)
    ref = np.linalg.solve(M, b[0].reshape(-1)).reshape(b[0].shape)
    assert _true_resid(U, b[0], x[0], mass, dims) <= 1e-10
    assert st[0]["true_rel_resid"] <= 1e-10
    assert rel_l2(x[0], ref) < 1e-10 * np.linalg.cond(M)
    if inner:
        assert st[0]["reliable_updates"] >= 1


@pytest.mark.parametrize("inner", [None, "f32"])
def test_cg_multi_rhs_ragged(lq, ctx, inner):
    import torch
    dims, mass = (6, 4, 4, 6), 0.2
    U = synth.gauge_field(dims, "near_identity", seed=83, eps=0.5)
    b = synth.fermion_field(dims, 3, seed=84)
    hi, lo = _gauges(lq, ctx, U, dims, inner, 18)
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    st = lq.cg_solve(ctx, hi, lo, mass, bd, xd, 3, tol=1e-10, maxiter=5000)
    x = xd.cpu().numpy()
    for k in range(3):
        assert _true_resid(U, b[k], x[k], mass, dims) <= 1e-10
        ref, _ = ocg.cg(U, b[k], mass, dims, tol=1e-12)
        assert rel_l2(x[k], ref) < 1e-8
        assert st[k]["iters"] > 0


@pytest.mark.parametrize("shape,nrhs", [("128,4,8", 5), ("128,8,8", 16), ("64,4,8", 3)])
def test_cg_multi_rhs_warp_shapes(lq, shape, nrhs, monkeypatch):
    """Mixed FP32 solves of several right-hand sides with the rhs-per-warp Dslash forced for
    the plain D_oe launches (the fused D_eo launch is tuned): every system reaches the
    FP64 true residual, checked with the oracle's operator."""
    import torch
    monkeypatch.setenv("LQCD_DSLASH_SHAPE", shape)
    monkeypatch.setenv("LQCD_CG_PAIRED", "0")   # the canonical layout's kernels
    ctx = lq.Context(0)
    dims, mass = (6, 4, 4, 6), 0.2
    U = synth.gauge_field(dims, "near_identity", seed=85, eps=0.5)
    b = synth.fermion_field(dims, nrhs, seed=86)
    hi, lo = _gauges(lq, ctx, U, dims, "f32", 12)
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    st = lq.cg_solve(ctx, hi, lo, mass, bd, xd, nrhs, tol=1e-10, maxiter=5000)
    x = xd.cpu().numpy()
    for k in range(nrhs):
        assert st[k]["true_rel_resid"] <= 1e-10
        assert _true_resid(U, b[k], x[k], mass, dims) <= 1.05e-10


@pytest.mark.parametrize("lo,recon,nrhs,shape", [("f32", 12, 2, None), ("f32", 12, 3, None), ("bf16", 12, 8, None),
                                                 ("f16", 18, 5, None), ("f32", 18, 8, "64,1,32"),
                                                 ("f32", 12, 7, "128,2,32"), ("bf16", 18, 4, "256,4,32")])
def test_cg_multi_rhs_paired_layout(lq, monkeypatch, lo, recon, nrhs, shape):
    """Mixed solves of several right-hand sides iterate on the paired colour-planar layout
    (odd counts pad the last pair; one source is zero and is solved at once): every system
    reaches the FP64 true residual with the oracle's operator, and the solutions agree with
    the canonical layout's solve of the same systems."""
    import torch
    if shape:
        monkeypatch.setenv("LQCD_DSLASH_SHAPE", shape)
    dims, mass = (6, 4, 4, 6), 0.2
    U = synth.gauge_field(dims, "near_identity", seed=87, eps=0.5)
    b = synth.fermion_field(dims, nrhs, seed=88)
    b[nrhs // 2] = 0.0
    xs = {}
    for layout in ("1", "0"):
        monkeypatch.setenv("LQCD_CG_PAIRED", layout)
        ctx = lq.Context(0)
        hi, low = _gauges(lq, ctx, U, dims, lo, recon)
        bd = torch.from_numpy(b).cuda()
        xd = torch.empty_like(bd)
        st = lq.cg_solve(ctx, hi, low, mass, bd, xd, nrhs, tol=1e-10, maxiter=5000)
        xs[layout] = xd.cpu().numpy()
        for k in range(nrhs):
            if k == nrhs // 2:
                assert np.count_nonzero(xs[layout][k]) == 0
                continue
            assert st[k]["true_rel_resid"] <= 1e-10
            assert _true_resid(U, b[k], xs[layout][k], mass, dims) <= 1.05e-10
    # both solutions meet a 1e-10 true residual: they agree to within cond(M) * 2e-10
    # (cond(M) ~ 400 here), far below anything a layout error would give
    for k in range(nrhs):
        if k != nrhs // 2:
            assert rel_l2(xs["1"][k], xs["0"][k]) < 1e-7


def test_cg_zero_source_and_failures(lq, ctx):
    import torch
    dims, mass = (4, 4, 4, 4), 0.1
    U = synth.gauge_field(dims, "haar", seed=85)
    hi, lo = _gauges(lq, ctx, U, dims, "f32")
    b = synth.fermion_field(dims, 2, seed=86)
    b[1] = 0.0
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    st = lq.cg_solve(ctx, hi, None, mass, bd, xd, 2, tol=1e-10)
    assert np.all(xd[1].cpu().numpy() == 0) and st[1]["true_rel_resid"] == 0.0
    with pytest.raises(lq.LQError, match="NOT_CONVERGED") as ei:
        lq.cg_solve(ctx, hi, lo, mass, bd, xd, 1, tol=1e-10, maxiter=5, check_every=5)
    assert ei.value.stats[0]["iters"] == 5 and ei.value.stats[0]["true_rel_resid"] > 1e-10
    bad = bd.clone()
    bad[0, 3, 1] = float("nan")
    with pytest.raises(lq.LQError, match="NUMERIC"):
        lq.cg_solve(ctx, hi, lo, mass, bad, xd, 1, tol=1e-10)
    with pytest.raises(lq.LQError, match="INVALID_ARG"):
        lq.cg_solve(ctx, lo, None, mass, bd, xd, 1)   # U_hi must be FP64


@pytest.fixture(scope="module")
def field_32c4():
    dims = (32, 32, 32, 32)
    return synth.gauge_field(dims, "haar", seed=4), synth.fermion_field(dims, 1, seed=5)


@pytest.fixture(scope="module")
def x64_32c4(lq, ctx, field_32c4):
    """The FP64 solution of the 32^4 system (the reference of the mixed solves' x error)."""
    import torch
    dims, mass = (32, 32, 32, 32), 0.01
    U, b = field_32c4
    hi, _ = _gauges(lq, ctx, U, dims)
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    st = lq.cg_solve(ctx, hi, None, mass, bd, xd, 1, tol=1e-10, maxiter=40000)
    return xd[0].cpu().numpy(), st[0]


@pytest.mark.parametrize("inner", [None, "f16", "f32", "bf16"])
def test_cg_32c4_haar_m001(lq, ctx, inner, field_32c4, x64_32c4):
    """The 32^4 Haar, m = 0.01 solve to 1e-10, verified with one application of the
    oracle's FP64 operator to the GPU solution; a mixed solution is also compared with the
    FP64 one (both solve the same system to 1e-10, so they differ by at most about
    cond(M) * 1e-10; the measured gap is far smaller)."""
    import torch
    dims, mass = (32, 32, 32, 32), 0.01
    U, b = field_32c4
    hi, lo = _gauges(lq, ctx, U, dims, inner)
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    st = lq.cg_solve(ctx, hi, lo, mass, bd, xd, 1, tol=1e-10, maxiter=40000)
    assert st[0]["true_rel_resid"] <= 1e-10
    x = xd[0].cpu().numpy()
    assert _true_resid(U, b[0], x, mass, dims) <= 1.05e-10
    x64, _ = x64_32c4
    assert rel_l2(x, x64) < 1e-5


def test_cg_bf16_inner_haar_m001_against_dense_solve(lq, ctx):
    """BF16 links at m = 0.01 on Haar links (the rounded operator differs from the FP64 one
    by far more than m^2): the mixed solve still reaches the FP64 true residual, and its
    solution matches the dense solve (the oracle pin of this case)."""
    import torch
    dims, mass = (4, 4, 4, 4), 0.01
    U = synth.gauge_field(dims, "haar", seed=4)
    b = synth.fermion_field(dims, 1, seed=5)
    hi, lo = _gauges(lq, ctx, U, dims, "bf16")
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    st = lq.cg_solve(ctx, hi, lo, mass, bd, xd, 1, tol=1e-10, maxiter=20000)
    x = xd[0].cpu().numpy()
    M = odslash.dense_normal(U, mass, dims)
    ref = np.linalg.solve(M, b[0].reshape(-1)).reshape(b[0].shape)
    assert st[0]["true_rel_resid"] <= 1e-10
    assert _true_resid(U, b[0], x, mass, dims) <= 1.05e-10
    assert rel_l2(x, ref) < 1e-10 * np.linalg.cond(M)


def test_cg_bf16_inner_near_identity(lq, ctx):
    """BF16 links (8 significant bits) carry the inner iteration of a well-conditioned
    system too (16^4, links near identity, m = 0.1)."""
    import torch
    dims, mass = (16, 16, 16, 16), 0.1
    U = synth.gauge_field(dims, "near_identity", seed=87, eps=0.2)
    b = synth.fermion_field(dims, 1, seed=88)
    hi, lo = _gauges(lq, ctx, U, dims, "bf16")
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    st = lq.cg_solve(ctx, hi, lo, mass, bd, xd, 1, tol=1e-10, maxiter=20000)
    assert st[0]["true_rel_resid"] <= 1e-10
    assert _true_resid(U, b[0], xd[0].cpu().numpy(), mass, dims) <= 1.05e-10
