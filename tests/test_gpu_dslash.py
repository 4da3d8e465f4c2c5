"""Parity of the CUDA half Dslash (dslash_eo) with the FP64 oracle, every storage format,
both parities, ragged and degenerate lattices, several right-hand-side counts."""
import numpy as np
import pytest

import synth
from oracle import dslash as odslash
from oracle.precision import quantize_links
from helpers import rel_l2, to_device_vec, from_device_vec, empty_vec, store_tolerance

pytestmark = pytest.mark.gpu

FORMATS = [("f64", 18, "f64"), ("f64", 12, "f64"),
           ("f32", 18, "f32"), ("f32", 12, "f32"), ("f32", 18, "bf16"),
           ("bf16", 18, "f32"), ("bf16", 12, "bf16"), ("bf16", 12, "f32"),
           ("f16", 18, "f16"), ("f16", 12, "f32")]


@pytest.fixture(scope="module")
def lq():
    import paper_1309_0551_gb300 as lq
    return lq


@pytest.fixture(scope="module")
def ctx(lq):
    return lq.Context(0)


def _run(lq, ctx, U, dims, gp, recon, vp, chi, parity):
    import torch
    g = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), gp, recon)
    cd = to_device_vec(chi, vp)
    out = empty_vec(chi.shape, vp)
    lq.dslash_eo(ctx, g, cd, out, parity, chi.shape[0])
    torch.cuda.synchronize()
    return from_device_vec(out), from_device_vec(cd)


@pytest.mark.parametrize("gp,recon,vp", FORMATS)
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 10), (2, 2, 2, 2)])
@pytest.mark.parametrize("parity", [0, 1])
def test_dslash_matches_oracle(lq, ctx, gp, recon, vp, dims, parity):
    U = synth.gauge_field(dims, "haar", seed=61)
    chi = synth.fermion_field(dims, 1, seed=62 + parity)
    got, chi_q = _run(lq, ctx, U, dims, gp, recon, vp, chi, parity)
    ref = odslash.dslash_eo_multi(quantize_links(U, gp, recon), chi_q, dims, parity)
    assert rel_l2(got, ref) < store_tolerance(vp)
    exact = odslash.dslash_eo_multi(U, chi, dims, parity)
    if gp in ("f64", "f32") and vp == gp:
        # against the unrounded FP64 operator: 1e-13 (FP64) and 1e-5 (FP32)
        assert rel_l2(got, exact) < (1e-13 if gp == "f64" else 1e-5)
    else:
        # the error the storage formats cost against the unrounded FP64 operator: each link
        # and input element rounded once (the 12-real third row rebuilt from rounded rows),
        # the output rounded once
        u = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}
        assert rel_l2(got, exact) < 8 * (u[gp] + u[vp])


@pytest.mark.parametrize("gp,recon,vp", [("f64", 18, "f64"), ("f32", 12, "f32"), ("bf16", 18, "bf16")])
@pytest.mark.parametrize("nrhs", [3, 16])
def test_multi_rhs_equals_single(lq, ctx, gp, recon, vp, nrhs):
    dims = (4, 4, 6, 4)
    U = synth.gauge_field(dims, "near_identity", seed=63, eps=0.2)
    chi = synth.fermion_field(dims, nrhs, seed=64)
    got, chi_q = _run(lq, ctx, U, dims, gp, recon, vp, chi, 0)
    ref = odslash.dslash_eo_multi(quantize_links(U, gp, recon), chi_q, dims, 0)
    for k in range(nrhs):
        assert rel_l2(got[k], ref[k]) < store_tolerance(vp)
        one, _ = _run(lq, ctx, U, dims, gp, recon, vp, chi[k:k + 1], 0)
        # the single-rhs launch may pick another launch shape (summation order): equal to
        # within the accumulation rounding
        assert rel_l2(got[k], one[0]) < store_tolerance(vp)


@pytest.mark.parametrize("gp,recon,vp", [("f64", 18, "f64"), ("f32", 18, "f32"), ("f32", 12, "f32"),
                                         ("bf16", 12, "bf16"), ("bf16", 18, "f32")])
def test_full_size_16c32_sampled(lq, ctx, gp, recon, vp):
    """The 16^3 x 32 near-identity (eps 0.3) workload of the throughput benchmark, checked
    on 400 sampled output sites per parity with the site-by-site oracle."""
    dims = (16, 16, 16, 32)
    U = synth.gauge_field(dims, "near_identity", seed=3, eps=0.3)
    Uq = quantize_links(U, gp, recon)
    rs = synth.rng(65)
    for parity in (0, 1):
        chi = synth.fermion_field(dims, 1, seed=66 + parity)
        got, chi_q = _run(lq, ctx, U, dims, gp, recon, vp, chi, parity)
        sites = np.sort(rs.choice(chi.shape[1], 400, replace=False))
        sites[-1] = chi.shape[1] - 1
        ref = odslash.dslash_eo_sites(Uq, chi_q[0], dims, parity, sites)
        assert rel_l2(got[0][sites], ref) < store_tolerance(vp)


@pytest.fixture(scope="module")
def field_32c4():
    return synth.gauge_field((32, 32, 32, 32), "near_identity", seed=3, eps=0.3)


@pytest.mark.parametrize("gp,recon", [("f32", 18), ("f32", 12)])
def test_full_size_32c4_sampled(lq, ctx, field_32c4, gp, recon):
    """The 32^4 near-identity (eps 0.3) lines of the benchmark (every launch reads its
    links from HBM), checked on 200 sampled output sites per parity, the last site
    included."""
    dims = (32, 32, 32, 32)
    U = field_32c4
    Uq = quantize_links(U, gp, recon)
    rs = synth.rng(68)
    for parity in (0, 1):
        chi = synth.fermion_field(dims, 1, seed=69 + parity)
        got, chi_q = _run(lq, ctx, U, dims, gp, recon, "f32", chi, parity)
        sites = np.sort(rs.choice(chi.shape[1], 200, replace=False))
        sites[-1] = chi.shape[1] - 1
        ref = odslash.dslash_eo_sites(Uq, chi_q[0], dims, parity, sites)
        assert rel_l2(got[0][sites], ref) < store_tolerance("f32")


def test_invalid_arguments(lq, ctx):
    import torch
    dims = (4, 4, 4, 4)
    U = torch.from_numpy(synth.gauge_field(dims, "unit")).cuda()
    with pytest.raises(lq.LQError, match="INVALID_ARG"):
        lq.lq_gauge_pack(ctx, (4, 4, 3, 4), U, "f32", 18)
    g = lq.lq_gauge_pack(ctx, dims, U, "f32", 18)
    v = empty_vec((17, 128, 3), "f32")
    with pytest.raises(lq.LQError, match="INVALID_ARG"):
        lq.dslash_eo(ctx, g, v, v, 0, 17)
    a = empty_vec((1, 128, 3), "f32")
    with pytest.raises(lq.LQError, match="INVALID_ARG"):
        lq.dslash_eo(ctx, g, a, a, 0, 1)           # in and out overlap
    with pytest.raises(lq.LQError, match="INVALID_ARG"):
        lq.dslash_eo(ctx, g, a, empty_vec((1, 128, 3), "f64"), 0, 1, vec_prec=lq.LQ_F64)


@pytest.mark.parametrize("gp,recon,vp", [("f64", 18, "f64"), ("f32", 12, "f32"), ("bf16", 18, "f32"),
                                         ("f16", 12, "f32")])
@pytest.mark.parametrize("nrhs", [1, 5, 8])
def test_dslash_multi_matches_single(lq, ctx, gp, recon, vp, nrhs):
    import torch
    dims_list = [(4, 4, 4, 4), (6, 4, 2, 10), (8, 8, 8, 8), (2, 2, 2, 2)]
    Us, ins, outs, refs = [], [], [], []
    for i, dims in enumerate(dims_list):
        U = synth.gauge_field(dims, "haar", seed=140 + i)
        chi = synth.fermion_field(dims, nrhs, seed=150 + i)
        g = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), gp, recon)
        cd = to_device_vec(chi, vp)
        Us.append(g)
        ins.append(cd)
        outs.append(empty_vec(chi.shape, vp))
        refs.append(odslash.dslash_eo_multi(quantize_links(U, gp, recon), from_device_vec(cd), dims, 1))
    lq.dslash_eo_multi(ctx, Us, ins, outs, 1, nrhs)
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert rel_l2(from_device_vec(o), r) < store_tolerance(vp)


@pytest.mark.parametrize("gp,recon", [("f32", 12), ("f32", 18), ("bf16", 12), ("f16", 18)])
@pytest.mark.parametrize("block,tile", [(64, 2), (128, 4), (256, 8), (256, 16), (128, 8), (64, 4), (64, 8),
                                        (128, 16)])
@pytest.mark.parametrize("nrhs", [3, 8, 13])
def test_rhs_warp_kernel(lq, gp, recon, block, tile, nrhs, monkeypatch):
    """The multi-RHS kernel with the right-hand sides spread over warps (block = 32 sites x
    block/32 warps, tile/(block/32) rhs per thread, tps 8), forced through the shape
    override, on a lattice whose half volume (240) is not a multiple of 32 and rhs counts
    that leave a partial tile."""
    import torch
    monkeypatch.setenv("LQCD_DSLASH_SHAPE", f"{block},{tile},8")
    ctx = lq.Context(0)
    dims = (6, 4, 2, 10)
    U = synth.gauge_field(dims, "haar", seed=66)
    g = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), gp, recon)
    Uq = quantize_links(U, gp, recon)
    for parity in (0, 1):
        chi = synth.fermion_field(dims, nrhs, seed=67 + parity)
        d = to_device_vec(chi, "f32")
        out = empty_vec(chi.shape, "f32")
        lq.dslash_eo(ctx, g, d, out, parity, nrhs)
        torch.cuda.synchronize()
        ref = odslash.dslash_eo_multi(Uq, from_device_vec(d), dims, parity)
        got = from_device_vec(out)
        for k in range(nrhs):
            assert rel_l2(got[k], ref[k]) < store_tolerance("f32")
    if tile <= nrhs:
        assert ctx.tune_report() == ""      # the forced shape was taken: nothing was tuned


@pytest.mark.parametrize("gp,recon", [("f32", 12), ("bf16", 18)])
@pytest.mark.parametrize("block,tile", [(64, 2), (128, 8), (256, 8), (64, 8)])
@pytest.mark.parametrize("nrhs", [3, 8])
def test_multi_rhs_warp_kernel(lq, gp, recon, block, tile, nrhs, monkeypatch):
    """The multi-lattice rhs-per-warp kernel, forced through the shape override, on four
    lattices of different sizes (half volumes 128, 240, 2048 and 8: partial 32-site blocks
    and a lattice smaller than one block)."""
    import torch
    monkeypatch.setenv("LQCD_DSLASH_SHAPE", f"{block},{tile},8")
    ctx = lq.Context(0)
    dims_list = [(4, 4, 4, 4), (6, 4, 2, 10), (8, 8, 8, 8), (2, 2, 2, 2)]
    Us, ins, outs, refs = [], [], [], []
    for i, dims in enumerate(dims_list):
        U = synth.gauge_field(dims, "haar", seed=160 + i)
        chi = synth.fermion_field(dims, nrhs, seed=170 + i)
        Us.append(lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), gp, recon))
        ins.append(to_device_vec(chi, "f32"))
        outs.append(empty_vec(chi.shape, "f32"))
        refs.append(odslash.dslash_eo_multi(quantize_links(U, gp, recon), from_device_vec(ins[-1]), dims, 0))
    lq.dslash_eo_multi(ctx, Us, ins, outs, 0, nrhs)
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert rel_l2(from_device_vec(o), r) < store_tolerance("f32")
    if tile <= nrhs:
        assert ctx.tune_report() == ""      # the forced shape was taken: nothing was tuned
