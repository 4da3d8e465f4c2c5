"""The paired colour-planar FP32 layout (lq_vec_pair / lq_vec_unpair) and the multi-RHS half
Dslash on it (dslash_eo_paired), against the FP64 oracle on the same rounded links: every
link storage format, both parities, odd and even numbers of right-hand sides, lattices
whose half volume is not a multiple of the 32-site warp, every launch shape, and sampled
sites of the 16^3 x 32 lattice with 8 right-hand sides."""
import numpy as np
import pytest

import synth
from oracle import dslash as odslash
from oracle.precision import quantize_links
from helpers import rel_l2, to_device_vec, from_device_vec, store_tolerance

pytestmark = pytest.mark.gpu

FORMATS = [("f32", 18), ("f32", 12), ("bf16", 12), ("bf16", 18), ("f16", 12), ("f16", 18)]
DIMS = [(4, 4, 4, 4), (6, 4, 2, 10), (8, 8, 4, 6)]


@pytest.fixture(scope="module")
def lq():
    import paper_1309_0551_gb300 as lq
    return lq


@pytest.fixture(scope="module")
def ctx(lq):
    return lq.Context(0)


def paired_expected(chi):
    """The layout written out from its definition: [pair][colour][site] of
    (Re v_2p, Re v_2p+1, Im v_2p, Im v_2p+1), zero padding for an odd last pair."""
    nrhs, Vh, _ = chi.shape
    npair = (nrhs + 1) // 2
    out = np.zeros((npair, 3, Vh, 4), dtype=np.float32)
    c64 = chi.astype(np.complex64)
    for r in range(nrhs):
        p, h = divmod(r, 2)
        out[p, :, :, h] = c64[r].real.T
        out[p, :, :, 2 + h] = c64[r].imag.T
    return out


def run_paired(lq, ctx, g, chi, parity):
    import torch
    nrhs, Vh, _ = chi.shape
    cd = to_device_vec(chi, "f32")
    pin = torch.empty(lq.paired_numel(Vh, nrhs), dtype=torch.float32, device="cuda")
    pout = torch.empty_like(pin)
    out = torch.empty_like(cd)
    lq.lq_vec_pair(ctx, Vh, nrhs, cd, pin)
    lq.dslash_eo_paired(ctx, g, pin, pout, parity, nrhs)
    lq.lq_vec_unpair(ctx, Vh, nrhs, pout, out)
    ctx.sync()
    return from_device_vec(out), from_device_vec(cd)


@pytest.mark.parametrize("nrhs", [1, 2, 3, 7, 8, 16])
def test_pair_layout_and_round_trip(lq, ctx, nrhs):
    import torch
    dims = (6, 4, 2, 10)
    Vh = synth.volume(dims) // 2
    chi = synth.fermion_field(dims, nrhs, seed=900 + nrhs)
    cd = to_device_vec(chi, "f32")
    pin = torch.full((lq.paired_numel(Vh, nrhs),), float("nan"), dtype=torch.float32, device="cuda")
    lq.lq_vec_pair(ctx, Vh, nrhs, cd, pin)
    back = torch.empty_like(cd)
    lq.lq_vec_unpair(ctx, Vh, nrhs, pin, back)
    ctx.sync()
    got = pin.cpu().numpy().reshape((nrhs + 1) // 2, 3, Vh, 4)
    assert np.array_equal(got, paired_expected(chi))
    assert torch.equal(torch.view_as_real(back), torch.view_as_real(cd))


@pytest.mark.parametrize("gp,recon", FORMATS)
@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("nrhs", [3, 8])
def test_paired_dslash_matches_oracle(lq, ctx, gp, recon, dims, parity, nrhs):
    import torch
    U = synth.gauge_field(dims, "haar", seed=910)
    chi = synth.fermion_field(dims, nrhs, seed=911 + parity)
    g = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), gp, recon)
    got, chi_q = run_paired(lq, ctx, g, chi, parity)
    ref = odslash.dslash_eo_multi(quantize_links(U, gp, recon), chi_q, dims, parity)
    for r in range(nrhs):
        assert rel_l2(got[r], ref[r]) < store_tolerance("f32"), r


@pytest.mark.parametrize("nrhs", [1, 2, 5, 16])
def test_paired_dslash_rhs_counts(lq, ctx, nrhs):
    import torch
    dims = (6, 4, 2, 10)
    U = synth.gauge_field(dims, "haar", seed=912)
    chi = synth.fermion_field(dims, nrhs, seed=913)
    g = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), "f32", 12)
    got, chi_q = run_paired(lq, ctx, g, chi, 1)
    ref = odslash.dslash_eo_multi(quantize_links(U, "f32", 12), chi_q, dims, 1)
    for r in range(nrhs):
        assert rel_l2(got[r], ref[r]) < store_tolerance("f32"), r


def test_paired_agrees_with_canonical_dslash(lq, ctx):
    """Same operator as dslash_eo on FP32 vectors, up to FP32 rounding order."""
    import torch
    dims, nrhs = (8, 8, 4, 6), 8
    U = synth.gauge_field(dims, "haar", seed=914)
    chi = synth.fermion_field(dims, nrhs, seed=915)
    g = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), "bf16", 12)
    got, _ = run_paired(lq, ctx, g, chi, 0)
    cd = to_device_vec(chi, "f32")
    out = torch.empty_like(cd)
    lq.dslash_eo(ctx, g, cd, out, 0, nrhs)
    ctx.sync()
    can = from_device_vec(out)
    assert rel_l2(got, can) < 2e-6


SHAPES = [(b, np_) for np_ in (1, 2, 4) for b in (64, 128, 256)]


@pytest.mark.parametrize("block,np_", SHAPES)
@pytest.mark.parametrize("nrhs", [5, 8])
def test_every_launch_shape(lq, monkeypatch, block, np_, nrhs):
    import torch
    npair = (nrhs + 1) // 2
    groups = -(-npair // np_)
    if block % (32 * groups):
        pytest.skip("shape does not hold whole pair groups")
    monkeypatch.setenv("LQCD_DSLASH_SHAPE", f"{block},{np_},32")
    ctx = lq.Context(0)
    dims = (6, 4, 2, 10)
    U = synth.gauge_field(dims, "haar", seed=916)
    chi = synth.fermion_field(dims, nrhs, seed=917)
    g = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), "f32", 18)
    got, chi_q = run_paired(lq, ctx, g, chi, 0)
    ref = odslash.dslash_eo_multi(U, chi_q, dims, 0)
    for r in range(nrhs):
        assert rel_l2(got[r], ref[r]) < store_tolerance("f32"), r


def test_full_size_16c32_nrhs8_sampled(lq, ctx):
    """The bench's multi-RHS workload (16^3 x 32, 8 right-hand sides, FP32 12-real links),
    in the launch shape the tuner picks, on 300 sampled sites per parity."""
    import torch
    dims, nrhs = (16, 16, 16, 32), 8
    U = synth.gauge_field(dims, "haar", seed=918)
    chi = synth.fermion_field(dims, nrhs, seed=919)
    g = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), "f32", 12)
    Uq = quantize_links(U, "f32", 12)
    sites = np.sort(synth.rng(920).choice(synth.volume(dims) // 2, 300, replace=False))
    for parity in (0, 1):
        got, chi_q = run_paired(lq, ctx, g, chi, parity)
        for r in (0, 3, 7):
            ref = odslash.dslash_eo_sites(Uq, chi_q[r], dims, parity, sites)
            assert rel_l2(got[r][sites], ref) < store_tolerance("f32")


def test_argument_errors(lq, ctx):
    import torch
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, "haar", seed=921)
    Vh = synth.volume(dims) // 2
    g64 = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), "f64", 18)
    g32 = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), "f32", 18)
    a = torch.zeros(lq.paired_numel(Vh, 4), dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    with pytest.raises(lq.LQError):
        lq.dslash_eo_paired(ctx, g64, a, b, 0, 4)
    with pytest.raises(lq.LQError):
        lq.dslash_eo_paired(ctx, g32, a, b, 0, 17)
    with pytest.raises(lq.LQError):
        lq.dslash_eo_paired(ctx, g32, a, a, 0, 4)
    with pytest.raises(lq.LQError):
        lq.dslash_eo_paired(ctx, g32, a[1:], b, 0, 4)
    with pytest.raises(lq.LQError):
        lq.lq_vec_pair(ctx, Vh, 0, a, b)
