"""Improved staggered Dslash (fat + Naik links) and the long-link builder against the
oracle."""
import numpy as np
import pytest

import synth
from oracle import improved
from oracle.precision import quantize_links
from helpers import rel_l2, to_device_vec, from_device_vec, empty_vec, store_tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    import paper_1309_0551_gb300 as lq
    return lq


@pytest.fixture(scope="module")
def ctx(lq):
    return lq.Context(0)


def _fields(dims, seed):
    g = synth.rng(seed)
    U = synth.gauge_field(dims, "haar", seed=seed)
    F = 0.6 * U + 0.1 * synth.complex_gaussian(g, (4, synth.volume(dims), 3, 3))
    return U, F


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 10), (2, 2, 2, 8)])
def test_long_links(lq, ctx, dims):
    import torch
    U, _ = _fields(dims, 221)
    Ud = torch.from_numpy(U).cuda()
    Ld = torch.empty_like(Ud)
    lq.lq_long_links(ctx, dims, Ud, -1.0 / 24, Ld)
    torch.cuda.synchronize()
    assert rel_l2(Ld.cpu().numpy(), improved.long_links(U, dims, -1.0 / 24)) < 1e-14


@pytest.mark.parametrize("gp,vp", [("f64", "f64"), ("f32", "f32"), ("bf16", "f32"), ("f16", "f16")])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 10), (2, 2, 2, 8)])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_improved_dslash_matches_oracle(lq, ctx, gp, vp, dims, nrhs):
    import torch
    U, F = _fields(dims, 222)
    L = improved.long_links(U, dims, -1.0 / 24)
    fat = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(F).cuda(), gp, 18)
    lng = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(L).cuda(), gp, 18)
    for parity in (0, 1):
        chi = synth.fermion_field(dims, nrhs, seed=223 + parity)
        cd = to_device_vec(chi, vp)
        out = empty_vec(chi.shape, vp)
        lq.dslash_eo_improved(ctx, fat, lng, cd, out, parity, nrhs)
        torch.cuda.synchronize()
        chi_q = from_device_vec(cd)
        Fq, Lq = quantize_links(F, gp, 18), quantize_links(L, gp, 18)
        ref = np.stack([improved.dslash_improved_eo(Fq, Lq, c, dims, parity) for c in chi_q])
        assert rel_l2(from_device_vec(out), ref) < store_tolerance(vp)


def test_improved_full_size_16c32_sampled(lq, ctx):
    import torch
    dims = (16, 16, 16, 32)
    U = synth.gauge_field(dims, "near_identity", seed=3, eps=0.3)
    Ud = torch.from_numpy(U).cuda()
    Ld = torch.empty_like(Ud)
    lq.lq_long_links(ctx, dims, Ud, -1.0 / 24, Ld)
    fat = lq.lq_gauge_pack(ctx, dims, Ud, "f32", 18)
    lng = lq.lq_gauge_pack(ctx, dims, Ld, "f32", 18)
    chi = synth.fermion_field(dims, 1, seed=224)
    cd = to_device_vec(chi, "f32")
    out = empty_vec(chi.shape, "f32")
    lq.dslash_eo_improved(ctx, fat, lng, cd, out, 1, 1)
    torch.cuda.synchronize()
    sites = np.sort(synth.rng(225).choice(chi.shape[1], 300, replace=False))
    L = improved.long_links(U, dims, -1.0 / 24)
    ref = improved.dslash_improved_eo_sites(U, L, from_device_vec(cd)[0], dims, 1, sites)
    assert rel_l2(from_device_vec(out)[0][sites], ref) < 1e-5
