"""The link-staging half Dslash (k_dslash_tma: whole x-rows per block, every link of the
block brought into shared memory by TMA bulk copies), forced through LQCD_DSLASH_SHAPE, against
the FP64 oracle on the same rounded links: every storage format it serves, both parities,
several right-hand sides, blocks that start at the y wrap, and the fused reduction of a
mixed-precision CG."""
import numpy as np
import pytest

import synth
from oracle import dslash as odslash
from oracle.precision import quantize_links
from helpers import rel_l2, to_device_vec, from_device_vec, empty_vec, store_tolerance

pytestmark = pytest.mark.gpu

LINK_BYTES = {("f32", 18): (72, 8), ("f32", 12): (48, 16), ("bf16", 18): (36, 4), ("bf16", 12): (24, 8),
              ("f16", 18): (36, 4), ("f16", 12): (24, 8)}


def tma_sites(dims, gp, recon):
    """The block size the library picks (0: the kernel does not apply)."""
    lb, mc = LINK_BYTES[(gp, recon)]
    Lxh, Ly = dims[0] // 2, dims[1]
    if (mc == 8 and Lxh % 2) or (mc == 4 and Lxh % 4):
        return 0
    best = 0
    for nr in range(1, Ly + 1):
        T = nr * Lxh
        if Ly % nr == 0 and T % 32 == 0 and 64 <= T <= 256 and 8 * T * lb <= 112 * 1024:
            best = T
    return best


@pytest.fixture(scope="module")
def lq():
    import paper_1309_0551_gb300 as lq
    return lq


@pytest.fixture
def ctx(lq, monkeypatch):
    monkeypatch.setenv("LQCD_DSLASH_SHAPE", "128,1,16")
    return lq.Context(0)


CASES = [(gp, recon, vp, dims)
         for (gp, recon, vp) in [("f32", 18, "f32"), ("f32", 12, "f32"), ("bf16", 12, "bf16"), ("bf16", 12, "f32"),
                                 ("bf16", 18, "f32"), ("f16", 12, "f16"), ("f16", 18, "f16")]
         for dims in [(16, 8, 4, 6), (8, 16, 2, 2), (12, 16, 2, 4), (16, 16, 4, 4)]
         if tma_sites(dims, gp, recon)]


@pytest.mark.parametrize("gp,recon,vp,dims", CASES)
@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_tma_kernel_matches_oracle(lq, ctx, gp, recon, vp, dims, parity, nrhs):
    import torch
    U = synth.gauge_field(dims, "haar", seed=801)
    chi = synth.fermion_field(dims, nrhs, seed=802 + parity)
    g = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), gp, recon)
    cd = to_device_vec(chi, vp)
    out = empty_vec(chi.shape, vp)
    lq.dslash_eo(ctx, g, cd, out, parity, nrhs)
    ctx.sync()
    got, chi_q = from_device_vec(out), from_device_vec(cd)
    ref = odslash.dslash_eo_multi(quantize_links(U, gp, recon), chi_q, dims, parity)
    assert rel_l2(got, ref) < store_tolerance(vp)


def test_tma_kernel_full_size_16c32_sampled(lq, ctx):
    import torch
    dims = (16, 16, 16, 32)
    assert tma_sites(dims, "f32", 18) == 128
    U = synth.gauge_field(dims, "near_identity", seed=3, eps=0.3)
    chi = synth.fermion_field(dims, 1, seed=2)
    g = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), "f32", 18)
    cd = to_device_vec(chi, "f32")
    out = empty_vec(chi.shape, "f32")
    sites = np.sort(synth.rng(803).choice(synth.volume(dims) // 2, 300, replace=False))
    for parity in (0, 1):
        lq.dslash_eo(ctx, g, cd, out, parity, 1)
        ctx.sync()
        got = from_device_vec(out)[0][sites]
        ref = odslash.dslash_eo_sites(U, from_device_vec(cd)[0], dims, parity, sites)
        assert rel_l2(got, ref) < 1e-5


def test_tma_kernel_in_mixed_cg(lq, ctx):
    """The fused D_eo with <p, Ap> (deferred per-block partials) runs in the link-staging
    kernel too: the mixed solve reaches the FP64 true residual."""
    import torch
    dims, mass = (16, 8, 4, 6), 0.2
    U = synth.gauge_field(dims, "haar", seed=804)
    b = synth.fermion_field(dims, 2, seed=805)
    Ud = torch.from_numpy(U).cuda()
    hi = lq.lq_gauge_pack(ctx, dims, Ud, "f64", 18)
    lo = lq.lq_gauge_pack(ctx, dims, Ud, "f32", 12)
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    st = lq.cg_solve(ctx, hi, lo, mass, bd, xd, 2, tol=1e-10, maxiter=5000)
    x = xd.cpu().numpy()
    for k in range(2):
        r = b[k] - odslash.normal_op(U, x[k], mass, dims)
        assert st[k]["true_rel_resid"] <= 1e-10
        assert np.linalg.norm(r) / np.linalg.norm(b[k]) <= 1.05e-10
