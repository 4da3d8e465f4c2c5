"""Parity of the CUDA Wilson hopping term (dslash_wilson_eo) and of the batched half Wilson
vector routines (su3_mat_hwvec_batch) with the FP64 oracle: every link storage format,
both parities, both signs, ragged and degenerate lattices, several right-hand sides, the
16^3 x 32 workload of the benchmark on sampled sites, and the argument checks."""
import numpy as np
import pytest

import synth
from oracle import su3 as osu3, wilson as owilson
from oracle.precision import quantize_links
from helpers import rel_l2, to_device_vec, from_device_vec, empty_vec

pytestmark = pytest.mark.gpu

FORMATS = [("f64", 18), ("f64", 12), ("f32", 18), ("f32", 12),
           ("bf16", 18), ("bf16", 12), ("f16", 18), ("f16", 12)]
TOL = {"f64": 1e-13, "f32": 1e-5}


@pytest.fixture(scope="module")
def lq():
    import paper_1309_0551_gb300 as lq
    return lq


@pytest.fixture(scope="module")
def ctx(lq):
    return lq.Context(0)


def _vp(gp):
    return "f64" if gp == "f64" else "f32"


def _run(lq, ctx, U, dims, gp, recon, psi, parity, sign):
    import torch
    g = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), gp, recon)
    d = to_device_vec(psi, _vp(gp))
    out = empty_vec(psi.shape, _vp(gp))
    lq.dslash_wilson_eo(ctx, g, d, out, parity, psi.shape[0], sign=sign)
    torch.cuda.synchronize()
    return from_device_vec(out), from_device_vec(d)


def _oracle(U, psi, dims, parity, sign):
    return np.stack([owilson.wilson_eo(U, p, dims, parity, sign) for p in psi])


@pytest.mark.parametrize("gp,recon", FORMATS)
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 10), (2, 2, 2, 2)])
@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("sign", [1, -1])
def test_wilson_matches_oracle(lq, ctx, gp, recon, dims, parity, sign):
    U = synth.gauge_field(dims, "haar", seed=71)
    psi = synth.spinor_field(dims, 1, seed=72 + parity)
    got, psi_q = _run(lq, ctx, U, dims, gp, recon, psi, parity, sign)
    ref = _oracle(quantize_links(U, gp, recon), psi_q, dims, parity, sign)
    assert rel_l2(got, ref) < TOL[_vp(gp)]
    if gp in ("f64", "f32"):
        exact = _oracle(U, psi, dims, parity, sign)
        assert rel_l2(got, exact) < TOL[gp]


@pytest.mark.parametrize("gp,recon", [("f64", 18), ("f32", 12), ("bf16", 18)])
def test_multi_rhs(lq, ctx, gp, recon):
    dims = (4, 6, 4, 4)
    U = synth.gauge_field(dims, "near_identity", seed=73, eps=0.2)
    psi = synth.spinor_field(dims, 5, seed=74)
    got, psi_q = _run(lq, ctx, U, dims, gp, recon, psi, 1, 1)
    ref = _oracle(quantize_links(U, gp, recon), psi_q, dims, 1, 1)
    for k in range(psi.shape[0]):
        assert rel_l2(got[k], ref[k]) < TOL[_vp(gp)]


def test_sign_minus_is_gamma5_conjugate(lq, ctx):
    """gamma_5 D(+1) gamma_5 = D(-1), on the device alone."""
    dims = (4, 4, 2, 6)
    U = synth.gauge_field(dims, "haar", seed=75)
    psi = synth.spinor_field(dims, 1, seed=76)
    g5 = np.array([1, 1, -1, -1])[:, None]
    plus, _ = _run(lq, ctx, U, dims, "f64", 18, psi * g5, 0, 1)
    minus, _ = _run(lq, ctx, U, dims, "f64", 18, psi, 0, -1)
    assert rel_l2(plus * g5, minus) < 1e-14


@pytest.mark.parametrize("gp,recon", [("f64", 18), ("f32", 18), ("f32", 12), ("bf16", 12)])
def test_full_size_16c32_sampled(lq, ctx, gp, recon):
    """The 16^3 x 32 near-identity (eps 0.3) workload of the benchmark, checked on 200
    sampled output sites per parity with the site-by-site oracle."""
    dims = (16, 16, 16, 32)
    U = synth.gauge_field(dims, "near_identity", seed=3, eps=0.3)
    Uq = quantize_links(U, gp, recon)
    rs = synth.rng(77)
    for parity in (0, 1):
        psi = synth.spinor_field(dims, 1, seed=78 + parity)
        got, psi_q = _run(lq, ctx, U, dims, gp, recon, psi, parity, 1)
        sites = np.sort(rs.choice(psi.shape[1], 200, replace=False))
        sites[-1] = psi.shape[1] - 1
        ref = owilson.wilson_eo_sites(Uq, psi_q[0], dims, parity, sites, 1)
        assert rel_l2(got[0][sites], ref) < TOL[_vp(gp)]


def test_argument_checks(lq, ctx):
    import torch
    dims = (4, 4, 4, 4)
    U = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(synth.gauge_field(dims, "unit")).cuda(), "f32", 18)
    Vh = 128
    a = torch.zeros((1, Vh, 4, 3), dtype=torch.complex64, device="cuda")
    b = torch.zeros_like(a)
    with pytest.raises(lq.LQError):
        lq.dslash_wilson_eo(ctx, U, a, b, 0, 1, sign=0)
    with pytest.raises(lq.LQError):
        lq.dslash_wilson_eo(ctx, U, a, a, 0, 1)                    # in == out
    with pytest.raises(lq.LQError):
        lq.dslash_wilson_eo(ctx, U, a.to(torch.complex128), b.to(torch.complex128), 0, 1)
    with pytest.raises(lq.LQError):
        lq.dslash_wilson_eo(ctx, U, a, b, 2, 1)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("adj", [0, 1])
@pytest.mark.parametrize("n", [1, 129, 4096 + 77])
def test_hwvec_batch(lq, ctx, prec, adj, n):
    import torch
    A, h = synth.hwvec_batch(n, seed=79 + n)
    dt = torch.complex128 if prec == "f64" else torch.complex64
    Ad = torch.from_numpy(A).to(dt).cuda()
    hd = torch.from_numpy(h).to(dt).cuda()
    c = torch.empty_like(hd)
    lq.su3_mat_hwvec_batch(ctx, Ad, hd, c, n, adj)
    torch.cuda.synchronize()
    An = Ad.cpu().to(torch.complex128).numpy()
    hn = hd.cpu().to(torch.complex128).numpy()
    ref = osu3.mult_adj_su3_mat_hwvec(An, hn) if adj else osu3.mult_su3_mat_hwvec(An, hn)
    assert rel_l2(c.cpu().to(torch.complex128).numpy(), ref) < (1e-15 if prec == "f64" else 1e-6)
    lq.su3_mat_hwvec_batch(ctx, Ad, hd, c, 0, adj)               # n = 0: no-op
