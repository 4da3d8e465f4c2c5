"""Molecular-dynamics pieces on the GPU: momentum update (scalar_mult_add_su3_matrix), link
update reunit(exp(eps P) U), and a leapfrog trajectory with the GPU force, against the
oracle."""
import numpy as np
import pytest

import synth
from oracle import md as omd, force as oforce
from helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    import paper_1309_0551_gb300 as lq
    return lq


@pytest.fixture(scope="module")
def ctx(lq):
    return lq.Context(0)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f32", 1e-6)])
@pytest.mark.parametrize("eps", [0.05, 0.7, 3.0])
def test_exp_mul_matches_oracle(lq, ctx, prec, tol, eps):
    import torch
    dims = (4, 4, 2, 6)
    U = synth.gauge_field(dims, "haar", seed=311)
    P = synth.momenta(dims, seed=312)
    ct = torch.complex128 if prec == "f64" else torch.complex64
    Ud, Pd = torch.from_numpy(U).to(ct).cuda(), torch.from_numpy(P).to(ct).cuda()
    out = torch.empty_like(Ud)
    lq.su3_exp_mul_batch(ctx, Pd, Ud, out, eps)
    torch.cuda.synchronize()
    Uq = Ud.cpu().to(torch.complex128).numpy()
    Pq = Pd.cpu().to(torch.complex128).numpy()
    ref = omd.update_links(Uq, Pq, eps)
    assert rel_l2(out.cpu().to(torch.complex128).numpy(), ref) < tol
    lq.su3_exp_mul_batch(ctx, Pd, Ud, Ud, eps)          # in place
    torch.cuda.synchronize()
    assert rel_l2(Ud.cpu().to(torch.complex128).numpy(), ref) < tol


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_scalar_mult_add(lq, ctx, prec):
    import torch
    ct = torch.complex128 if prec == "f64" else torch.complex64
    A = synth.momenta((2, 2, 2, 2), seed=313)
    B = synth.momenta((2, 2, 2, 2), seed=314)
    Ad, Bd = torch.from_numpy(A).to(ct).cuda(), torch.from_numpy(B).to(ct).cuda()
    lq.su3_scalar_mult_add_batch(ctx, Ad, Bd, Ad, -0.25)
    torch.cuda.synchronize()
    ref = omd.update_momenta(torch.from_numpy(A).to(ct).to(torch.complex128).numpy(),
                             torch.from_numpy(B).to(ct).to(torch.complex128).numpy(), -0.25)
    assert rel_l2(Ad.cpu().to(torch.complex128).numpy(), ref) < (1e-15 if prec == "f64" else 1e-7)


def test_leapfrog_trajectory_matches_oracle_and_conserves_energy(lq, ctx):
    import torch
    dims, mass, tau = (4, 4, 4, 4), 0.5, 0.2
    U = synth.gauge_field(dims, "near_identity", seed=304, eps=0.5)
    chi = synth.fermion_field(dims, 1, seed=305)[0]
    P = synth.momenta(dims, seed=306)
    H0 = omd.kinetic(P) + oforce.action(U, chi, mass, dims)
    cd = torch.from_numpy(chi).cuda()
    dH = []
    for n in (10, 20):
        Ud, Pd = torch.from_numpy(U).cuda(), torch.from_numpy(P).cuda()
        S = lq.md_leapfrog(ctx, dims, Ud, Pd, cd, mass, tau / n, n)
        torch.cuda.synchronize()
        U1, P1 = Ud.cpu().numpy(), Pd.cpu().numpy()
        assert abs(S - oforce.action(U1, chi, mass, dims)) < 1e-12 * abs(S)
        dH.append(abs(omd.kinetic(P1) + S - H0))
        if n == 10:
            # the same trajectory with the oracle's pieces
            Ur = U
            Pr = P + 0.5 * (tau / n) * oforce.force_ta(Ur, oforce.link_gradient(Ur, chi, mass, dims))
            for k in range(n):
                Ur = omd.update_links(Ur, Pr, tau / n)
                F = oforce.force_ta(Ur, oforce.link_gradient(Ur, chi, mass, dims))
                Pr = Pr + (tau / n if k < n - 1 else 0.5 * tau / n) * F
            assert rel_l2(U1, Ur) < 1e-12 and rel_l2(P1, Pr) < 1e-12
    assert 3.0 < dH[0] / dH[1] < 5.0


def test_repack_and_reused_work_gauge(lq, ctx):
    """lq_gauge_repack writes a new field into an existing gauge object (every format gives
    the same Dslash as a fresh pack); md_leapfrog with a caller-owned work gauge and force
    buffer reused across calls equals the call that makes its own."""
    import torch
    dims = (4, 4, 2, 6)
    U1 = torch.from_numpy(synth.gauge_field(dims, "haar", seed=321)).cuda()
    U2 = torch.from_numpy(synth.gauge_field(dims, "haar", seed=322)).cuda()
    chi = torch.from_numpy(synth.fermion_field(dims, 1, seed=323)).cuda()
    for prec, recon in (("f64", 18), ("f32", 12), ("bf16", 12)):
        g = lq.lq_gauge_pack(ctx, dims, U1, prec, recon)
        lq.lq_gauge_repack(ctx, g, U2)
        fresh = lq.lq_gauge_pack(ctx, dims, U2, prec, recon)
        vin = chi if prec == "f64" else chi.to(torch.complex64)
        a, b = torch.empty_like(vin), torch.empty_like(vin)
        lq.dslash_eo(ctx, g, vin, a, 1)
        lq.dslash_eo(ctx, fresh, vin, b, 1)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
    dims, mass = (4, 4, 4, 4), 0.5
    U = torch.from_numpy(synth.gauge_field(dims, "near_identity", seed=324, eps=0.5)).cuda()
    P = torch.from_numpy(synth.momenta(dims, seed=325)).cuda()
    c = torch.from_numpy(synth.fermion_field(dims, 1, seed=326)[0]).cuda()
    work = lq.lq_gauge_pack(ctx, dims, U, "f64", 18)
    F = torch.empty_like(U)
    Ua, Pa = U.clone(), P.clone()
    for _ in range(2):
        Sa = lq.md_leapfrog(ctx, dims, Ua, Pa, c, mass, 0.02, 5, work=work, F=F)
    Ub, Pb = U.clone(), P.clone()
    for _ in range(2):
        Sb = lq.md_leapfrog(ctx, dims, Ub, Pb, c, mass, 0.02, 5)
    torch.cuda.synchronize()
    assert torch.equal(Ua, Ub) and torch.equal(Pa, Pb) and Sa == Sb
