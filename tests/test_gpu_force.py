"""The fermion force (dslash_force) and its autograd wrapper against the oracle's gradients,
FP64 finite differences and torch.autograd.gradcheck."""
import numpy as np
import pytest

import synth
from oracle import force as oforce, dslash as odslash
from helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    import paper_1309_0551_gb300 as lq
    return lq


@pytest.fixture(scope="module")
def ctx(lq):
    return lq.Context(0)


def _force(lq, ctx, U, chi, mass, dims, prec):
    import torch
    ct = torch.complex128 if prec == "f64" else torch.complex64
    g = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), prec, 18)
    cd = torch.from_numpy(chi).to(ct).cuda()
    dU = torch.empty(U.shape, dtype=ct, device="cuda")
    F = torch.empty(U.shape, dtype=ct, device="cuda")
    dchi = torch.empty_like(cd)
    S = lq.dslash_force(ctx, g, mass, cd, dSdU=dU, force_TA=F, dSdchi=dchi, want_S=True)
    c = lambda t: t.cpu().to(torch.complex128).numpy()  # noqa: E731
    return S, c(dU), c(F), c(dchi)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f32", 1e-5)])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 6)])
def test_force_matches_oracle(lq, ctx, prec, tol, dims):
    mass = 0.3
    U = synth.gauge_field(dims, "haar", seed=121)
    chi = synth.fermion_field(dims, 1, seed=122)[0]
    S, G, F, dchi = _force(lq, ctx, U, chi, mass, dims, prec)
    G_ref = oforce.link_gradient(U, chi, mass, dims)
    assert abs(S - oforce.action(U, chi, mass, dims)) <= tol * abs(S)
    assert rel_l2(G, G_ref) < tol
    assert rel_l2(F, oforce.force_ta(U, G_ref)) < tol
    assert rel_l2(dchi, oforce.dS_dchi(U, chi, mass, dims)) < tol


def test_force_fp64_against_finite_differences(lq, ctx):
    """Central differences of the action in single link coordinates (h = 1e-6), evaluated
    site by site so that rounding does not swamp the 1e-8 bound."""
    dims, mass = (4, 4, 4, 4), 0.3
    U = synth.gauge_field(dims, "haar", seed=123)
    chi = synth.fermion_field(dims, 1, seed=124)[0]
    _, G, F, dchi = _force(lq, ctx, U, chi, mass, dims, "f64")
    scale = np.abs(G).max()
    g = synth.rng(125)
    h = 1e-6
    for _ in range(32):
        mu, s = int(g.integers(0, 4)), int(g.integers(0, synth.volume(dims)))
        a, b = int(g.integers(0, 3)), int(g.integers(0, 3))
        for unit, part in ((1.0, "re"), (1j, "im")):
            Up, Um = U.copy(), U.copy()
            Up[mu, s, a, b] += unit * h
            Um[mu, s, a, b] -= unit * h
            p1 = odslash.dslash_eo(Up, chi, dims, 1)
            p2 = odslash.dslash_eo(Um, chi, dims, 1)
            fd = float(np.sum(np.sum(np.abs(p1) ** 2, -1) - np.sum(np.abs(p2) ** 2, -1))) / (2 * h)
            an = G[mu, s, a, b].real if part == "re" else G[mu, s, a, b].imag
            assert abs(fd - an) < 1e-8 * scale, (mu, s, a, b, part, fd, an)
    # dS/dchi: S is quadratic in chi, so the central difference is exact up to rounding
    for _ in range(8):
        s, c = int(g.integers(0, chi.shape[0])), int(g.integers(0, 3))
        cp, cm = chi.copy(), chi.copy()
        cp[s, c] += h
        cm[s, c] -= h
        fd = (oforce.action(U, cp, mass, dims) - oforce.action(U, cm, mass, dims)) / (2 * h)
        assert abs(fd - dchi[s, c].real) < 1e-6 * max(1.0, abs(dchi[s, c].real))


def test_autograd_function_and_gradcheck(lq, ctx):
    import torch
    from paper_1309_0551_gb300.autograd import DslashAction, force_ta
    dims, mass = (2, 2, 2, 4), 0.4
    U = synth.gauge_field(dims, "haar", seed=126)
    chi = synth.fermion_field(dims, 1, seed=127)[0]
    Ut = torch.from_numpy(U).cuda().requires_grad_(True)
    ct = torch.from_numpy(chi).cuda().requires_grad_(True)
    S = DslashAction.apply(Ut, ct, mass, ctx, dims)
    S.backward()
    assert rel_l2(Ut.grad.cpu().numpy(), oforce.link_gradient(U, chi, mass, dims)) < 1e-13
    assert rel_l2(ct.grad.cpu().numpy(), oforce.dS_dchi(U, chi, mass, dims)) < 1e-13
    # PyTorch's own finite-difference check of the complex-gradient convention
    Ug = torch.from_numpy(U).cuda().requires_grad_(True)
    cg = torch.from_numpy(chi).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda u, c: DslashAction.apply(u, c, mass, ctx, dims), (Ug, cg),
                                    eps=1e-6, atol=1e-6, rtol=1e-5, fast_mode=True)
    F = force_ta(ctx, torch.from_numpy(U).cuda(), torch.from_numpy(chi).cuda(), mass, dims).cpu().numpy()
    assert rel_l2(F, oforce.force_ta(U, oforce.link_gradient(U, chi, mass, dims))) < 1e-13


def test_force_full_size_32c64_sampled(lq, ctx):
    """The 32^3 x 64 Haar, m = 0.05 workload: FP64 and FP32 forces checked on 200 sampled
    links against the oracle's link-by-link gradient."""
    dims, mass = (32, 32, 32, 64), 0.05
    U = synth.gauge_field(dims, "haar", seed=6)
    chi = synth.fermion_field(dims, 1, seed=7)[0]
    V = synth.volume(dims)
    rs = synth.rng(128)
    links = [(int(rs.integers(0, 4)), int(rs.integers(0, V))) for _ in range(200)]
    links.append((3, V - 1))
    G_ref = oforce.link_gradient_sites(U, chi, mass, dims, links)
    F_ref = np.stack([oforce.force_ta(U[mu, s], Gr) for (mu, s), Gr in zip(links, G_ref)])
    for prec, tol in (("f64", 1e-13), ("f32", 1e-5)):
        _, G, F, _ = _force(lq, ctx, U, chi, mass, dims, prec)
        assert rel_l2(np.stack([G[mu, s] for mu, s in links]), G_ref) < tol
        assert rel_l2(np.stack([F[mu, s] for mu, s in links]), F_ref) < tol
