"""Pins for the oracle's CG solvers (closed form, dense solve) and for the action gradients
(central finite differences, which are exact up to rounding for a quadratic action)."""
import numpy as np
import pytest

import synth
from oracle import cg, dslash, force, geometry as geo, su3


def test_cg_free_field_plane_wave_closed_form():
    dims, mass = (4, 4, 4, 8), 0.2
    U = synth.gauge_field(dims, "unit")
    x, y, z, t = geo.coords(dims)
    p = [2 * np.pi * k / L for k, L in zip((1, 0, 3, 5), dims)]
    phi = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[..., None] * np.array([1, 2j, -1])
    b = geo.full_to_cb(phi, dims, 0)
    lam = 4 * sum(np.sin(q) ** 2 for q in p)
    sol, info = cg.cg(U, b, mass, dims, tol=1e-12)
    assert np.abs(sol - b / (mass ** 2 + lam)).max() < 1e-12
    assert info["iters"] <= 2   # a single eigenvector: CG is exact after one step


@pytest.mark.parametrize("dims,mass", [((4, 4, 4, 4), 0.1), ((4, 4, 2, 6), 0.3)])
def test_cg_matches_dense_solve(dims, mass):
    U = synth.gauge_field(dims, "haar", seed=41)
    b = synth.fermion_field(dims, 1, 42)[0]
    M = dslash.dense_normal(U, mass, dims)
    ref = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    sol, info = cg.cg(U, b, mass, dims, tol=1e-10)
    assert info["true_rel_resid"] <= 1e-10
    cond = np.linalg.cond(M)
    assert np.linalg.norm(sol - ref) / np.linalg.norm(ref) < 1e-10 * cond


@pytest.mark.parametrize("prec,recon", [("f32", 18), ("bf16", 12), ("f16", 12), ("bf16", 18)])
def test_mixed_cg_reaches_fp64_tolerance(prec, recon):
    dims, mass = (4, 4, 4, 4), 0.1
    U = synth.gauge_field(dims, "haar", seed=43)
    b = synth.fermion_field(dims, 1, 44)[0]
    ref, _ = cg.cg(U, b, mass, dims, tol=1e-12)
    sol, info = cg.mixed_cg(U, b, mass, dims, tol=1e-10, prec=prec, recon=recon)
    assert info["true_rel_resid"] <= 1e-10
    assert info["reliable_updates"] >= 1
    M = dslash.dense_normal(U, mass, dims)
    assert np.linalg.norm(sol - ref) / np.linalg.norm(ref) < 1e-10 * np.linalg.cond(M)


def test_replaced_beta_hand_values():
    # r_k = (1, 0, 0), ||r_k||^2 = 1.  Orthogonal new residual: the Fletcher-Reeves value.
    rk = np.array([1.0, 0.0, 0.0], dtype=complex)
    assert cg.replaced_beta(np.array([0.0, 2.0, 1j]), rk, 1.0) == 5.0
    # r_new = (3, 4i, 0): Re<r_new, r_new - r_k> = 25 - 3 = 22
    assert cg.replaced_beta(np.array([3.0, 4j, 0.0]), rk, 1.0) == 22.0
    # r_new = (2, 0, 0) with ||r_k||^2 = 2: (4 - 2) / 2 = 1; r_new = r_k / 2: negative -> 0
    assert cg.replaced_beta(np.array([2.0, 0, 0], dtype=complex), rk, 2.0) == 1.0
    assert cg.replaced_beta(0.5 * rk, rk, 1.0) == 0.0


def test_mixed_cg_with_exact_inner_is_plain_cg():
    """With nothing rounded (FP64 links and vectors inside) the reliable updates replace the
    residual by itself up to rounding: the iteration is the textbook CG, so it takes the
    FP64 solver's iteration count (within the few extra iterations its checks cost) and
    lands on the dense solution."""
    dims, mass = (4, 4, 4, 4), 0.01
    U = synth.gauge_field(dims, "haar", seed=4)
    b = synth.fermion_field(dims, 1, 5)[0]
    _, ref_info = cg.cg(U, b, mass, dims, tol=1e-10, maxiter=5000)
    sol, info = cg.mixed_cg(U, b, mass, dims, tol=1e-10, prec="f64", recon=18, vec_prec="f64",
                            maxiter=5000)
    assert info["true_rel_resid"] <= 1e-10
    assert abs(info["iters"] - ref_info["iters"]) <= 0.03 * ref_info["iters"]
    M = dslash.dense_normal(U, mass, dims)
    ref = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    assert np.linalg.norm(sol - ref) / np.linalg.norm(ref) < 1e-10 * np.linalg.cond(M)


def test_mixed_cg_bf16_links_haar_m001():
    """BF16 links (8 significant bits) at m = 0.01 on Haar links, where the rounded operator
    differs from the FP64 one by far more than m^2: the reliable updates with the
    Polak-Ribiere beta still reach the FP64 true residual 1e-10."""
    dims, mass = (4, 4, 4, 4), 0.01
    U = synth.gauge_field(dims, "haar", seed=4)
    b = synth.fermion_field(dims, 1, 5)[0]
    sol, info = cg.mixed_cg(U, b, mass, dims, tol=1e-10, prec="bf16", recon=12, maxiter=12000)
    assert info["true_rel_resid"] <= 1e-10
    M = dslash.dense_normal(U, mass, dims)
    ref = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    assert np.linalg.norm(sol - ref) / np.linalg.norm(ref) < 1e-10 * np.linalg.cond(M)


# ---------------------------------------------------------------- gradients -----------

DIMS, MASS = (4, 4, 4, 4), 0.3


@pytest.fixture(scope="module")
def field():
    U = synth.gauge_field(DIMS, "haar", seed=45)
    chi = synth.fermion_field(DIMS, 1, 46)[0]
    return U, chi


def _delta_psi2(U1, U2, chi):
    """S(U1) - S(U2) evaluated site by site: psi is identical wherever the links agree, so
    the difference is summed only where it is non-zero (no cancellation of two big sums)."""
    p1 = force.dslash_eo(U1, chi, DIMS, 1)
    p2 = force.dslash_eo(U2, chi, DIMS, 1)
    d = np.sum(np.abs(p1) ** 2, axis=-1) - np.sum(np.abs(p2) ** 2, axis=-1)
    return float(np.sum(d))


def test_action_definition(field):
    U, chi = field
    M = dslash.dense_normal(U, MASS, DIMS)
    S_dense = float(np.vdot(chi.reshape(-1), M @ chi.reshape(-1)).real)
    assert abs(force.action(U, chi, MASS, DIMS) - S_dense) < 1e-12 * S_dense


def test_dS_dchi_finite_difference(field):
    U, chi = field
    grad = force.dS_dchi(U, chi, MASS, DIMS)
    h = 1e-6
    g = synth.rng(47)
    for _ in range(6):
        s, c = int(g.integers(0, chi.shape[0])), int(g.integers(0, 3))
        for unit, part in ((1.0, "re"), (1j, "im")):
            cp, cm = chi.copy(), chi.copy()
            cp[s, c] += unit * h
            cm[s, c] -= unit * h
            fd = (force.action(U, cp, MASS, DIMS) - force.action(U, cm, MASS, DIMS)) / (2 * h)
            an = grad[s, c].real if part == "re" else grad[s, c].imag
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def test_link_gradient_finite_difference(field):
    U, chi = field
    G = force.link_gradient(U, chi, MASS, DIMS)
    scale = np.abs(G).max()
    h = 1e-6
    g = synth.rng(48)
    for _ in range(24):
        mu, s = int(g.integers(0, 4)), int(g.integers(0, synth.volume(DIMS)))
        a, b = int(g.integers(0, 3)), int(g.integers(0, 3))
        for unit, part in ((1.0, "re"), (1j, "im")):
            Up, Um = U.copy(), U.copy()
            Up[mu, s, a, b] += unit * h
            Um[mu, s, a, b] -= unit * h
            fd = _delta_psi2(Up, Um, chi) / (2 * h)
            an = G[mu, s, a, b].real if part == "re" else G[mu, s, a, b].imag
            assert abs(fd - an) < 1e-8 * scale, (mu, s, a, b, part, fd, an)


def _gell_mann():
    L = np.zeros((8, 3, 3), dtype=np.complex128)
    L[0][0, 1] = L[0][1, 0] = 1
    L[1][0, 1], L[1][1, 0] = -1j, 1j
    L[2][0, 0], L[2][1, 1] = 1, -1
    L[3][0, 2] = L[3][2, 0] = 1
    L[4][0, 2], L[4][2, 0] = -1j, 1j
    L[5][1, 2] = L[5][2, 1] = 1
    L[6][1, 2], L[6][2, 1] = -1j, 1j
    L[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return L


def _expm_antiherm(X):
    w, v = np.linalg.eigh(-1j * X)            # X = i H
    return (v * np.exp(1j * w)[None, :]) @ np.conj(v.T)


def test_force_ta_directional_derivatives(field):
    U, chi = field
    F = force.force_ta(U, force.link_gradient(U, chi, MASS, DIMS))
    # F is traceless anti-Hermitian
    assert np.abs(F + su3.adj(F)).max() < 1e-12
    assert np.abs(np.trace(F, axis1=-2, axis2=-1)).max() < 1e-12
    h = 1e-4
    g = synth.rng(49)
    scale = np.abs(F).max()
    for _ in range(6):
        mu, s = int(g.integers(0, 4)), int(g.integers(0, synth.volume(DIMS)))
        for lam in _gell_mann():
            X = 1j * lam
            Up, Um = U.copy(), U.copy()
            Up[mu, s] = _expm_antiherm(h * X) @ U[mu, s]
            Um[mu, s] = _expm_antiherm(-h * X) @ U[mu, s]
            fd = _delta_psi2(Up, Um, chi) / (2 * h)
            an = np.trace(X @ F[mu, s]).real
            assert abs(fd - an) < 1e-7 * scale, (mu, s, fd, an)


def test_link_gradient_sites_matches_full(field):
    U, chi = field
    G = force.link_gradient(U, chi, MASS, DIMS)
    g = synth.rng(50)
    links = [(int(g.integers(0, 4)), int(g.integers(0, synth.volume(DIMS)))) for _ in range(40)]
    Gs = force.link_gradient_sites(U, chi, MASS, DIMS, links)
    for (mu, s), Gl in zip(links, Gs):
        assert np.abs(Gl - G[mu, s]).max() < 1e-13
