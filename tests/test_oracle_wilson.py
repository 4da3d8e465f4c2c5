"""Pins for the oracle's Wilson hopping term and the two half Wilson vector routines of
Table 1: the Clifford algebra of the gamma matrices, brute force against the dense
operator, the free-field plane-wave closed form, gamma_5-hermiticity and the sign as the
adjoint, gauge covariance, and the half-spinor form against the full 4x4 form."""
import numpy as np
import pytest

import synth
from oracle import dslash, geometry as geo, su3, wilson


def test_gamma_matrices_clifford_hermitian_chiral():
    G = wilson.GAMMA
    for mu in range(4):
        assert np.abs(G[mu] - np.conj(G[mu]).T).max() == 0          # Hermitian
        for nu in range(4):
            anti = G[mu] @ G[nu] + G[nu] @ G[mu]
            assert np.abs(anti - 2 * (mu == nu) * np.eye(4)).max() == 0
        # chiral basis: block off-diagonal, so (1 +- gamma) is fixed by its upper half
        assert np.abs(G[mu][0:2, 0:2]).max() == 0 and np.abs(G[mu][2:4, 2:4]).max() == 0
    assert np.abs(wilson.gamma5() - np.diag([1, 1, -1, -1])).max() == 0


def test_hwvec_routines():
    A, h = synth.hwvec_batch(64, 301)
    g = synth.complex_gaussian(synth.rng(302), (64, 2, 3))
    Ah = su3.mult_su3_mat_hwvec(A, h)
    # <g, A h> = <A^dag g, h> for each spin component and item
    lhs = np.sum(np.conj(g) * Ah, axis=-1)
    rhs = np.sum(np.conj(su3.mult_adj_su3_mat_hwvec(A, g)) * h, axis=-1)
    assert np.abs(lhs - rhs).max() < 1e-13
    # unitary A: A^dag (A h) = h; spin components are independent colour vectors
    assert np.abs(su3.mult_adj_su3_mat_hwvec(A, Ah) - h).max() < 1e-13
    for s in range(2):
        assert np.abs(Ah[:, s] - su3.mult_su3_mat_vec(A, h[:, s])).max() == 0


@pytest.mark.parametrize("dims", [(4, 2, 2, 4), (2, 4, 4, 2), (4, 4, 2, 2)])
@pytest.mark.parametrize("sign", [1, -1])
def test_stencil_and_projected_match_dense(dims, sign):
    U = synth.gauge_field(dims, "haar", seed=303)
    V = synth.volume(dims)
    D = wilson.dense_wilson(U, dims, sign)
    psi = synth.spinor_field(dims, 1, 304, sites="full")[0]
    ref = (D @ psi.reshape(-1)).reshape(V, 4, 3)
    full = psi.reshape(geo.shape(dims) + (4, 3))
    assert np.abs(wilson.wilson_full(U, full, dims, sign).reshape(V, 4, 3) - ref).max() < 1e-13
    assert np.abs(wilson.wilson_full_projected(U, full, dims, sign).reshape(V, 4, 3) - ref).max() < 1e-13
    # even/odd blocks: the hopping term only joins opposite parities
    for p in (0, 1):
        rows = dslash.parity_indices(dims, p)
        cols = dslash.parity_indices(dims, 1 - p)
        ri = (12 * rows[:, None] + np.arange(12)).reshape(-1)
        ci = (12 * cols[:, None] + np.arange(12)).reshape(-1)
        same = (12 * rows[:, None] + np.arange(12)).reshape(-1)
        assert np.abs(D[np.ix_(ri, same)]).max() == 0
        v = synth.spinor_field(dims, 1, 305 + p)[0]
        blk = D[np.ix_(ri, ci)] @ v.reshape(-1)
        assert np.abs(wilson.wilson_eo(U, v, dims, p, sign).reshape(-1) - blk).max() < 1e-13


def test_gamma5_hermiticity_and_sign_is_adjoint():
    dims = (4, 2, 4, 2)
    U = synth.gauge_field(dims, "haar", seed=307)
    V = synth.volume(dims)
    Dp = wilson.dense_wilson(U, dims, 1)
    Dm = wilson.dense_wilson(U, dims, -1)
    G5 = np.kron(np.eye(V), np.kron(wilson.gamma5(), np.eye(3)))
    assert np.abs(Dm - np.conj(Dp).T).max() < 1e-14
    assert np.abs(G5 @ Dp @ G5 - Dm).max() < 1e-14


@pytest.mark.parametrize("sign", [1, -1])
def test_free_field_plane_waves(sign):
    dims = (4, 6, 4, 8)
    V = synth.volume(dims)
    one = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, V, 3, 3))
    x, y, z, t = geo.coords(dims)
    g = synth.rng(308)
    for _ in range(5):
        n = [int(g.integers(0, Lm)) for Lm in dims]
        p = [2 * np.pi * k / Lm for k, Lm in zip(n, dims)]
        chi = synth.complex_gaussian(g, (4, 3))
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        psi = phase[..., None, None] * chi
        # D e^{ipx} chi = sum_mu (2 cos p_mu - 2 i s gamma_mu sin p_mu) e^{ipx} chi
        K = sum(2 * np.cos(q) * np.eye(4) - 2j * sign * np.sin(q) * wilson.GAMMA[mu] for mu, q in enumerate(p))
        want = phase[..., None, None] * wilson.spin_mul(K, chi)
        assert np.abs(wilson.wilson_full(one, psi, dims, sign) - want).max() < 1e-12


def test_gauge_covariance():
    dims = (4, 4, 2, 4)
    U = synth.gauge_field(dims, "haar", seed=309)
    g = synth.haar_su3(synth.rng(310), synth.volume(dims)).reshape(geo.shape(dims) + (3, 3))
    Ul = geo.gauge_lattice(U, dims)
    Ug = np.stack([su3.mult_su3_na(su3.mult_su3_nn(g, Ul[mu]), np.roll(g, -1, axis=geo.AXIS[mu]))
                   for mu in range(4)]).reshape(U.shape)
    psi = synth.spinor_field(dims, 1, 311, sites="full")[0].reshape(geo.shape(dims) + (4, 3))
    gpsi = wilson.colour_mul(g, psi)
    lhs = wilson.wilson_full(Ug, gpsi, dims, 1)
    rhs = wilson.colour_mul(g, wilson.wilson_full(U, psi, dims, 1))
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(psi) < 1e-13


def test_projection_roundtrip():
    psi = synth.complex_gaussian(synth.rng(312), (16, 4, 3))
    for mu in range(4):
        for eps in (1, -1):
            P = np.eye(4) + eps * wilson.GAMMA[mu]
            full = wilson.spin_mul(P, psi)
            h = wilson.half_project(psi, mu, eps)
            assert np.abs(wilson.half_reconstruct(h, mu, eps) - full).max() < 1e-14
            # rank 2: the projection of the projection is twice the projection
            assert np.abs(wilson.spin_mul(P, full) - 2 * full).max() < 1e-14


def test_sitewise_matches_stencil():
    dims = (4, 6, 2, 4)
    U = synth.gauge_field(dims, "near_identity", seed=313, eps=0.3)
    for p in (0, 1):
        v = synth.spinor_field(dims, 1, 314 + p)[0]
        ref = wilson.wilson_eo(U, v, dims, p, -1)
        sites = np.array([0, 3, 17, len(v) - 1])
        assert np.abs(wilson.wilson_eo_sites(U, v, dims, p, sites, -1) - ref[sites]).max() < 1e-13
