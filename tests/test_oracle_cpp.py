"""Pins of the FP64 C++ oracle (oracle/cpp/oracle.cpp) against things other than itself: the
brute-force dense D, anti-Hermiticity, gauge covariance, the free-field plane-wave spectrum,
the CG closed form and dense solve, the hand-computed Table 1 examples -- and, as a second
independent check, the numpy oracle."""
import numpy as np
import pytest

import synth
from oracle import cxx, dslash, geometry as geo, su3
from oracle.precision import third_row


def _rel(a, b):
    return np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1))


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 2, 4), (4, 4, 4, 4), (4, 2, 6, 4)])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_dslash_against_dense_D(dims, out_parity):
    U = synth.gauge_field(dims, "haar", seed=501)
    chi = synth.fermion_field(dims, 1, 502)[0]
    D = dslash.dense_block(dslash.dense_D(U, dims), dims, out_parity)
    ref = (D @ chi.reshape(-1)).reshape(chi.shape)
    got = cxx.dslash_eo(U, chi, dims, out_parity, threads=2)
    assert _rel(got, ref) < 1e-14


def test_anti_hermiticity():
    dims = (4, 4, 6, 4)
    U = synth.gauge_field(dims, "haar", seed=503)
    x = synth.fermion_field(dims, 1, 504)[0]
    y = synth.fermion_field(dims, 1, 505)[0]
    lhs = np.vdot(y, cxx.dslash_eo(U, x, dims, 1))          # <y, D_oe x>, y odd
    rhs = -np.vdot(cxx.dslash_eo(U, y, dims, 0), x)         # -<D_eo y, x>
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_gauge_covariance():
    dims = (4, 4, 4, 6)
    V = synth.volume(dims)
    U = synth.gauge_field(dims, "haar", seed=506)
    gx = synth.haar_su3(synth.rng(507), V)
    Ug = np.empty_like(U)
    for mu in range(4):
        nb = np.array([geo.neighbour_lex(dims, x, mu, +1) for x in range(V)])
        Ug[mu] = gx @ U[mu] @ np.conj(np.swapaxes(gx[nb], -1, -2))
    par = geo.parity(dims).reshape(-1)
    ev, od = np.flatnonzero(par == 0), np.flatnonzero(par == 1)
    chi = synth.fermion_field(dims, 1, 508)[0]
    lhs = cxx.dslash_eo(Ug, np.einsum("sab,sb->sa", gx[ev], chi), dims, 1)
    rhs = np.einsum("sab,sb->sa", gx[od], cxx.dslash_eo(U, chi, dims, 1))
    assert _rel(lhs, rhs) < 1e-13


def test_free_field_plane_wave():
    dims = (4, 6, 4, 8)
    U = synth.gauge_field(dims, "unit")
    x, y, z, t = geo.coords(dims)
    p = [2 * np.pi * k / L for k, L in zip((1, 2, 3, 1), dims)]
    phi = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[..., None] * np.array([1, -2j, 0.5])
    b = geo.full_to_cb(phi, dims, 0)
    mass = 0.3
    lam = mass ** 2 + 4 * sum(np.sin(q) ** 2 for q in p)
    assert _rel(cxx.normal_op(U, b, mass, dims), lam * b) < 1e-14
    sol, info = cxx.cg(U, b, mass, dims, tol=1e-12)
    assert np.abs(sol - b / lam).max() < 1e-12 and info["iters"] <= 2


def test_cg_against_dense_solve():
    dims, mass = (4, 4, 4, 4), 0.1
    U = synth.gauge_field(dims, "haar", seed=509)
    b = synth.fermion_field(dims, 1, 510)[0]
    M = dslash.dense_normal(U, mass, dims)
    ref = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    sol, info = cxx.cg(U, b, mass, dims, tol=1e-10, threads=3)
    assert info["true_rel_resid"] <= 1e-10
    assert _rel(sol, ref) < 1e-10 * np.linalg.cond(M)


def test_threads_do_not_change_the_operator():
    dims = (8, 4, 4, 8)
    U = synth.gauge_field(dims, "haar", seed=511)
    chi = synth.fermion_field(dims, 1, 512)[0]
    one = cxx.dslash_eo(U, chi, dims, 1, threads=1)
    assert np.array_equal(one, cxx.dslash_eo(U, chi, dims, 1, threads=cxx.max_threads()))


def test_matches_numpy_oracle():
    dims, mass = (8, 8, 4, 6), 0.2
    U = synth.gauge_field(dims, "near_identity", seed=513, eps=0.3)
    chi = synth.fermion_field(dims, 1, 514)[0]
    for par in (0, 1):
        assert _rel(cxx.dslash_eo(U, chi, dims, par, 4), dslash.dslash_eo(U, chi, dims, par)) < 1e-14
    assert _rel(cxx.normal_op(U, chi, mass, dims, 4), dslash.normal_op(U, chi, mass, dims)) < 1e-14


def _golden():
    import os
    out = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "su3_hand_examples.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split("=", 1)
            out[k.strip()] = np.array([complex(t) for t in v.split()])
    return out


def test_table1_hand_examples():
    """The hand-computed Gaussian-integer examples (Table 1, Eqs. (1.1)-(2.3)): exact."""
    G = _golden()
    A, B = G["A"].reshape(1, 3, 3), G["B"].reshape(1, 3, 3)
    a = G["a"].reshape(1, 3)
    assert np.array_equal(cxx.su3_mat_vec(A, a, 1)[0], G["adj_mat_vec"])
    assert np.array_equal(cxx.su3_mat_vec(A, a, 0)[0], G["mat_vec"])
    assert np.array_equal(cxx.su3_mul(A, B, 0, 0)[0], G["nn"].reshape(3, 3))
    assert np.array_equal(cxx.su3_mul(A, B, 1, 0)[0], G["an"].reshape(3, 3))
    assert np.array_equal(cxx.su3_mul(A, B, 0, 1)[0], G["na"].reshape(3, 3))


def test_table1_routines():
    g = synth.rng(515)
    A, B = synth.haar_su3(g, 50), synth.haar_su3(g, 50)
    b = synth.complex_gaussian(g, (50, 3))
    assert _rel(cxx.su3_mat_vec(A, b, 0), np.einsum("nab,nb->na", A, b)) < 1e-15
    assert _rel(cxx.su3_mat_vec(A, b, 1), np.einsum("nba,nb->na", np.conj(A), b)) < 1e-15
    assert _rel(cxx.su3_mul(A, B, 0, 0), A @ B) < 1e-15
    assert _rel(cxx.su3_mul(A, B, 1, 0), np.conj(np.swapaxes(A, -1, -2)) @ B) < 1e-15
    assert _rel(cxx.su3_mul(A, B, 0, 1), A @ np.conj(np.swapaxes(B, -1, -2))) < 1e-15
    # Eq. (1.1)-(2.3): first component of the adjoint mat-vec, written out
    c0 = np.conj(A[:, 0, 0]) * b[:, 0] + np.conj(A[:, 1, 0]) * b[:, 1] + np.conj(A[:, 2, 0]) * b[:, 2]
    assert np.abs(cxx.su3_mat_vec(A, b, 1)[:, 0] - c0).max() < 1e-15
    # closure: the product of SU(3) matrices is SU(3)
    C = cxx.su3_mul(A, B)
    assert np.abs(np.conj(np.swapaxes(C, -1, -2)) @ C - np.eye(3)).max() < 1e-14
    assert np.abs(C[:, 2] - third_row(C[:, 0], C[:, 1])).max() < 1e-14
