"""Pins for the oracle's staggered Dslash: brute force against the dense D, anti-Hermiticity,
gauge covariance and the free-field spectrum of -D^2."""
import numpy as np
import pytest

import synth
from oracle import dslash, geometry as geo, su3


def _cb_vec(dims, seed, par_sites="half"):
    return synth.fermion_field(dims, 1, seed)[0]


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 2, 4), (4, 4, 4, 4), (4, 2, 6, 4)])
def test_stencil_matches_dense_D(dims):
    U = synth.gauge_field(dims, "haar", seed=21)
    D = dslash.dense_D(U, dims)
    V = synth.volume(dims)
    chi = synth.fermion_field(dims, 1, 22, sites="full")[0]
    full = chi.reshape(geo.shape(dims) + (3,))
    ref = (D @ chi.reshape(-1)).reshape(V, 3)
    got = dslash.dslash_full(U, full, dims).reshape(V, 3)
    assert np.abs(got - ref).max() < 1e-13
    # even/odd blocks agree with the dense blocks in checkerboard order
    for p in (0, 1):
        v = _cb_vec(dims, 23 + p)
        blk = dslash.dense_block(D, dims, p)
        assert np.abs(dslash.dslash_eo(U, v, dims, p).reshape(-1) - blk @ v.reshape(-1)).max() < 1e-13


def test_dense_D_is_anti_hermitian_and_blocks():
    dims = (4, 4, 2, 4)
    U = synth.gauge_field(dims, "haar", seed=24)
    D = dslash.dense_D(U, dims)
    assert np.abs(D + np.conj(D.T)).max() < 1e-15
    Deo = dslash.dense_block(D, dims, 0)
    Doe = dslash.dense_block(D, dims, 1)
    assert np.abs(Deo + np.conj(Doe.T)).max() < 1e-15
    # D only connects opposite parities
    ev = dslash.parity_indices(dims, 0)
    r = (3 * ev[:, None] + np.arange(3)).reshape(-1)
    assert np.abs(D[np.ix_(r, r)]).max() == 0


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8)])
def test_stencil_anti_hermitian_inner_product(dims):
    U = synth.gauge_field(dims, "haar", seed=25)
    x = _cb_vec(dims, 26)   # even
    y = _cb_vec(dims, 27)   # odd
    lhs = np.vdot(y, dslash.dslash_eo(U, x, dims, 1))        # <y, D_oe x>
    rhs = -np.vdot(dslash.dslash_eo(U, y, dims, 0), x)       # -<D_eo y, x>
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_gauge_covariance():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, "haar", seed=28)
    g = synth.haar_su3(synth.rng(29), synth.volume(dims)).reshape(geo.shape(dims) + (3, 3))
    Ul = geo.gauge_lattice(U, dims)
    Ug = np.empty_like(Ul)
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=geo.AXIS[mu])
        Ug[mu] = su3.mult_su3_na(su3.mult_su3_nn(g, Ul[mu]), g_fwd)   # g(x) U g(x+mu)^dag
    chi = synth.fermion_field(dims, 1, 30, sites="full")[0].reshape(geo.shape(dims) + (3,))
    lhs = dslash.dslash_full(Ug.reshape(U.shape), su3.mult_su3_mat_vec(g, chi), dims)
    rhs = su3.mult_su3_mat_vec(g, dslash.dslash_full(U, chi, dims))
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(chi) < 1e-13


@pytest.mark.parametrize("dims,mass", [((4, 4, 4, 4), 0.1), ((4, 6, 2, 8), 0.5)])
def test_free_field_plane_waves(dims, mass):
    U = synth.gauge_field(dims, "unit")
    x, y, z, t = geo.coords(dims)
    g = synth.rng(31)
    for _ in range(4):
        n = [int(g.integers(0, L)) for L in dims]
        p = [2 * np.pi * n[m] / dims[m] for m in range(4)]
        c = synth.complex_gaussian(g, (3,))
        phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
        phi = phase[..., None] * c
        lam = 4 * sum(np.sin(pm) ** 2 for pm in p)
        # -D^2 phi = lam phi on the full lattice
        DDphi = dslash.dslash_full(U, dslash.dslash_full(U, phi, dims), dims)
        assert np.abs(-DDphi - lam * phi).max() < 1e-12
        # and M = m^2 - D_eo D_oe on the even sites
        pe = geo.full_to_cb(phi, dims, 0)
        assert np.abs(dslash.normal_op(U, pe, mass, dims) - (mass ** 2 + lam) * pe).max() < 1e-12


def test_normal_op_matches_dense_and_is_hpd():
    dims = (4, 4, 4, 4)
    mass = 0.05
    U = synth.gauge_field(dims, "haar", seed=32)
    M = dslash.dense_normal(U, mass, dims)
    p = _cb_vec(dims, 33)
    assert np.abs(dslash.normal_op(U, p, mass, dims).reshape(-1) - M @ p.reshape(-1)).max() < 1e-12
    assert np.abs(M - np.conj(M.T)).max() < 1e-13
    assert np.linalg.eigvalsh(M).min() >= mass ** 2 * (1 - 1e-9)


def test_multi_rhs_is_columnwise():
    dims = (4, 4, 2, 2)
    U = synth.gauge_field(dims, "haar", seed=34)
    chi = synth.fermion_field(dims, 3, 35)
    out = dslash.dslash_eo_multi(U, chi, dims, 0)
    for k in range(3):
        assert np.array_equal(out[k], dslash.dslash_eo(U, chi[k], dims, 0))


def test_sitewise_dslash_matches_stencil():
    dims = (4, 6, 2, 4)
    U = synth.gauge_field(dims, "haar", seed=36)
    for p in (0, 1):
        v = _cb_vec(dims, 37 + p)
        full = dslash.dslash_eo(U, v, dims, p)
        sites = np.arange(0, full.shape[0], 7)
        assert np.abs(dslash.dslash_eo_sites(U, v, dims, p, sites) - full[sites]).max() < 1e-13
