"""Pins for the oracle's improved (fat + Naik) staggered Dslash: brute force against the
dense operator, anti-Hermiticity, gauge covariance, the free-field spectrum, and the
telescoping of long links built from a pure gauge."""
import numpy as np
import pytest

import synth
from oracle import dslash, geometry as geo, improved, su3


def _fields(dims, seed):
    g = synth.rng(seed)
    V = synth.volume(dims)
    U = synth.gauge_field(dims, "haar", seed=seed)
    F = 0.6 * U + 0.1 * synth.complex_gaussian(g, (4, V, 3, 3))   # a generic non-unitary fat field
    L = improved.long_links(U, dims, -1.0 / 24)
    return U, F, L


@pytest.mark.parametrize("dims", [(4, 4, 2, 4), (6, 4, 4, 2), (2, 2, 2, 8)])
def test_stencil_matches_dense(dims):
    U, F, L = _fields(dims, 201)
    D = improved.dense_D_improved(F, L, dims)
    V = synth.volume(dims)
    chi = synth.fermion_field(dims, 1, 202, sites="full")[0]
    got = improved.dslash_improved_full(F, L, chi.reshape(geo.shape(dims) + (3,)), dims).reshape(V, 3)
    assert np.abs(got - (D @ chi.reshape(-1)).reshape(V, 3)).max() < 1e-13
    assert np.abs(D + np.conj(D.T)).max() < 1e-14
    for p in (0, 1):
        v = synth.fermion_field(dims, 1, 203 + p)[0]
        blk = dslash.dense_block(D, dims, p)
        assert np.abs(improved.dslash_improved_eo(F, L, v, dims, p).reshape(-1) - blk @ v.reshape(-1)).max() < 1e-13


def test_gauge_covariance():
    dims = (4, 4, 4, 4)
    U, F, L = _fields(dims, 204)
    F = U.copy()                              # a covariant fat field
    g = synth.haar_su3(synth.rng(205), synth.volume(dims)).reshape(geo.shape(dims) + (3, 3))
    Ul = geo.gauge_lattice(U, dims)
    Ug = np.empty_like(Ul)
    for mu in range(4):
        Ug[mu] = su3.mult_su3_na(su3.mult_su3_nn(g, Ul[mu]), np.roll(g, -1, axis=geo.AXIS[mu]))
    Ug = Ug.reshape(U.shape)
    Lg = improved.long_links(Ug, dims, -1.0 / 24)
    chi = synth.fermion_field(dims, 1, 206, sites="full")[0].reshape(geo.shape(dims) + (3,))
    lhs = improved.dslash_improved_full(Ug, Lg, su3.mult_su3_mat_vec(g, chi), dims)
    rhs = su3.mult_su3_mat_vec(g, improved.dslash_improved_full(F, L, chi, dims))
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(chi) < 1e-13


def test_long_links_of_a_pure_gauge_telescope():
    dims = (4, 6, 4, 4)
    g = synth.haar_su3(synth.rng(207), synth.volume(dims)).reshape(geo.shape(dims) + (3, 3))
    U = np.stack([su3.mult_su3_na(g, np.roll(g, -1, axis=geo.AXIS[mu])) for mu in range(4)])
    L = geo.gauge_lattice(improved.long_links(U.reshape(4, -1, 3, 3), dims, 0.5), dims)
    for mu in range(4):
        ref = 0.5 * su3.mult_su3_na(g, np.roll(g, -3, axis=geo.AXIS[mu]))   # g(x) g(x+3mu)^dag
        assert np.abs(L[mu] - ref).max() < 1e-14


@pytest.mark.parametrize("dims,cf,cn", [((4, 4, 4, 8), 1.0, -1.0 / 24), ((6, 4, 8, 4), 0.625, -0.2)])
def test_free_field_spectrum(dims, cf, cn):
    V = synth.volume(dims)
    one = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, V, 3, 3))
    F, L = cf * one, cn * one
    x, y, z, t = geo.coords(dims)
    g = synth.rng(208)
    for _ in range(4):
        p = [2 * np.pi * int(g.integers(0, Lm)) / Lm for Lm in dims]
        phi = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[..., None] * synth.complex_gaussian(g, (3,))
        lam = 4 * sum((cf * np.sin(q) + cn * np.sin(3 * q)) ** 2 for q in p)
        DD = improved.dslash_improved_full(F, L, improved.dslash_improved_full(F, L, phi, dims), dims)
        assert np.abs(-DD - lam * phi).max() < 1e-12


def test_sitewise_matches_stencil():
    dims = (6, 4, 4, 2)
    U, F, L = _fields(dims, 209)
    for p in (0, 1):
        v = synth.fermion_field(dims, 1, 210 + p)[0]
        full = improved.dslash_improved_eo(F, L, v, dims, p)
        sites = np.arange(0, full.shape[0], 5)
        assert np.abs(improved.dslash_improved_eo_sites(F, L, v, dims, p, sites) - full[sites]).max() < 1e-13
