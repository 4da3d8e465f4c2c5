"""Property-based pins of the oracle's operators over random even lattice shapes, seeds and
fields: the staggered D is anti-Hermitian (<y, D x> = -<D y, x>), the Wilson hopping term
satisfies gamma_5 D(+1) gamma_5 = D(-1) = D(+1)^dag in the inner product, and both are
gauge covariant.  Each is a fact of the mathematics, independent of the stencil code."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import synth  # noqa: E402
from oracle import dslash, geometry as geo, su3, wilson  # noqa: E402

dims_st = st.tuples(*[st.sampled_from([2, 4, 6]) for _ in range(4)])
seed_st = st.integers(min_value=0, max_value=2**31 - 1)
field_st = st.sampled_from(["haar", "near_identity"])


def _field(dims, kind, seed):
    return synth.gauge_field(dims, kind, seed=seed, eps=0.4) if kind == "near_identity" else \
        synth.gauge_field(dims, kind, seed=seed)


def _gauge_transform(U, g, dims):
    Ul = geo.gauge_lattice(U, dims)
    return np.stack([su3.mult_su3_na(su3.mult_su3_nn(g, Ul[mu]), np.roll(g, -1, axis=geo.AXIS[mu]))
                     for mu in range(4)]).reshape(np.shape(U))


@settings(max_examples=25, deadline=None)
@given(dims_st, seed_st, field_st)
def test_staggered_anti_hermitian(dims, seed, kind):
    U = _field(dims, kind, seed)
    shp = geo.shape(dims) + (3,)
    x = synth.fermion_field(dims, 1, seed + 1, sites="full")[0].reshape(shp)
    y = synth.fermion_field(dims, 1, seed + 2, sites="full")[0].reshape(shp)
    lhs = np.vdot(y, dslash.dslash_full(U, x, dims))
    rhs = -np.vdot(dslash.dslash_full(U, y, dims), x)
    assert abs(lhs - rhs) <= 1e-12 * (1 + abs(lhs))


@settings(max_examples=20, deadline=None)
@given(dims_st, seed_st, field_st)
def test_wilson_gamma5_hermiticity(dims, seed, kind):
    U = _field(dims, kind, seed)
    shp = geo.shape(dims) + (4, 3)
    x = synth.spinor_field(dims, 1, seed + 1, sites="full")[0].reshape(shp)
    y = synth.spinor_field(dims, 1, seed + 2, sites="full")[0].reshape(shp)
    g5 = wilson.gamma5()
    # <y, D(+1) x> = <D(-1) y, x>, and D(-1) = gamma_5 D(+1) gamma_5
    lhs = np.vdot(y, wilson.wilson_full(U, x, dims, 1))
    rhs = np.vdot(wilson.wilson_full(U, y, dims, -1), x)
    assert abs(lhs - rhs) <= 1e-12 * (1 + abs(lhs))
    conj = wilson.spin_mul(g5, wilson.wilson_full(U, wilson.spin_mul(g5, x), dims, 1))
    assert np.abs(conj - wilson.wilson_full(U, x, dims, -1)).max() < 1e-12


@settings(max_examples=15, deadline=None)
@given(dims_st, seed_st)
def test_gauge_covariance_both_operators(dims, seed):
    U = synth.gauge_field(dims, "haar", seed=seed)
    g = synth.haar_su3(synth.rng(seed + 3), synth.volume(dims)).reshape(geo.shape(dims) + (3, 3))
    Ug = _gauge_transform(U, g, dims)
    chi = synth.fermion_field(dims, 1, seed + 4, sites="full")[0].reshape(geo.shape(dims) + (3,))
    lhs = dslash.dslash_full(Ug, su3.mult_su3_mat_vec(g, chi), dims)
    rhs = su3.mult_su3_mat_vec(g, dslash.dslash_full(U, chi, dims))
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(chi)
    psi = synth.spinor_field(dims, 1, seed + 5, sites="full")[0].reshape(geo.shape(dims) + (4, 3))
    lhs = wilson.wilson_full(Ug, wilson.colour_mul(g, psi), dims, 1)
    rhs = wilson.colour_mul(g, wilson.wilson_full(U, psi, dims, 1))
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(psi)
