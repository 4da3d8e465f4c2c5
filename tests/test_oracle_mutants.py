"""The oracle's pins reject plausible mistakes: each test plants one in a copy of an oracle
routine (on the CPU) and checks that a pin used elsewhere in the suite fails on it, while
the unmodified routine passes.  Planted: a backward hop without the adjoint, a staggered
phase taken from the wrong coordinate, the Wilson projectors swapped, a TA projection
that forgets the trace, and the Fletcher-Reeves beta after a reliable update."""
import numpy as np

import synth
from oracle import dslash, force, geometry as geo, wilson
from oracle.su3 import adj, mult_su3_mat_vec, mult_adj_su3_mat_vec


def _stencil(U, chi, dims, backward, eta):
    Ul = geo.gauge_lattice(U, dims)
    out = np.zeros_like(chi)
    for mu in range(4):
        ax = geo.AXIS[mu]
        hop = mult_su3_mat_vec(Ul[mu], np.roll(chi, -1, axis=ax)) - \
            backward(np.roll(Ul[mu], 1, axis=ax), np.roll(chi, 1, axis=ax))
        out += eta[mu][..., None] * hop
    return out


def _anti_hermitian(op, dims):
    shp = geo.shape(dims) + (3,)
    x = synth.fermion_field(dims, 1, 401, sites="full")[0].reshape(shp)
    y = synth.fermion_field(dims, 1, 402, sites="full")[0].reshape(shp)
    return abs(np.vdot(y, op(x)) + np.vdot(op(y), x)) < 1e-12


def test_backward_hop_without_adjoint_is_caught():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, "haar", seed=403)
    eta = geo.eta(dims)
    good = lambda c: _stencil(U, c, dims, mult_adj_su3_mat_vec, eta)
    bad = lambda c: _stencil(U, c, dims, mult_su3_mat_vec, eta)
    assert _anti_hermitian(good, dims)
    assert np.abs(good(np.ones(geo.shape(dims) + (3,), complex)) -
                  dslash.dslash_full(U, np.ones(geo.shape(dims) + (3,), complex), dims)).max() < 1e-13
    assert not _anti_hermitian(bad, dims)


def test_phase_from_the_wrong_coordinate_is_caught():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, "haar", seed=404)
    x, y, z, t = geo.coords(dims)
    eta = geo.eta(dims).copy()
    eta[1] = (-1.0) ** y          # eta_y must depend on x, not on y
    bad = lambda c: _stencil(U, c, dims, mult_adj_su3_mat_vec, eta)
    assert not _anti_hermitian(bad, dims)


def test_swapped_wilson_projectors_are_caught():
    """The free-field closed form fixes which projector goes with which hop."""
    dims = (4, 4, 4, 4)
    V = synth.volume(dims)
    one = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, V, 3, 3))
    x, y, z, t = geo.coords(dims)
    p = [2 * np.pi / 4, 0.0, 2 * np.pi * 2 / 4, 2 * np.pi * 3 / 4]
    chi = synth.complex_gaussian(synth.rng(405), (4, 3))
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    psi = phase[..., None, None] * chi
    K = sum(2 * np.cos(q) * np.eye(4) - 2j * np.sin(q) * wilson.GAMMA[mu] for mu, q in enumerate(p))
    want = phase[..., None, None] * wilson.spin_mul(K, chi)
    assert np.abs(wilson.wilson_full(one, psi, dims, 1) - want).max() < 1e-12
    swapped = wilson.wilson_full(one, psi, dims, -1)   # (1 + gamma) forward, (1 - gamma) backward
    assert np.abs(swapped - want).max() > 1e-3


def test_ta_without_trace_removal_is_caught():
    """F = TA(U G^dag) must be traceless anti-Hermitian (an su(3) element)."""
    A = synth.complex_gaussian(synth.rng(406), (32, 3, 3))
    good = force.ta(A)
    bad = 0.5 * (A - adj(A))
    for F, ok in ((good, True), (bad, False)):
        traceless = np.abs(np.trace(F, axis1=-2, axis2=-1)).max() < 1e-13
        antiherm = np.abs(F + adj(F)).max() < 1e-13
        assert (traceless and antiherm) == ok


def test_fletcher_reeves_beta_after_replacement_is_caught(monkeypatch):
    """The mixed CG's pin at 4^4, BF16 links, m = 0.01 (1e-10 within 12000 iterations)
    fails when the beta after a residual replacement is ||r_new||^2 / ||r_k||^2."""
    from oracle import cg
    dims, mass = (4, 4, 4, 4), 0.01
    U = synth.gauge_field(dims, "haar", seed=4)
    b = synth.fermion_field(dims, 1, 5)[0]
    monkeypatch.setattr(cg, "replaced_beta",
                        lambda r_new, r_k, rr_k: float(np.vdot(r_new, r_new).real) / rr_k)
    _, info = cg.mixed_cg(U, b, mass, dims, tol=1e-10, prec="bf16", recon=12, maxiter=12000)
    assert info["true_rel_resid"] > 1e-10
