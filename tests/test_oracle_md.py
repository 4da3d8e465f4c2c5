"""Pins for the oracle's molecular-dynamics pieces: the matrix exponential against
scipy's expm and a closed form, reunitarisation, and second-order energy conservation of
the leapfrog integrator with the oracle's force."""
import numpy as np
import pytest

import synth
from oracle import force, md, su3


def test_expm_against_scipy_and_closed_form():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    P = synth.momenta((2, 2, 2, 2), seed=301).reshape(-1, 3, 3)[:50]
    E = md.expm_antihermitian(0.7 * P)
    for k in range(50):
        assert np.abs(E[k] - scipy_linalg.expm(0.7 * P[k])).max() < 1e-13
    theta = 0.37
    X = 1j * theta * np.diag([1.0, -1.0, 0.0])
    assert np.abs(md.expm_antihermitian(X) - np.diag([np.exp(1j * theta), np.exp(-1j * theta), 1])).max() < 1e-15
    one = np.eye(3)
    assert np.abs(su3.mult_su3_na(E, E) - one).max() < 1e-14
    assert np.abs(np.linalg.det(E) - 1).max() < 1e-14


def test_reunitarize():
    U = synth.haar_su3(synth.rng(302), 100)
    assert np.abs(md.reunitarize(U) - U).max() < 1e-14
    noisy = U + 1e-3 * synth.complex_gaussian(synth.rng(303), (100, 3, 3))
    R = md.reunitarize(noisy)
    assert np.abs(su3.mult_su3_na(R, R) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(R) - 1).max() < 1e-14


def test_update_momenta_hand_example():
    A = np.array([[1 + 2j, 0, 1], [3 - 1j, 2j, 0], [0, 1 + 1j, -1]])
    B = np.array([[1j, 1, 0], [0, 1, -1], [2, 0, 1j]])
    # A + 2B by hand
    assert np.array_equal(md.update_momenta(A, B, 2.0),
                          np.array([[1 + 4j, 2, 1], [3 - 1j, 2 + 2j, -2], [4, 1 + 1j, -1 + 2j]]))


def _leapfrog(U, P, chi, mass, dims, eps, nsteps):
    P = P + 0.5 * eps * force.force_ta(U, force.link_gradient(U, chi, mass, dims))
    for k in range(nsteps):
        U = md.update_links(U, P, eps)
        F = force.force_ta(U, force.link_gradient(U, chi, mass, dims))
        P = P + (eps if k < nsteps - 1 else 0.5 * eps) * F
    return U, P


def test_leapfrog_energy_error_is_second_order():
    dims, mass, tau = (4, 4, 4, 4), 0.5, 0.2
    U = synth.gauge_field(dims, "near_identity", seed=304, eps=0.5)
    chi = synth.fermion_field(dims, 1, seed=305)[0]
    P = synth.momenta(dims, seed=306)
    H0 = md.kinetic(P) + force.action(U, chi, mass, dims)
    dH = []
    for n in (10, 20):
        U1, P1 = _leapfrog(U, P, chi, mass, dims, tau / n, n)
        dH.append(abs(md.kinetic(P1) + force.action(U1, chi, mass, dims) - H0))
    assert 3.0 < dH[0] / dH[1] < 5.0          # halving the step divides the error by ~4
    # reversibility: flip the momenta and integrate back
    U1, P1 = _leapfrog(U, P, chi, mass, dims, tau / 10, 10)
    U2, P2 = _leapfrog(U1, -P1, chi, mass, dims, tau / 10, 10)
    assert np.abs(U2 - U).max() < 1e-10 and np.abs(P2 + P).max() < 1e-10
