"""Checks of the seeded input generators: SU(3) membership, Haar moments, near-identity
scaling, determinism and layout."""
import numpy as np
import pytest

import synth


def _unitarity(U):
    return np.abs(np.conj(np.swapaxes(U, -1, -2)) @ U - np.eye(3)).max()


@pytest.mark.parametrize("kind", ["haar", "near_identity"])
def test_links_are_special_unitary(kind):
    U = synth.gauge_field((4, 4, 4, 4), kind, seed=51, eps=0.3).reshape(-1, 3, 3)
    assert _unitarity(U) < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14


def test_haar_moments():
    # For Haar measure on SU(3): E[Tr U] = 0, E[|Tr U|^2] = 1, E[(Tr U)^3] = 1 (the last one
    # is the det = 1 invariant; it is 0 on U(3), so it checks the det phase fix).
    n = 100000
    U = synth.haar_su3(synth.rng(52), n)
    tr = np.trace(U, axis1=1, axis2=2)
    se = 1.0 / np.sqrt(n)
    assert abs(tr.mean()) < 4 * se
    assert abs(np.mean(np.abs(tr) ** 2) - 1) < 4 * se
    assert abs(np.mean(tr ** 3) - 1) < 4 * np.sqrt(6) * se


def test_near_identity_scales_with_eps():
    g = [synth.near_identity_su3(synth.rng(53), 2000, e) for e in (0.01, 0.02)]
    d = [np.abs(u - np.eye(3)).mean() for u in g]
    assert 1.8 < d[1] / d[0] < 2.2


def test_determinism_and_shapes():
    a = synth.gauge_field((2, 2, 2, 4), "haar", seed=7)
    b = synth.gauge_field((2, 2, 2, 4), "haar", seed=7)
    assert a.shape == (4, 32, 3, 3) and np.array_equal(a, b)
    f = synth.fermion_field((2, 2, 2, 4), 3, seed=8)
    assert f.shape == (3, 16, 3)
    with pytest.raises(ValueError):
        synth.check_dims((3, 4, 4, 4))
