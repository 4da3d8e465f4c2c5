"""Pins for the oracle's SU(3) routines (Table 1, Eqs. (1.1)-(2.3)) and storage formats."""
import os

import numpy as np
import pytest

import synth
from oracle import su3, precision

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "su3_hand_examples.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split("=", 1)
        out[k.strip()] = np.array([complex(t) for t in v.split()])
    return out


G = _golden()
A = G["A"].reshape(3, 3)
B = G["B"].reshape(3, 3)
a = G["a"]
b = G["b"]


def test_hand_examples():
    assert np.array_equal(su3.mult_adj_su3_mat_vec(A, a), G["adj_mat_vec"])
    assert np.array_equal(su3.mult_su3_mat_vec(A, a), G["mat_vec"])
    assert np.array_equal(su3.mult_su3_nn(A, B), G["nn"].reshape(3, 3))
    assert np.array_equal(su3.mult_su3_an(A, B), G["an"].reshape(3, 3))
    assert np.array_equal(su3.mult_su3_na(A, B), G["na"].reshape(3, 3))
    assert np.array_equal(su3.su3_projector(a, b), G["projector"].reshape(3, 3))


def test_adjoint_matvec_equals_conjugate_transpose_product():
    U = synth.haar_su3(synth.rng(11), 64)
    v = synth.complex_gaussian(synth.rng(12), (64, 3))
    ref = np.matmul(np.conj(np.swapaxes(U, 1, 2)), v[..., None])[..., 0]
    assert np.abs(su3.mult_adj_su3_mat_vec(U, v) - ref).max() < 1e-14


def test_unitary_closure_and_inverse():
    g = synth.rng(13)
    U, W = synth.haar_su3(g, 200), synth.haar_su3(g, 200)
    one = np.eye(3)
    # U U^dag = U^dag U = 1 fixes the conjugation and the transposition in an/na
    assert np.abs(su3.mult_su3_na(U, U) - one).max() < 1e-14
    assert np.abs(su3.mult_su3_an(U, U) - one).max() < 1e-14
    # product of SU(3) is SU(3)
    C = su3.mult_su3_nn(U, W)
    assert np.abs(su3.mult_su3_an(C, C) - one).max() < 1e-14
    assert np.abs(np.linalg.det(C) - 1).max() < 1e-14
    # A^dag b undoes A b
    v = synth.complex_gaussian(g, (200, 3))
    assert np.abs(su3.mult_adj_su3_mat_vec(U, su3.mult_su3_mat_vec(U, v)) - v).max() < 1e-14
    # associativity (U W) v = U (W v)
    lhs = su3.mult_su3_mat_vec(C, v)
    rhs = su3.mult_su3_mat_vec(U, su3.mult_su3_mat_vec(W, v))
    assert np.abs(lhs - rhs).max() < 1e-13


def test_four_direction_routines():
    g = synth.rng(14)
    U = synth.haar_su3(g, 4 * 10).reshape(4, 10, 3, 3)
    v = synth.complex_gaussian(g, (4, 10, 3))
    # with only one non-zero input the sum reduces to the single product
    e0 = np.zeros_like(v)
    e0[2] = v[2]
    assert np.abs(su3.mult_su3_mat_vec_sum_4dir(U, e0) - su3.mult_su3_mat_vec(U[2], v[2])).max() == 0
    # 4dir adjoint outputs undo the forward products direction by direction
    fwd = np.stack([su3.mult_su3_mat_vec(U[m], v[0]) for m in range(4)])
    back = su3.mult_adj_su3_mat_vec_4dir(U, fwd[0])
    assert np.abs(back[0] - v[0]).max() < 1e-14
    sep = su3.mult_adj_su3_mat_4vec(U, v[1])
    assert all(np.array_equal(sep[m], su3.mult_adj_su3_mat_vec(U[m], v[1])) for m in range(4))
    assert np.array_equal(su3.sub_four_su3_vecs(a, np.stack([a, a, a, a])), -3 * a)
    assert np.array_equal(su3.add_su3_vector(a, b), a + b)
    assert np.array_equal(su3.scalar_mult_add_su3_vector(a, b, 2.0), a + 2 * b)
    assert np.array_equal(su3.scalar_mult_add_su3_matrix(A, B, -1.0), A - B)


def test_projector_identities():
    g = synth.rng(15)
    x, y, z = (synth.complex_gaussian(g, (50, 3)) for _ in range(3))
    P = su3.su3_projector(x, y)
    # (x y^dag) z = x (y^dag z);  Tr(x y^dag) = y^dag x
    lhs = su3.mult_su3_mat_vec(P, z)
    rhs = x * np.sum(np.conj(y) * z, axis=-1)[:, None]
    assert np.abs(lhs - rhs).max() < 1e-13
    assert np.abs(np.trace(P, axis1=1, axis2=2) - np.sum(np.conj(y) * x, axis=-1)).max() < 1e-13


def test_bf16_rounding_ties_to_even_and_library_agreement():
    one = 1.0
    assert precision.round_bf16(np.array([one + 2.0 ** -8]))[0] == 1.0          # tie -> even
    assert precision.round_bf16(np.array([one + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    assert precision.round_bf16(np.array([-(one + 2.0 ** -8 + 2.0 ** -20)]))[0] == -(1 + 2.0 ** -7)
    torch = pytest.importorskip("torch")
    x = synth.rng(16).standard_normal(10000).astype(np.float32).astype(np.float64)
    lib = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(precision.round_bf16(x), lib)


def test_fp16_fp32_rounding():
    x = np.array([1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 1.0 + 2.0 ** -24])
    assert np.array_equal(precision.round_real(x, "f16"), [1.0, 1.0 + 2.0 ** -9, 1.0])
    assert np.array_equal(precision.round_real(x, "f32"), [1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 1.0])


def test_third_row_reconstruction():
    U = synth.haar_su3(synth.rng(17), 1000)
    r2 = precision.third_row(U[:, 0], U[:, 1])
    assert np.abs(r2 - U[:, 2]).max() < 1e-14
    assert np.abs(precision.quantize_links(U, "f64", 12) - U).max() < 1e-14
    # compressed reduced-precision links are still close to the original
    Q = precision.quantize_links(U, "bf16", 12)
    assert np.abs(Q - U).max() < 2e-2
