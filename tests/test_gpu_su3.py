"""Parity of the batched SU(3) products (Table 1 routines) with the oracle."""
import numpy as np
import pytest

import synth
from oracle import su3
from helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    import paper_1309_0551_gb300 as lq
    return lq


@pytest.fixture(scope="module")
def ctx(lq):
    return lq.Context(0)


def _dev(a, prec):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if prec == "f64" else t.to(torch.complex64)).cuda()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", [1024, 1000, 1, 0, 300001])
@pytest.mark.parametrize("adjA,adjB", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_su3_mul_batch(lq, ctx, prec, n, adjA, adjB):
    import torch
    A, B = synth.su3_pairs(max(n, 1), seed=2)
    A, B = A[:n], B[:n]
    Ad, Bd = _dev(A, prec), _dev(B, prec)
    C = torch.empty_like(Ad)
    lq.su3_mul_batch(ctx, Ad, Bd, C, n, adjA, adjB)
    torch.cuda.synchronize()
    if n == 0:
        return
    Aq = Ad.cpu().to(torch.complex128).numpy()
    Bq = Bd.cpu().to(torch.complex128).numpy()
    opA = su3.adj(Aq) if adjA else Aq
    opB = su3.adj(Bq) if adjB else Bq
    ref = su3.mult_su3_nn(opA, opB)
    err = rel_l2(C.cpu().to(torch.complex128).numpy(), ref)
    assert err < (1e-14 if prec == "f64" else 1e-6)
    # named routines of Table 1
    if (adjA, adjB) == (1, 0):
        assert rel_l2(C.cpu().to(torch.complex128).numpy(), su3.mult_su3_an(Aq, Bq)) < (1e-14 if prec == "f64" else 1e-6)
    if (adjA, adjB) == (0, 1):
        assert rel_l2(C.cpu().to(torch.complex128).numpy(), su3.mult_su3_na(Aq, Bq)) < (1e-14 if prec == "f64" else 1e-6)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", [4096, 777, 1])
@pytest.mark.parametrize("adj", [0, 1])
def test_su3_matvec_batch(lq, ctx, prec, n, adj):
    import torch
    A = synth.haar_su3(synth.rng(71), n)
    b = synth.complex_gaussian(synth.rng(72), (n, 3))
    Ad, bd = _dev(A, prec), _dev(b, prec)
    c = torch.empty_like(bd)
    lq.su3_matvec_batch(ctx, Ad, bd, c, n, adj)
    torch.cuda.synchronize()
    Aq = Ad.cpu().to(torch.complex128).numpy()
    bq = bd.cpu().to(torch.complex128).numpy()
    ref = su3.mult_adj_su3_mat_vec(Aq, bq) if adj else su3.mult_su3_mat_vec(Aq, bq)
    assert rel_l2(c.cpu().to(torch.complex128).numpy(), ref) < (1e-14 if prec == "f64" else 1e-6)


def _upload(z, prec):
    """complex128 numpy array -> CUDA tensor of the storage format ``prec``, rounded once
    from FP64 by the oracle (so the kernel and the reference see the same values)."""
    import torch
    from oracle.precision import round_complex
    q = round_complex(z, prec)
    t = torch.from_numpy(np.ascontiguousarray(q))
    if prec == "f64":
        return t.cuda()
    if prec == "f32":
        return t.to(torch.complex64).cuda()
    dt = torch.bfloat16 if prec == "bf16" else torch.float16
    return torch.view_as_real(t).to(dt).contiguous().cuda()


@pytest.mark.parametrize("mat,recon,vec", [("f64", 18, "f64"), ("f64", 12, "f64"), ("f32", 18, "f32"),
                                           ("f32", 12, "f32"), ("bf16", 18, "bf16"), ("bf16", 12, "bf16"),
                                           ("bf16", 12, "f32"), ("f16", 18, "f16"), ("f16", 12, "f16")])
@pytest.mark.parametrize("n", [4096, 777, 1, 0])
@pytest.mark.parametrize("adj", [0, 1])
def test_su3_matvec_batch_ex_formats(lq, ctx, mat, recon, vec, n, adj):
    """mult_su3_mat_vec / mult_adj_su3_mat_vec (Table 1, Eqs. (1.1)-(2.3)) with 16-bit and
    12-real storage: against the oracle applied to the same rounded operands (row 2 of a
    12-real matrix rebuilt from the rounded rows 0 and 1), within one output rounding."""
    import torch
    from helpers import from_device_vec, empty_vec, store_tolerance
    from oracle.precision import quantize_links, round_complex
    m = max(n, 1)
    A = synth.haar_su3(synth.rng(73), m)[:n]
    b = synth.complex_gaussian(synth.rng(74), (m, 3))[:n]
    Ad = _upload(np.ascontiguousarray(A[:, :2, :] if recon == 12 else A), mat)
    bd = _upload(b, vec)
    c = empty_vec((n, 3), vec)
    lq.su3_matvec_batch_ex(ctx, Ad, bd, c, n, adj, mat, recon, vec)
    ctx.sync()
    if n == 0:
        return
    Aq = quantize_links(A, mat, recon)
    bq = round_complex(b, vec)
    ref = su3.mult_adj_su3_mat_vec(Aq, bq) if adj else su3.mult_su3_mat_vec(Aq, bq)
    assert rel_l2(from_device_vec(c), ref) < store_tolerance(vec)
    # and against the unrounded FP64 operation: the error the storage format costs
    exact = su3.mult_adj_su3_mat_vec(A, b) if adj else su3.mult_su3_mat_vec(A, b)
    u = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}
    assert rel_l2(from_device_vec(c), exact) < 8 * (u[mat] + u[vec]) + 1e-13


def test_su3_matvec_batch_ex_rejects_bad_pairs(lq, ctx):
    import torch
    A = torch.zeros((4, 3, 3), dtype=torch.complex128, device="cuda")
    b = torch.zeros((4, 3), dtype=torch.complex64, device="cuda")
    c = torch.empty_like(b)
    with pytest.raises(lq.LQError, match="INVALID_ARG"):
        lq.su3_matvec_batch_ex(ctx, A, b, c, 4, 0, "f64", 18, "f32")
    with pytest.raises(lq.LQError, match="INVALID_ARG"):
        lq.su3_matvec_batch_ex(ctx, A, b, c, 4, 0, "f32", 14, "f32")
