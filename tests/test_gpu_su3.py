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
