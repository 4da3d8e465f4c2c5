"""The t-split decomposition on one GPU: several sub-domains in one process (LocalComm,
faces moved by device copies), each applying dslash_eo_halo with its ghost faces and ghost
links.  Gathered, the parts equal the whole-lattice oracle: FP64 to 1e-13, reduced storage
within one output rounding of the oracle on the rounded links; the split-lattice FP64 CG
(inner products summed over the parts) reaches the oracle's true residual 1e-10."""
import numpy as np
import pytest

import synth
from oracle import dslash as odslash
from oracle.precision import quantize_links
from helpers import rel_l2, store_tolerance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lq():
    import paper_1309_0551_gb300 as lq
    return lq


@pytest.fixture(scope="module")
def ctx(lq):
    return lq.Context(0)


def _parts(lq, ctx, U, dims, P, prec, recon):
    import torch
    from paper_1309_0551_gb300 import halo
    split = halo.TSplit(dims, P)
    comm = halo.LocalComm(P)
    Ud = torch.from_numpy(U).cuda()
    U_parts = [split.gauge_part(Ud, k) for k in range(P)]
    gauges = [lq.lq_gauge_pack(ctx, split.local, u, prec, recon) for u in U_parts]
    halo.setup_halo(ctx, comm, split, gauges, U_parts)
    return split, comm, halo.LibOps(ctx, gauges), halo


@pytest.mark.parametrize("dims,P", [((4, 4, 4, 8), 2), ((6, 4, 2, 8), 4), ((4, 2, 4, 4), 1), ((8, 8, 4, 12), 3)])
@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f64", 12), ("f32", 12), ("bf16", 12), ("f32", 18)])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_split_dslash_equals_whole_lattice(lq, ctx, dims, P, prec, recon, nrhs):
    import torch
    U = synth.gauge_field(dims, "haar", seed=711)
    chi = synth.fermion_field(dims, nrhs, 712)
    split, comm, ops, halo = _parts(lq, ctx, U, dims, P, prec, recon)
    ct = torch.complex128 if prec == "f64" else torch.complex64
    Uq = quantize_links(U, prec, recon)
    for par in (0, 1):
        inp = [split.vec_part(torch.from_numpy(chi).to(ct).cuda(), k) for k in range(P)]
        out = [torch.empty_like(v) for v in inp]
        halo.apply_dslash(ops, comm, split, inp, out, par)
        got = torch.cat(out, dim=1).cpu().to(torch.complex128).numpy()
        src = torch.from_numpy(chi).to(ct).to(torch.complex128).numpy()
        for r in range(nrhs):
            ref = odslash.dslash_eo(Uq, src[r], dims, par)
            tol = 1e-13 if prec == "f64" else store_tolerance("f32")
            assert rel_l2(got[r], ref) < tol, (par, r)


def test_split_cg_fp64(lq, ctx):
    import torch
    dims, mass, P = (8, 8, 8, 8), 0.1, 2
    U = synth.gauge_field(dims, "haar", seed=713)
    b = synth.fermion_field(dims, 1, 714)
    split, comm, ops, halo = _parts(lq, ctx, U, dims, P, "f64", 18)
    bp = [split.vec_part(torch.from_numpy(b).cuda(), k) for k in range(P)]
    x, info = halo.cg(ops, comm, split, bp, mass, tol=1e-10, maxiter=2000)
    xg = torch.cat(x, dim=1).cpu().numpy()[0]
    r = b[0] - odslash.normal_op(U, xg, mass, dims)
    assert info["true_rel_resid"] <= 1e-10
    assert np.linalg.norm(r) / np.linalg.norm(b[0]) <= 1.05e-10
    # the whole-lattice library solve takes the same iteration (up to summation order)
    hi = lq.lq_gauge_pack(ctx, dims, torch.from_numpy(U).cuda(), "f64", 18)
    bd = torch.from_numpy(b).cuda()
    xd = torch.empty_like(bd)
    st = lq.cg_solve(ctx, hi, None, mass, bd, xd, 1, tol=1e-10, maxiter=2000)
    assert abs(st[0]["iters"] - info["iters"]) <= 20
    assert rel_l2(xg, xd[0].cpu().numpy()) < 1e-8


def test_vector_kernels(lq, ctx):
    import torch
    g = synth.rng(715)
    for dt, tol in ((torch.complex128, 1e-14), (torch.complex64, 1e-6)):
        x = torch.from_numpy(synth.complex_gaussian(g, (3, 1000, 3))).to(dt).cuda()
        y = torch.from_numpy(synth.complex_gaussian(g, (3, 1000, 3))).to(dt).cuda()
        res = torch.empty(1, dtype=torch.float64, device="cuda")
        lq.lq_vec_dot(ctx, x, y, res)
        xn, yn = x.cpu().to(torch.complex128).numpy(), y.cpu().to(torch.complex128).numpy()
        ref = np.vdot(xn, yn).real
        assert abs(float(res) - ref) < 1e-12 * np.linalg.norm(xn) * np.linalg.norm(yn)
        lq.lq_vec_axpby(ctx, 0.5, x, -2.0, y)
        assert rel_l2(y.cpu().to(torch.complex128).numpy(), 0.5 * xn - 2.0 * yn) < tol
