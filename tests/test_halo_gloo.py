"""Host logic of the t-split decomposition (paper_1309_0551_gb300.halo) on the CPU: the face
exchange and the split-lattice CG, run with two gloo ranks (DistComm) and with several parts
in one process (LocalComm), each part's operator being the oracle's sub-domain Dslash.  The
gathered results equal the whole-lattice oracle: the operator to rounding, the CG solution
to its tolerance."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIMS, MASS = (4, 4, 2, 8), 0.4


class OracleOps:
    """Per-part operations of the halo CG done by the oracle (numpy) on CPU tensors."""

    def __init__(self, U_parts, dims_loc):
        self.U = U_parts
        self.ghost_Ut = [None] * len(U_parts)
        self.dims = dims_loc

    def dslash(self, j, inp, ghost_bwd, ghost_fwd, out, out_parity, a1=0.0, w1=None, c=1.0):
        import torch
        from oracle import partition
        d = partition.dslash_eo_halo(self.U[j], self.ghost_Ut[j], inp.numpy()[0], ghost_bwd.numpy()[0],
                                     ghost_fwd.numpy()[0], self.dims, out_parity)
        res = c * d + (a1 * w1.numpy()[0] if w1 is not None else 0.0)
        out.copy_(torch.from_numpy(res[None]))

    def dot(self, x, y):
        import torch
        return torch.tensor([float(np.vdot(x.numpy(), y.numpy()).real)], dtype=torch.float64)

    def axpby(self, a, x, b, y):
        y.copy_(a * x + b * y)


def _setup(U, split, parts):
    import torch
    U_parts = [torch.from_numpy(U) for _ in parts]
    U_parts = [split.gauge_part(torch.from_numpy(U), k) for k in parts]
    ops = OracleOps([u.numpy() for u in U_parts], split.local)
    return U_parts, ops


def _run_parts(comm, split, U, chi, b):
    import torch
    from paper_1309_0551_gb300 import halo
    parts = comm.parts
    U_parts, ops = _setup(U, split, parts)
    links = [split.last_slice_links(u) for u in U_parts]
    bwd, _ = comm.exchange(links, links)
    for j in range(len(parts)):
        ops.ghost_Ut[j] = bwd[j].numpy()
    out = {}
    for par in (0, 1):
        inp = [split.vec_part(torch.from_numpy(chi), k) for k in parts]
        o = [torch.empty_like(v) for v in inp]
        halo.apply_dslash(ops, comm, split, inp, o, par)
        out[par] = [v.numpy() for v in o]
    bp = [split.vec_part(torch.from_numpy(b), k) for k in parts]
    x, info = halo.cg(ops, comm, split, bp, MASS, tol=1e-10, maxiter=500)
    return out, [v.numpy() for v in x], info


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    import synth
    from paper_1309_0551_gb300 import halo
    dist.init_process_group("gloo", rank=rank, world_size=world)
    U = synth.gauge_field(DIMS, "haar", seed=701)
    chi = synth.fermion_field(DIMS, 1, 702)
    b = synth.fermion_field(DIMS, 1, 703)
    comm = halo.DistComm()
    out, x, info = _run_parts(comm, halo.TSplit(DIMS, world), U, chi, b)
    q.put((rank, out, x, info))
    dist.barrier()
    dist.destroy_process_group()


def _check(outs, xs, infos, U, chi, b):
    from oracle import cg as ocg, dslash
    for par in (0, 1):
        got = np.concatenate(outs[par], axis=-2)[0]
        ref = dslash.dslash_eo(U, chi[0], DIMS, par)
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    x = np.concatenate(xs, axis=-2)[0]
    r = b[0] - dslash.normal_op(U, x, MASS, DIMS)
    assert np.linalg.norm(r) / np.linalg.norm(b[0]) <= 1.05e-10
    ref, rinfo = ocg.cg(U, b[0], MASS, DIMS, tol=1e-10)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-8
    for info in infos:
        assert info["true_rel_resid"] <= 1e-10 and abs(info["iters"] - rinfo["iters"]) <= 2


def test_two_gloo_ranks():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    U = synth.gauge_field(DIMS, "haar", seed=701)
    chi = synth.fermion_field(DIMS, 1, 702)
    b = synth.fermion_field(DIMS, 1, 703)
    outs = {par: [r[1][par][0] for r in res] for par in (0, 1)}
    _check(outs, [r[2][0] for r in res], [r[3] for r in res], U, chi, b)


@pytest.mark.parametrize("P", [1, 4])
def test_parts_in_one_process(P):
    pytest.importorskip("torch")
    import synth
    from paper_1309_0551_gb300 import halo
    U = synth.gauge_field(DIMS, "haar", seed=701)
    chi = synth.fermion_field(DIMS, 1, 702)
    b = synth.fermion_field(DIMS, 1, 703)
    out, x, info = _run_parts(halo.LocalComm(P), halo.TSplit(DIMS, P), U, chi, b)
    _check(out, x, [info], U, chi, b)
