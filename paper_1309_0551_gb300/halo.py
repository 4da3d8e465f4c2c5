"""Lattices split in t across processes or GPUs (the method's parallel mode, Table 4):
sub-domain geometry, face exchange, and the FP64 CG on a split lattice.

Host orchestration only.  The arithmetic runs in the library's kernels (``dslash_eo_halo``,
``lq_vec_axpby``, ``lq_vec_dot``, through ``LibOps``); this module moves faces between
sub-domains and sums inner products across them.  Two communicators:

* ``DistComm``: one sub-domain per rank of a ``torch.distributed`` process group (NCCL for
  GPU ranks, gloo for CPU ranks): faces by point-to-point send/recv to the t neighbours,
  inner products by ``all_reduce``;
* ``LocalComm``: every sub-domain in this process (several sub-domains on one device):
  faces by copies, sums in process.

Geometry (``lqcd.h``, "t-split domain decomposition"): Lt is cut into P parts of Lt/P
(even) slices; part k is the lattice (Lx, Ly, Lz, Lt/P) of the global slices
[k Lt/P, (k+1) Lt/P); its one-parity fields are the contiguous ranges
[k Vh/P, (k+1) Vh/P) of the global ones; a face is the first or last Vs/2 sites
(Vs = Lx Ly Lz) of a part's array.
"""
from __future__ import annotations

import math


class TSplit:
    def __init__(self, dims, nparts: int):
        Lx, Ly, Lz, Lt = (int(d) for d in dims)
        if nparts < 1 or Lt % nparts or (Lt // nparts) % 2:
            raise ValueError(f"Lt = {Lt} must split into {nparts} parts of an even number of slices")
        self.dims = (Lx, Ly, Lz, Lt)
        self.P = nparts
        self.local = (Lx, Ly, Lz, Lt // nparts)
        self.Vs = Lx * Ly * Lz
        self.Vsh = self.Vs // 2
        self.Vh_local = self.Vsh * (Lt // nparts)

    def gauge_part(self, U, k):
        """Links of part k from a canonical (4, V, 3, 3) field (a contiguous copy)."""
        n = self.Vs * self.local[3]
        return U[:, k * n:(k + 1) * n].contiguous()

    def vec_part(self, v, k):
        """Part k of a one-parity field (..., Vh, 3) (a contiguous copy)."""
        return v[..., k * self.Vh_local:(k + 1) * self.Vh_local, :].contiguous()

    def last_slice_links(self, U_part):
        """U_t on the last slice of a part: the ghost links of the next part, (Vs, 3, 3)."""
        return U_part[3, -self.Vs:].contiguous()

    def faces(self, v_part):
        """(first-slice face, last-slice face) of a part's field, contiguous copies."""
        return v_part[..., :self.Vsh, :].contiguous(), v_part[..., -self.Vsh:, :].contiguous()


def _real(t):
    import torch
    return torch.view_as_real(t) if t.is_complex() else t


class LocalComm:
    """All P sub-domains in this process: faces by copies, sums in process."""

    def __init__(self, nparts: int):
        self.P = nparts
        self.parts = list(range(nparts))

    def exchange(self, lo, hi):
        """lo[j], hi[j]: first- and last-slice faces of the owned parts.  Returns, per part,
        (ghost_bwd, ghost_fwd) = (previous part's last face, next part's first face)."""
        P = self.P
        return [hi[(k - 1) % P].clone() for k in range(P)], [lo[(k + 1) % P].clone() for k in range(P)]

    def allreduce(self, vals):
        """Sum of the owned parts' values (tensors of one element) as a float."""
        return math.fsum(float(v) for v in vals)


class DistComm:
    """One sub-domain per rank of a torch.distributed group (the rank's part index)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.P = dist.get_world_size(group)
        self.parts = [self.rank]

    def exchange(self, lo, hi):
        import torch
        lo, hi = lo[0], hi[0]
        if self.P == 1:
            return [hi.clone()], [lo.clone()]
        bwd, fwd = torch.empty_like(hi), torch.empty_like(lo)
        prev, nxt = (self.rank - 1) % self.P, (self.rank + 1) % self.P
        d = self.dist
        g = lambda r: r if self.group is None else d.get_global_rank(self.group, r)  # noqa: E731
        # Order: a rank sends hi (to next) before lo (to prev) and receives bwd (from prev)
        # before fwd (from next); with two parts, prev == next, and messages between one
        # pair of ranks match in order: hi -> bwd, lo -> fwd.
        ops = [d.P2POp(d.isend, _real(hi), g(nxt), self.group), d.P2POp(d.isend, _real(lo), g(prev), self.group),
               d.P2POp(d.irecv, _real(bwd), g(prev), self.group), d.P2POp(d.irecv, _real(fwd), g(nxt), self.group)]
        for w in d.batch_isend_irecv(ops):
            w.wait()
        return [bwd], [fwd]

    def allreduce(self, vals):
        t = vals[0].clone()
        self.dist.all_reduce(t, group=self.group)
        return float(t)


class LibOps:
    """Per-part operations in the library's kernels; ``gauges[j]`` is the packed gauge of
    owned part j with its ghost links set (``setup_halo``)."""

    def __init__(self, ctx, gauges, stream=None):
        from . import lq_vec_axpby, lq_vec_dot, dslash_eo_halo
        self.ctx, self.gauges, self.stream = ctx, gauges, stream
        self._axpby, self._dot, self._dslash = lq_vec_axpby, lq_vec_dot, dslash_eo_halo

    def dslash(self, j, inp, ghost_bwd, ghost_fwd, out, out_parity, a1=0.0, w1=None, c=1.0):
        nrhs = inp.shape[0] if inp.dim() == 3 else 1
        self._dslash(self.ctx, self.gauges[j], inp, ghost_bwd, ghost_fwd, out, out_parity, nrhs, a1, w1, c,
                     stream=self.stream)

    def dot(self, x, y):
        import torch
        r = torch.empty(1, dtype=torch.float64, device=x.device)
        self._dot(self.ctx, x, y, r, stream=self.stream)
        return r

    def axpby(self, a, x, b, y):
        self._axpby(self.ctx, a, x, b, y, stream=self.stream)


def setup_halo(ctx, comm, split, gauges, U_parts, stream=None):
    """Give every owned part's gauge the previous part's last-slice U_t (one exchange)."""
    from . import lq_gauge_set_halo
    links = [split.last_slice_links(U) for U in U_parts]
    bwd, _ = comm.exchange(links, links)
    for g, gl in zip(gauges, bwd):
        lq_gauge_set_halo(ctx, g, gl, stream)


def apply_dslash(ops, comm, split, inp, out, out_parity, a1=0.0, w1=None, c=1.0):
    """out[j] = a1 w1[j] + c D inp[j] on every owned part, after the face exchange."""
    lo, hi = zip(*[split.faces(v) for v in inp])
    bwd, fwd = comm.exchange(list(lo), list(hi))
    for j in range(len(inp)):
        ops.dslash(j, inp[j], bwd[j], fwd[j], out[j], out_parity, a1, None if w1 is None else w1[j], c)


def normal_op(ops, comm, split, p, out, tmp, mass):
    """out = (m^2 - D_eo D_oe) p on the even sites of every owned part (tmp: odd-site work)."""
    apply_dslash(ops, comm, split, p, tmp, 1)
    apply_dslash(ops, comm, split, tmp, out, 0, a1=mass * mass, w1=p, c=-1.0)


def cg(ops, comm, split, b, mass, tol=1e-10, maxiter=10000, max_restarts=5):
    """FP64 CG on M = m^2 - D_eo D_oe over a split lattice from x = 0, the iteration of
    cg_solve's FP64 solve: the iterated residual triggers an FP64 true-residual check, and
    a residual replacement keeps p with the Polak-Ribiere beta.  Inner products are
    summed across the parts (``comm.allreduce``).  ``b``: the owned parts' sources.
    Returns (x parts, dict(iters, true_rel_resid, restarts))."""
    import torch
    J = range(len(b))

    def dot(xs, ys):
        return comm.allreduce([ops.dot(u, v) for u, v in zip(xs, ys)])

    x = [torch.zeros_like(v) for v in b]
    r = [v.clone() for v in b]
    p = [v.clone() for v in b]
    Ap = [torch.empty_like(v) for v in b]
    tmp = [torch.empty_like(v) for v in b]
    bb = dot(b, b)
    if bb == 0.0:
        return x, dict(iters=0, true_rel_resid=0.0, restarts=0)
    rr = bb
    it = restarts = 0
    while it < maxiter:
        normal_op(ops, comm, split, p, Ap, tmp, mass)
        alpha = rr / dot(p, Ap)
        for j in J:
            ops.axpby(alpha, p[j], 1.0, x[j])
            ops.axpby(-alpha, Ap[j], 1.0, r[j])
        rr_new = dot(r, r)
        it += 1
        beta = rr_new / rr
        if rr_new <= tol * tol * bb:
            rt = [torch.empty_like(v) for v in b]
            normal_op(ops, comm, split, x, rt, tmp, mass)
            for j in J:
                ops.axpby(1.0, b[j], -1.0, rt[j])              # rt = b - M x
            trr = dot(rt, rt)
            if math.sqrt(trr / bb) <= tol or restarts >= max_restarts:
                break
            restarts += 1
            for j in J:
                ops.axpby(alpha, Ap[j], 1.0, r[j])             # r_k = r + alpha Ap
            beta = max(0.0, (trr - dot(r, rt)) / rr)
            r = rt
            rr_new = trr
        for j in J:
            ops.axpby(1.0, r[j], beta, p[j])                   # p = r + beta p
        rr = rr_new
    rt = [torch.empty_like(v) for v in b]
    normal_op(ops, comm, split, x, rt, tmp, mass)
    for j in J:
        ops.axpby(1.0, b[j], -1.0, rt[j])
    return x, dict(iters=it, true_rel_resid=math.sqrt(dot(rt, rt) / bb), restarts=restarts)
