#!/usr/bin/env python
"""Staggered Dslash throughput on one GB300 (GFLOP/s at 570 flops per site, HBM GB/s and
its fraction of the measured copy bandwidth), plus the CG time to a 1e-10 residual with
mixed precision against FP64.

Workload (one "step"): 100 applications of the full staggered Dslash D = D_eo + D_oe on a
16^3 x 32 lattice (two half-Dslash launches each: t = D_oe chi, out = D_eo t), links
exp(i 0.3 H) re-projected to SU(3), Gaussian vectors, seeded.  To keep the timed region
honest about HBM, the launches cycle over a ring of K device copies of the packed links
and vectors whose total size exceeds three times the L2 cache, so no launch finds its
links in L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec f32 --recon 18]
    python bench.py --impl reference       # the FP64 C++ oracle on the host cores

Under torchrun every rank runs its own replica (independent lattices, no collective on the
data path); the value is the flops of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Dslash GFLOP/s & HBM GB/s vs ~8 TB/s; mixed-prec CG time to 1e-10 vs FP64"
DIMS = (16, 16, 16, 32)
APPS = 100                 # Dslash applications per step
FLOPS_PER_SITE = 570
BYTES = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}
# GB300's nominal FP64 rate, 1.25 TFLOP/s (about two FP64 FMAs per SM and clock: 152 SMs at
# 2.07 GHz), for context; the FP64 kernels' ALU roofline divides by the rate measured on the
# device itself (lq_fp64_fma_rate, independent FMA chains on every SM).
FP64_NOMINAL_GFLOPS = 1250.0

# DRAM bytes per k_dslash launch from an ncu capture of the same workload (key: storage
# format), with the hash of the kernel sources it was taken on.  A changed kernel makes the
# figure stale and the bench reports null.
NCU_TRAFFIC = {
    # dram__bytes_read.sum + dram__bytes_write.sum of one k_dslash<f32,18,f32,1,1> launch
    # (block 64, grid 1024): 39,351,296 + 0 B
    "f32/18/f32/16x16x16x32/1": (39351296, "f81bd9b598756ec1"),
}
KERNEL_SOURCES = ("paper_1309_0551_gb300/csrc/dslash_args.cuh",
                  "paper_1309_0551_gb300/csrc/dslash_kernel.cuh",
                  "paper_1309_0551_gb300/csrc/dslash_site.cuh",
                  "paper_1309_0551_gb300/csrc/lqcd_internal.cuh",
                  "paper_1309_0551_gb300/csrc/tune.cuh")


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def site_bytes(prec, recon, vec, nrhs=1):
    """Algorithmic bytes per output site of a half Dslash: 8 links read once (shared by all
    right-hand sides), each input vector read once (its 8-fold neighbour reuse served on
    chip), each output written once."""
    return 8 * recon * BYTES[prec] + nrhs * 2 * 6 * BYTES[vec]


def parse():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--prec", default="f32", choices=["f64", "f32", "bf16", "f16"])
    p.add_argument("--recon", type=int, default=18, choices=[18, 12])
    p.add_argument("--vec", default=None, help="vector storage (default: f64 for f64 links, else f32)")
    p.add_argument("--lattice", default="16,16,16,32", help="Lx,Ly,Lz,Lt of the Dslash workload")
    p.add_argument("--nrhs", type=int, default=1, help="right-hand sides per Dslash launch")
    p.add_argument("--field", default="near_identity", choices=["near_identity", "haar"])
    p.add_argument("--streams", type=int, default=4,
                   help="independent applications in flight (graph branches)")
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--variants", default="all",
                   help="comma-separated variant groups: formats, l2_warm, 32c4, lone, improved, wilson, "
                        "multi_rhs, su3")
    p.add_argument("--no-cg", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cg-maxiter", type=int, default=20000,
                   help="iteration cap of the CG comparison (small values: short runs for profiling)")
    p.add_argument("--no-batched-force", action="store_true")
    return p.parse_args()


# ------------------------------------------------------------------ distributed -------

def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


def dist_init(world, use_cuda):
    if world <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group("nccl" if use_cuda else "gloo")
    return dist


def max_over_ranks(dist, value, device=None):
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks ------------

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.15)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                try:
                    rows.append((float(f[1]), float(f[2]), f[3], f[4:]))
                except ValueError:
                    pass
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for n, v in zip(names, r[3][1:]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ GPU arm -----------

def make_ring(lq, ctx, U_dev, dims, prec, recon, vec, K, seed=2, nrhs=1):
    import torch
    import synth
    Vh = synth.volume(dims) // 2
    chi = synth.fermion_field(dims, nrhs, seed=seed)
    gauges = [lq.lq_gauge_pack(ctx, dims, U_dev, prec, recon) for _ in range(K)]
    host = torch.from_numpy(chi)

    def vec_tensor(src=None):
        if vec == "f64":
            return (src.cuda() if src is not None else torch.empty((nrhs, Vh, 3), dtype=torch.complex128, device="cuda"))
        if vec == "f32":
            return (src.to(torch.complex64).cuda() if src is not None
                    else torch.empty((nrhs, Vh, 3), dtype=torch.complex64, device="cuda"))
        dt = torch.bfloat16 if vec == "bf16" else torch.float16
        if src is not None:
            return torch.view_as_real(src).to(dt).contiguous().cuda()
        return torch.empty((nrhs, Vh, 3, 2), dtype=dt, device="cuda")

    def ring_of(src=None):
        # the K copies as views of one contiguous tensor (a step's inputs or outputs move
        # between host and device as one copy)
        one = vec_tensor(src)
        whole = torch.empty((K,) + tuple(one.shape), dtype=one.dtype, device="cuda")
        if src is not None:
            whole.copy_(one.unsqueeze(0).expand_as(whole))
        return [whole[k] for k in range(K)]

    ins = ring_of(host)
    ts = ring_of()
    outs = ring_of()
    return gauges, ins, ts, outs


def ring_size(bytes_per_copy, l2_bytes, nstreams=4):
    """Copies so that the ring holds > 3x L2; a multiple of 2*nstreams, so that the
    applications that share a copy always run on the same stream (in order)."""
    m = 2 * nstreams
    k = max(m, -(-3 * l2_bytes // bytes_per_copy))
    return -(-k // m) * m


def run_step(lq, ctx, gauges, ins, ts, outs, vec_code, streams, apps=APPS, nrhs=1):
    """One step: `apps` applications of D.  Application a runs on streams[a % S] (the
    applications are independent; the two halves of one are ordered on its stream), and
    half-Dslash launch h uses ring copy h mod K.  Returns the number of launches."""
    K = len(gauges)
    S = len(streams)
    h = 0
    for a in range(apps):
        s = streams[a % S]
        c = h % K
        c2 = (h + 1) % K
        lq.dslash_eo(ctx, gauges[c], ins[c], ts[c], 1, nrhs, vec_code, s)      # t = D_oe chi
        lq.dslash_eo(ctx, gauges[c2], ts[c], outs[c], 0, nrhs, vec_code, s)    # out = D_eo t
        h += 2
    return 2 * apps


class GraphStep:
    """A step captured once as a CUDA graph (after an eager run that tunes launch shapes)
    and replayed; `fn(streams)` issues the step's launches on the given streams."""

    def __init__(self, torch, fn, nstreams=2):
        self.torch = torch
        fn([torch.cuda.current_stream()])          # eager: tunes, checks
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        side = [torch.cuda.Stream() for _ in range(nstreams - 1)]
        with torch.cuda.graph(self.graph):
            main = torch.cuda.current_stream()
            for s in side:
                s.wait_stream(main)
            self.launches = fn([main] + side)
            for s in side:
                main.wait_stream(s)
        torch.cuda.synchronize()

    def __call__(self):
        self.graph.replay()
        return self.launches


def time_steps(torch, fn, steps, warmup, stream, dist=None, device=None, sampler=None):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if sampler:
        sampler.start()
    e0.record(stream)
    launches = 0
    for _ in range(steps):
        launches += fn()
    e1.record(stream)
    e1.synchronize()
    clocks = sampler.stop() if sampler else None
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    return max_over_ranks(dist, ms, device), launches, clocks


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_model() -> str:
    """The host CPU's model name (lscpu / /proc/cpuinfo), or the platform's machine name."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def _oracle_dslash_rate(cxx, U, chi, dims, threads, seconds):
    """Half-Dslash applications of the C++ oracle on `threads` threads for about `seconds`:
    (GFLOP/s, applications, elapsed)."""
    Vh = synth_volume(dims) // 2
    cxx.dslash_eo(U, chi, dims, 1, threads)   # warm-up (pages, thread pool)
    n, t0 = 0, time.perf_counter()
    while True:
        cxx.dslash_eo(U, chi, dims, 1 - (n & 1), threads)
        n += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    return n * Vh * FLOPS_PER_SITE / dt / 1e9, n, dt


def synth_volume(dims):
    import synth
    return synth.volume(dims)


def cpu_baseline(dims, seconds=4.0, fp64_cg_iters=None):
    """The FP64 C++ oracle (plain loops, OpenMP over sites) timed on the host: half-Dslash
    applications at the benchmark's lattice size on one core and on every core (~`seconds`
    each), and 50 iterations of its FP64 CG at 32^4 on every core (s/iteration; the time to
    solution is extrapolated with the GPU's FP64 iteration count when given)."""
    import synth
    from oracle import cxx
    U = synth.gauge_field(dims, "near_identity", seed=3, eps=0.3)
    chi = synth.fermion_field(dims, 1, seed=2)[0]
    nproc = os.cpu_count() or 1
    threads = min(nproc, cxx.max_threads())
    one, n1, dt1 = _oracle_dslash_rate(cxx, U, chi, dims, 1, seconds)
    allc, na, dta = _oracle_dslash_rate(cxx, U, chi, dims, threads, seconds)
    d4 = (32, 32, 32, 32)
    U4 = synth.gauge_field(d4, "haar", seed=4)
    b4 = synth.fermion_field(d4, 1, seed=5)[0]
    t0 = time.perf_counter()
    _, info = cxx.cg(U4, b4, 0.01, d4, tol=1e-30, maxiter=50, max_restarts=0, threads=threads)
    s_it = (time.perf_counter() - t0) / info["iters"]
    cg = {"workload": "32^4 Haar, m 0.01: FP64 CG of the C++ oracle, 50 iterations", "threads": threads,
          "s_per_iter": round(s_it, 4)}
    if fp64_cg_iters:
        cg["extrapolated_seconds_to_1e-10"] = round(s_it * fp64_cg_iters, 1)
        cg["extrapolated_with_iters"] = fp64_cg_iters
    return {"value": round(allc, 3), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
            "cpu": cpu_model(), "nproc": nproc,
            "sample": f"{na} half-Dslash applications of the FP64 C++ oracle on the "
                      f"{'x'.join(map(str, dims))} lattice on {threads} threads ({dta:.1f} s)",
            "single_core": {"value": round(one, 3), "unit": "GFLOP/s", "cores": 1,
                            "sample": f"{n1} half-Dslash applications on 1 thread ({dt1:.1f} s)"},
            "cg_32c4": cg}


def run_variants(lq, ctx, torch, U_dev, l2, stream, nstreams, groups="all", fp64_peak=FP64_NOMINAL_GFLOPS):
    """The per-format, operator and SU(3)-batch lines; `groups` (comma-separated, or "all")
    picks among formats, l2_warm, 32c4, lone, improved, wilson, multi_rhs, su3."""
    import synth
    sel = set(groups.split(","))

    def want(name):
        return "all" in sel or name in sel

    out = {}
    forms = [("f64", 18, "f64"), ("f64", 12, "f64"), ("f32", 18, "f32"), ("f32", 12, "f32"),
             ("bf16", 18, "bf16"), ("bf16", 12, "bf16"), ("f16", 12, "f16")]
    peak, _ = measured_peak()
    Vh = (DIMS[0] * DIMS[1] * DIMS[2] * DIMS[3]) // 2
    if want("formats"):
        # the error each storage format costs: one half Dslash of the ring's input against the
        # library's FP64 operator (FP64 links and vectors, pinned to the oracle at 1e-13 by the
        # tests) applied to the unrounded input
        chi64 = torch.from_numpy(synth.fermion_field(DIMS, 1, seed=2)).cuda()
        g64 = lq.lq_gauge_pack(ctx, DIMS, U_dev, "f64", 18)
        ref64 = torch.empty_like(chi64)
        lq.dslash_eo(ctx, g64, chi64, ref64, 1, 1, lq.LQ_F64)
        torch.cuda.synchronize()
        del g64

        def as_c128(t):
            if t.is_complex():
                return t.to(torch.complex128)
            return torch.view_as_complex(t.float().contiguous()).to(torch.complex128)

        for prec, recon, vec in forms:
            sb = site_bytes(prec, recon, vec)
            K = ring_size(Vh * sb, l2, nstreams)
            gauges, ins, ts, outs = make_ring(lq, ctx, U_dev, DIMS, prec, recon, vec, K)
            vc = lq.PREC[vec]
            g = GraphStep(torch, lambda ss: run_step(lq, ctx, gauges, ins, ts, outs, vc, ss, APPS), nstreams)
            ms, launches, _ = time_steps(torch, g, 10, 3, stream)
            del g
            us = ms * 1000.0 / launches
            gbs = Vh * sb / us / 1e3
            lq.dslash_eo(ctx, gauges[0], ins[0], ts[0], 1, 1, vc)
            torch.cuda.synchronize()
            err = float(torch.linalg.vector_norm(as_c128(ts[0]) - ref64) / torch.linalg.vector_norm(ref64))
            out[f"{prec}/{recon}/{vec}"] = {"gflops": round(Vh * FLOPS_PER_SITE / us / 1e3, 1),
                                           "gbs": round(gbs, 1), "frac": round(gbs / peak, 3),
                                           "us_per_half": round(us, 2), "bytes_per_site": sb, "ring": K,
                                           "rel_err_vs_fp64": float("%.3g" % err)}
            del gauges, ins, ts, outs
            torch.cuda.empty_cache()
    if want("l2_warm"):
        # FP32-18 with one copy of links and vectors (40.9 MB, L2-resident): the L2-warm number
        # beside the flushed ones above; "frac" is still against the HBM copy bandwidth
        sb = site_bytes("f32", 18, "f32")
        gauges, ins, ts, outs = make_ring(lq, ctx, U_dev, DIMS, "f32", 18, "f32", 1)
        K = 2 * nstreams
        gauges, ins, ts, outs = gauges * K, ins * K, [ts[0]] * K, [outs[0]] * K
        g = GraphStep(torch, lambda ss: run_step(lq, ctx, gauges, ins, ts, outs, lq.PREC["f32"], ss, APPS), nstreams)
        ms, launches, _ = time_steps(torch, g, 10, 3, stream)
        del g
        us = ms * 1000.0 / launches
        gbs = Vh * sb / us / 1e3
        out["f32/18/f32/l2_warm"] = {"gflops": round(Vh * FLOPS_PER_SITE / us / 1e3, 1), "gbs": round(gbs, 1),
                                     "frac": round(gbs / peak, 3), "us_per_half": round(us, 2), "bytes_per_site": sb,
                                     "ring": 1}
        del gauges, ins, ts, outs
        torch.cuda.empty_cache()
    if want("32c4"):
        # FP32 and BF16 at 32^4 (109-327 MB per copy: every launch reads its links from HBM)
        d4 = (32, 32, 32, 32)
        Vh4 = synth.volume(d4) // 2
        U4 = torch.from_numpy(synth.gauge_field(d4, "near_identity", seed=3, eps=0.3)).cuda()
        for prec, recon, vec in (("f32", 18, "f32"), ("f32", 12, "f32"), ("bf16", 18, "bf16"), ("bf16", 12, "bf16")):
            sb = site_bytes(prec, recon, vec)
            K = ring_size(Vh4 * sb, l2, nstreams)
            gauges, ins, ts, outs = make_ring(lq, ctx, U4, d4, prec, recon, vec, K)
            vc = lq.PREC[vec]
            g = GraphStep(torch, lambda ss: run_step(lq, ctx, gauges, ins, ts, outs, vc, ss, APPS), nstreams)
            ms, launches, _ = time_steps(torch, g, 5, 3, stream)
            del g
            us = ms * 1000.0 / launches
            gbs = Vh4 * sb / us / 1e3
            out[f"{prec}/{recon}/{vec}/32x32x32x32"] = {"gflops": round(Vh4 * FLOPS_PER_SITE / us / 1e3, 1),
                                                      "gbs": round(gbs, 1), "frac": round(gbs / peak, 3),
                                                      "us_per_half": round(us, 2), "bytes_per_site": sb, "ring": K}
            del gauges, ins, ts, outs
            torch.cuda.empty_cache()
        del U4
        torch.cuda.empty_cache()
    if want("lone"):
        # one stream: each half Dslash waits for the previous one (the way a solver issues
        # them), so a launch's ramp-up and tail are not hidden by other launches in flight;
        # shapes tuned for lone launches (a context of its own, tuning mode 1)
        lctx = lq.Context(torch.cuda.current_device())
        lctx.set_tuning(1)
        for prec, recon, vec, dims in (("f32", 18, "f32", DIMS), ("bf16", 12, "bf16", DIMS),
                                       ("f32", 12, "f32", (32, 32, 32, 32)),
                                       ("bf16", 12, "bf16", (32, 32, 32, 32))):
            Vhl = synth.volume(dims) // 2
            Ul = U_dev if dims == DIMS else torch.from_numpy(
                synth.gauge_field(dims, "near_identity", seed=3, eps=0.3)).cuda()
            sb = site_bytes(prec, recon, vec)
            K = ring_size(Vhl * sb, l2, 1)
            gauges, ins, ts, outs = make_ring(lq, lctx, Ul, dims, prec, recon, vec, K)
            vc = lq.PREC[vec]
            g = GraphStep(torch, lambda ss: run_step(lq, lctx, gauges, ins, ts, outs, vc, ss, APPS), 1)
            ms, launches, _ = time_steps(torch, g, 10, 3, stream)
            del g
            us = ms * 1000.0 / launches
            gbs = Vhl * sb / us / 1e3
            dkey = f"g={prec}/{recon} v={vec} dims={'x'.join(map(str, dims))} nrhs=1"
            out[f"lone/{prec}/{recon}/{vec}/{'x'.join(map(str, dims))}"] = {
                "gflops": round(Vhl * FLOPS_PER_SITE / us / 1e3, 1), "gbs": round(gbs, 1),
                "frac": round(gbs / peak, 3), "us_per_half": round(us, 2), "bytes_per_site": sb, "ring": K,
                "streams": 1, "launch_shape": [l for l in lctx.tune_report().splitlines() if dkey in l]}
            del gauges, ins, ts, outs, Ul
            torch.cuda.empty_cache()
        del lctx
    if want("improved"):
        # improved staggered Dslash: fat one-hop + Naik three-hop links (16 hops, 1146 flops)
        for prec in ("f32", "bf16"):
            vec = "f32" if prec == "f32" else "bf16"
            sb = 2 * 8 * 18 * BYTES[prec] + 12 * BYTES[vec]
            K = ring_size(Vh * sb, l2, nstreams)
            Ld = torch.empty_like(U_dev)
            lq.lq_long_links(ctx, DIMS, U_dev, -1.0 / 24, Ld)
            fats = [lq.lq_gauge_pack(ctx, DIMS, U_dev, prec, 18) for _ in range(K)]
            lngs = [lq.lq_gauge_pack(ctx, DIMS, Ld, prec, 18) for _ in range(K)]
            del Ld
            _, ins, ts, outs = make_ring(lq, ctx, U_dev, DIMS, "f32", 12, vec, 1)
            ins, ts, outs = ins * K, [ts[0]] * K, [outs[0]] * K
            vc = lq.PREC[vec]

            def istep(ss, fats=fats, lngs=lngs, ins=ins, vc=vc):
                h = 0
                for a in range(APPS):
                    s_ = ss[a % len(ss)]
                    c, c2 = h % K, (h + 1) % K
                    lq.dslash_eo_improved(ctx, fats[c], lngs[c], ins[c], itmp[a % len(ss)], 1, 1, vc, s_)
                    lq.dslash_eo_improved(ctx, fats[c2], lngs[c2], itmp[a % len(ss)], iout[a % len(ss)], 0, 1, vc, s_)
                    h += 2
                return 2 * APPS
            itmp = [torch.empty_like(ins[0]) for _ in range(nstreams)]
            iout = [torch.empty_like(ins[0]) for _ in range(nstreams)]
            g = GraphStep(torch, istep, nstreams)
            ms, launches, _ = time_steps(torch, g, 10, 3, stream)
            del g
            us = ms * 1000.0 / launches
            gbs = Vh * sb / us / 1e3
            out[f"improved/{prec}/18/{vec}"] = {"gflops": round(Vh * 1146 / us / 1e3, 1), "gbs": round(gbs, 1),
                                                "frac": round(gbs / peak, 3), "us_per_half": round(us, 2),
                                                "bytes_per_site": sb, "ring": K}
            del fats, lngs, ins, ts, outs, itmp, iout
            torch.cuda.empty_cache()
    if want("wilson"):
        # Wilson hopping term through half Wilson vectors (8 hops, 1320 flops per site)
        for prec, recon in (("f32", 18), ("f32", 12), ("bf16", 12), ("f64", 18)):
            vec = "f64" if prec == "f64" else "f32"
            sb = 8 * recon * BYTES[prec] + 2 * 24 * BYTES[vec]
            K = ring_size(Vh * sb, l2, nstreams)
            wg = [lq.lq_gauge_pack(ctx, DIMS, U_dev, prec, recon) for _ in range(K)]
            dt = torch.complex128 if vec == "f64" else torch.complex64
            host = torch.from_numpy(synth.spinor_field(DIMS, 1, seed=9)).to(dt)
            wins = [host.cuda() for _ in range(K)]
            wtmp = [torch.empty_like(wins[0]) for _ in range(nstreams)]
            wout = [torch.empty_like(wins[0]) for _ in range(nstreams)]
            vc = lq.PREC[vec]

            def wstep(ss, wg=wg, wins=wins, wtmp=wtmp, wout=wout, vc=vc, K=K):
                h = 0
                for a in range(APPS):
                    s_ = ss[a % len(ss)]
                    c, c2 = h % K, (h + 1) % K
                    lq.dslash_wilson_eo(ctx, wg[c], wins[c], wtmp[a % len(ss)], 1, 1, vc, 1, s_)
                    lq.dslash_wilson_eo(ctx, wg[c2], wtmp[a % len(ss)], wout[a % len(ss)], 0, 1, vc, 1, s_)
                    h += 2
                return 2 * APPS
            g = GraphStep(torch, wstep, nstreams)
            ms, launches, _ = time_steps(torch, g, 10, 3, stream)
            del g
            us = ms * 1000.0 / launches
            gbs = Vh * sb / us / 1e3
            out[f"wilson/{prec}/{recon}/{vec}"] = {"gflops": round(Vh * 1320 / us / 1e3, 1), "gbs": round(gbs, 1),
                                                   "frac": round(gbs / peak, 3), "us_per_half": round(us, 2),
                                                   "bytes_per_site": sb, "ring": K}
            del wg, wins, wtmp, wout
            torch.cuda.empty_cache()
    if want("multi_rhs"):
        # multi-RHS Dslash (links loaded once per site for all right-hand sides): canonical
        # [rhs][site][3] vectors through dslash_eo, and the paired colour-planar layout
        # through dslash_eo_paired (converted once, outside the timed region)
        for layout in ("canonical", "paired"):
            for prec, recon, nrhs in (("f32", 12, 8), ("f32", 18, 8), ("bf16", 12, 8), ("f32", 12, 16)):
                sb = 8 * recon * BYTES[prec] + nrhs * 12 * BYTES["f32"]
                K = ring_size(Vh * sb, l2, nstreams)
                gauges = [lq.lq_gauge_pack(ctx, DIMS, U_dev, prec, recon) for _ in range(K)]
                chi = torch.from_numpy(synth.fermion_field(DIMS, nrhs, seed=12)).to(torch.complex64).cuda()
                if layout == "paired":
                    pchi = torch.empty(lq.paired_numel(Vh, nrhs), dtype=torch.float32, device="cuda")
                    lq.lq_vec_pair(ctx, Vh, nrhs, chi, pchi)
                    ins = [pchi.clone() for _ in range(K)]
                    del pchi
                else:
                    ins = [chi.clone() for _ in range(K)]
                del chi
                ts = [torch.empty_like(ins[0]) for _ in range(K)]
                outs = [torch.empty_like(ins[0]) for _ in range(K)]

                def mstep(ss, gauges=gauges, ins=ins, ts=ts, outs=outs, nrhs=nrhs, layout=layout):
                    h = 0
                    for a in range(APPS):
                        s_ = ss[a % len(ss)]
                        c, c2 = h % K, (h + 1) % K
                        if layout == "paired":
                            lq.dslash_eo_paired(ctx, gauges[c], ins[c], ts[c], 1, nrhs, s_)
                            lq.dslash_eo_paired(ctx, gauges[c2], ts[c], outs[c], 0, nrhs, s_)
                        else:
                            lq.dslash_eo(ctx, gauges[c], ins[c], ts[c], 1, nrhs, lq.LQ_F32, s_)
                            lq.dslash_eo(ctx, gauges[c2], ts[c], outs[c], 0, nrhs, lq.LQ_F32, s_)
                        h += 2
                    return 2 * APPS
                g = GraphStep(torch, mstep, nstreams)
                ms, launches, _ = time_steps(torch, g, 10, 3, stream)
                del g
                us = ms * 1000.0 / launches
                gbs = Vh * sb / us / 1e3
                name = "multi_rhs" if layout == "canonical" else "multi_rhs_paired"
                out[f"{name}/{prec}/{recon}/nrhs{nrhs}"] = {
                    "gflops": round(Vh * nrhs * FLOPS_PER_SITE / us / 1e3, 1), "gbs": round(gbs, 1),
                    "frac": round(gbs / peak, 3), "us_per_half": round(us, 2), "bytes_per_site": sb, "ring": K,
                    "layout": layout}
                del gauges, ins, ts, outs
                torch.cuda.empty_cache()
    if want("su3"):
        # mult_su3_mat_vec / mult_adj_su3_mat_vec over the 4V links of the lattice; like the
        # Dslash lines, `nstreams` independent batches in flight (graph branches), each
        # launch on its own ring copy (inputs larger than L2)
        n = 4 * 2 * Vh
        A = torch.from_numpy(synth.haar_su3(synth.rng(9), n))
        b = torch.from_numpy(synth.complex_gaussian(synth.rng(10), (n, 3)))
        for prec, dt in (("f64", torch.complex128), ("f32", torch.complex64)):
            per = n * 30 * BYTES[prec]
            K = ring_size(per, l2, nstreams)
            As = [A.to(dt).cuda() for _ in range(K)]
            bs = [b.to(dt).cuda() for _ in range(K)]
            cs = [torch.empty_like(bs[0]) for _ in range(K)]
            for adj in (0, 1):
                def step(ss):
                    for i in range(2 * APPS):
                        lq.su3_matvec_batch(ctx, As[i % K], bs[i % K], cs[i % K], n, adj, None, ss[i % len(ss)])
                    return 2 * APPS
                g = GraphStep(torch, step, nstreams)
                ms, launches, _ = time_steps(torch, g, 5, 2, stream)
                del g
                us = ms * 1000.0 / launches
                gbs = per / us / 1e3
                out[f"su3_matvec/{prec}/adj{adj}"] = {"gflops": round(n * 66 / us / 1e3, 1), "gbs": round(gbs, 1),
                                                      "frac": round(gbs / peak, 3), "us": round(us, 2), "n": n}
            del As, bs, cs
        # the same mat-vec with 12-real and 16-bit storage (su3_matvec_batch_ex)
        for mat, recon, vec in (("f64", 12, "f64"), ("f32", 12, "f32"), ("bf16", 18, "bf16"),
                                ("bf16", 12, "bf16"), ("f16", 12, "f16"), ("bf16", 12, "f32")):
            per = n * (recon * BYTES[mat] + 12 * BYTES[vec])
            K = ring_size(per, l2, nstreams)
            rows = A[:, :2, :].contiguous() if recon == 12 else A

            def dev(z, prec):
                if prec == "f64":
                    return z.cuda()
                if prec == "f32":
                    return z.to(torch.complex64).cuda()
                dt = torch.bfloat16 if prec == "bf16" else torch.float16
                return torch.view_as_real(z).to(dt).contiguous().cuda()
            As = [dev(rows, mat) for _ in range(K)]
            bs = [dev(b, vec) for _ in range(K)]
            cs = [torch.empty_like(bs[0]) for _ in range(K)]
            for adj in (0, 1):
                def step(ss, As=As, bs=bs, cs=cs, mat=mat, recon=recon, vec=vec, adj=adj):
                    for i in range(2 * APPS):
                        lq.su3_matvec_batch_ex(ctx, As[i % K], bs[i % K], cs[i % K], n, adj, mat, recon, vec,
                                               ss[i % len(ss)])
                    return 2 * APPS
                g = GraphStep(torch, step, nstreams)
                ms, launches, _ = time_steps(torch, g, 5, 2, stream)
                del g
                us = ms * 1000.0 / launches
                gbs = per / us / 1e3
                out[f"su3_matvec/{mat}/{recon}/{vec}/adj{adj}"] = {
                    "gflops": round(n * 66 / us / 1e3, 1), "gbs": round(gbs, 1), "frac": round(gbs / peak, 3),
                    "us": round(us, 2), "n": n, "bytes_per_item": recon * BYTES[mat] + 12 * BYTES[vec]}
            del As, bs, cs
        ctx.sync()   # every bulk-copy wait of the batched kernels delivered (LQ_ERR_TIMEOUT otherwise)
        # mult_su3_nn / an / na over the 4V links (pairs of Haar matrices)
        B2 = torch.from_numpy(synth.haar_su3(synth.rng(11), n))
        for prec, dt in (("f64", torch.complex128), ("f32", torch.complex64)):
            per = n * 54 * BYTES[prec]
            K = ring_size(per, l2, nstreams)
            As = [A.to(dt).cuda() for _ in range(K)]
            Bs = [B2.to(dt).cuda() for _ in range(K)]
            Cs = [torch.empty_like(As[0]) for _ in range(K)]
            for adjA, adjB in ((0, 0), (1, 0), (0, 1)):
                def step(ss):
                    for i in range(2 * APPS):
                        lq.su3_mul_batch(ctx, As[i % K], Bs[i % K], Cs[i % K], n, adjA, adjB, None, ss[i % len(ss)])
                    return 2 * APPS
                g = GraphStep(torch, step, nstreams)
                ms, launches, _ = time_steps(torch, g, 5, 2, stream)
                del g
                us = ms * 1000.0 / launches
                gbs = per / us / 1e3
                out[f"su3_mul/{prec}/adj{adjA}{adjB}"] = {"gflops": round(n * 198 / us / 1e3, 1), "gbs": round(gbs, 1),
                                                         "frac": round(gbs / peak, 3), "us": round(us, 2), "n": n}
            del As, Bs, Cs
        # the 1024-pair FP64 product of the 4^4 configuration: latency of one call
        Ad, Bd = A[:1024].cuda(), B2[:1024].cuda()
        Cd = torch.empty_like(Ad)
        g = GraphStep(torch, lambda ss: [lq.su3_mul_batch(ctx, Ad, Bd, Cd, 1024, 0, 0, None, ss[0]) for _ in range(20)] and 20, 1)
        ms, launches, _ = time_steps(torch, g, 5, 2, stream)
        out["su3_mul/f64/1024_pairs_us"] = round(ms * 1000.0 / launches, 2)
    # FP64 kernels are bound by GB300's FP64 ALU, not by HBM: their roofline is the measured
    # FP64 FMA rate (algorithmic flops, the same counts as "gflops")
    for k, v in out.items():
        if isinstance(v, dict) and "/f64/" in f"/{k}/":
            v["bound"] = "fp64_alu"
            v["alu_frac"] = round(v["gflops"] / fp64_peak, 3)
    return out


def run_cg(lq, ctx, torch, maxiter=20000):
    """32^4, Haar links, m = 0.01, Gaussian source: FP64 CG against mixed precision."""
    import synth
    dims, mass = (32, 32, 32, 32), 0.01
    U = torch.from_numpy(synth.gauge_field(dims, "haar", seed=4)).cuda()
    b = torch.from_numpy(synth.fermion_field(dims, 1, seed=5)).cuda()
    x = torch.empty_like(b)
    hi = lq.lq_gauge_pack(ctx, dims, U, "f64", 18)
    res = {"workload": "32^4 Haar SU(3), m=0.01, Gaussian source, tol 1e-10 (FP64 true residual)"}
    x64 = None
    for name, prec, recon in (("fp64", None, 18), ("mixed_f32_12", "f32", 12), ("mixed_f16_12", "f16", 12),
                              ("mixed_bf16_12", "bf16", 12)):
        lo = lq.lq_gauge_pack(ctx, dims, U, prec, recon) if prec else None
        try:  # a short solve first: tunes the launch shapes outside the timed solve
            lq.cg_solve(ctx, hi, lo, mass, b, x, 1, tol=1e-10, maxiter=200)
        except lq.LQError:
            pass
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            st = lq.cg_solve(ctx, hi, lo, mass, b, x, 1, tol=1e-10, maxiter=maxiter)[0]
            ok = True
        except lq.LQError as e:
            st, ok = e.stats[0], False
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        res[name] = {"seconds": round(dt, 4), "iters": st["iters"], "reliable_updates": st["reliable_updates"],
                     "true_rel_resid": st["true_rel_resid"], "converged": ok}
        if prec is None:
            x64 = x.clone()
        elif x64 is not None:
            # error of the mixed solution against the FP64 solution of the same system
            res[name]["x_rel_err_vs_fp64"] = float(torch.linalg.vector_norm(x - x64) / torch.linalg.vector_norm(x64))
    if res["fp64"]["converged"]:
        for k in ("mixed_f32_12", "mixed_f16_12", "mixed_bf16_12"):
            if res[k]["converged"]:
                res[k]["speedup_vs_fp64"] = round(res["fp64"]["seconds"] / res[k]["seconds"], 2)
    return res


def run_multi_rhs_cg(lq, ctx, torch):
    """24^4 Haar, m = 0.05, 8 right-hand sides, FP32-12 inner, tol 1e-10: one multi-RHS
    solve on the paired layout, the same solve on the canonical layout, and the 8 systems
    solved one at a time."""
    import synth
    dims, mass, nrhs = (24, 24, 24, 24), 0.05, 8
    U = torch.from_numpy(synth.gauge_field(dims, "haar", seed=6)).cuda()
    b = torch.from_numpy(synth.fermion_field(dims, nrhs, seed=7)).cuda()
    x = torch.empty_like(b)
    hi = lq.lq_gauge_pack(ctx, dims, U, "f64", 18)
    lo = lq.lq_gauge_pack(ctx, dims, U, "f32", 12)
    res = {"workload": "24^4 Haar SU(3), m=0.05, 8 Gaussian sources, FP32 inner (12-real), tol 1e-10 "
                       "(FP64 true residual)"}
    prev = os.environ.get("LQCD_CG_PAIRED")

    def solve(bb, xx, n):
        try:  # a short solve first: tunes the launch shapes outside the timed solve
            lq.cg_solve(ctx, hi, lo, mass, bb, xx, n, tol=1e-10, maxiter=200)
        except lq.LQError:
            pass
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = lq.cg_solve(ctx, hi, lo, mass, bb, xx, n, tol=1e-10, maxiter=20000)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, st

    try:
        for name, flag in (("paired", "1"), ("canonical", "0")):
            os.environ["LQCD_CG_PAIRED"] = flag
            dt, st = solve(b, x, nrhs)
            it = max(s_["iters"] for s_ in st)
            res[name] = {"seconds": round(dt, 4), "iters": it, "us_per_iter": round(1e6 * dt / it, 1),
                         "max_true_rel_resid": max(s_["true_rel_resid"] for s_ in st)}
        total = 0.0
        for k in range(nrhs):
            dt, _ = solve(b[k:k + 1].contiguous(), x[k:k + 1], 1)
            total += dt
        res["one_at_a_time_seconds"] = round(total, 4)
        res["speedup_paired_vs_one_at_a_time"] = round(total / res["paired"]["seconds"], 2)
        res["speedup_paired_vs_canonical"] = round(res["canonical"]["seconds"] / res["paired"]["seconds"], 3)
    finally:
        if prev is None:
            os.environ.pop("LQCD_CG_PAIRED", None)
        else:
            os.environ["LQCD_CG_PAIRED"] = prev
    return res


def run_batched(lq, ctx, torch):
    """Lattices 8^4, 12^4, 16^4, 24^4, 8 Gaussian right-hand sides each, links exp(i 0.2 H),
    m = 0.1, FP32 inner iteration (12-real links), tol 1e-8: one batched solve against the
    four solves one after the other."""
    import synth
    dims_list = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16), (24, 24, 24, 24)]
    his, los, bs = [], [], []
    for i, d in enumerate(dims_list):
        U = torch.from_numpy(synth.gauge_field(d, "near_identity", seed=5 + i, eps=0.2)).cuda()
        his.append(lq.lq_gauge_pack(ctx, d, U, "f64", 18))
        los.append(lq.lq_gauge_pack(ctx, d, U, "f32", 12))
        bs.append(torch.from_numpy(synth.fermion_field(d, 8, seed=105 + i)).cuda())
    xs = [torch.empty_like(b) for b in bs]
    kw = dict(tol=1e-8, maxiter=20000)
    lq.cg_solve_batched(ctx, his, los, [0.1] * 4, bs, xs, 8, **kw)      # tunes the shapes
    for h, l, b, x in zip(his, los, bs, xs):
        lq.cg_solve(ctx, h, l, 0.1, b, x, 8, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = lq.cg_solve_batched(ctx, his, los, [0.1] * 4, bs, xs, 8, **kw)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    for h, l, b, x in zip(his, los, bs, xs):
        lq.cg_solve(ctx, h, l, 0.1, b, x, 8, **kw)
    torch.cuda.synchronize()
    t_sep = time.perf_counter() - t0
    tune = [l for l in ctx.tune_report().splitlines() if "dslash_multi" in l and "8x8x8x8,12x12" in l]
    return {"workload": "8^4+12^4+16^4+24^4, 8 RHS each, eps 0.2, m 0.1, FP32 inner (12-real), tol 1e-8",
            "batched_seconds": round(t_batch, 4), "separate_seconds": round(t_sep, 4),
            "speedup": round(t_sep / t_batch, 3),
            "max_iters": max(s["iters"] for lat in st for s in lat),
            "max_true_rel_resid": max(s["true_rel_resid"] for lat in st for s in lat),
            "autotuned_multi_dslash": tune}


def run_force(lq, ctx, torch):
    """32^3 x 64, Haar links, m = 0.05, Gaussian chi: dslash_force (psi, dS/dchi, G and the
    TA force) in FP32 and FP64."""
    import synth
    dims, mass = (32, 32, 32, 64), 0.05
    U = torch.from_numpy(synth.gauge_field(dims, "haar", seed=6)).cuda()
    chi0 = torch.from_numpy(synth.fermion_field(dims, 1, seed=7)[0])
    V = synth.volume(dims)
    out = {"workload": "32^3x64 Haar, m 0.05: psi = D_oe chi, dS/dchi, dS/dU and TA(U G^dag)"}
    peak, _ = measured_peak()
    for prec, ct in (("f32", torch.complex64), ("f64", torch.complex128)):
        g = lq.lq_gauge_pack(ctx, dims, U, prec, 18)
        chi = chi0.to(ct).cuda()
        dU = torch.empty(U.shape, dtype=ct, device="cuda")
        F = torch.empty(U.shape, dtype=ct, device="cuda")
        dchi = torch.empty_like(chi)
        for _ in range(2):
            lq.dslash_force(ctx, g, mass, chi, dSdU=dU, force_TA=F, dSdchi=dchi)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        n = 5
        for _ in range(n):
            lq.dslash_force(ctx, g, mass, chi, dSdU=dU, force_TA=F, dSdchi=dchi)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / n
        s = BYTES[prec]
        # two half Dslash (site_bytes each over V/2 sites) + the link pass: read U and the two
        # vectors, write G and F
        nbytes = 2 * (V // 2) * site_bytes(prec, 18, prec) + 4 * V * 18 * s * 3 + 2 * (V // 2) * 6 * s
        out[prec] = {"ms": round(ms, 3), "gbs": round(nbytes / ms / 1e6, 1),
                     "frac": round(nbytes / ms / 1e6 / peak, 3), "bytes": nbytes}
        del g, dU, F, dchi
        torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    import paper_1309_0551_gb300 as lq
    import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = dist_init(world, True)
    device = torch.device("cuda", local)
    lq.load()  # raises if the library has not been built (__graft_entry__.build())
    ctx = lq.Context(local)
    ctx.set_tuning(2)  # launch shapes for several applications in flight (--streams)
    stream = torch.cuda.current_stream()
    prec, recon = args.prec, args.recon
    vec = args.vec or ("f64" if prec == "f64" else "f32")
    vc = lq.PREC[vec]
    props = torch.cuda.get_device_properties(local)
    l2 = int(getattr(props, "L2_cache_size", 128 << 20))
    dims = tuple(int(v) for v in args.lattice.split(","))
    nrhs = args.nrhs
    Vh = synth.volume(dims) // 2
    sb = site_bytes(prec, recon, vec, nrhs)
    K = ring_size(Vh * sb, l2, args.streams)
    U_host = synth.gauge_field(dims, args.field, seed=3 + rank, eps=0.3)
    U_dev = torch.from_numpy(U_host).cuda()
    gauges, ins, ts, outs = make_ring(lq, ctx, U_dev, dims, prec, recon, vec, K, seed=2 + rank, nrhs=nrhs)

    # ---- device-resident throughput
    step = GraphStep(torch, lambda ss: run_step(lq, ctx, gauges, ins, ts, outs, vc, ss, nrhs=nrhs), args.streams)
    sampler = ClockSampler(local)
    ms, launches, clocks = time_steps(torch, step, args.steps, args.warmup, stream, dist, device, sampler)
    flops = args.steps * APPS * 2 * Vh * nrhs * FLOPS_PER_SITE * world
    value = flops / (ms * 1e-3) / 1e9
    us_per_launch = ms * 1000.0 / launches
    achieved = Vh * sb / us_per_launch / 1e3  # GB/s
    peak, peak_kind = measured_peak()
    key = f"{prec}/{recon}/{vec}/{'x'.join(map(str, dims))}/{nrhs}"
    traffic = None
    if key in NCU_TRAFFIC and NCU_TRAFFIC[key][1] == kernel_hash():
        traffic = NCU_TRAFFIC[key][0]

    # ---- end to end through the public API: every step copies its inputs in from pinned host
    # memory, issues every half-Dslash as its own dslash_eo call through the binding and the C
    # ABI (no graph: argument checks, tuning-table lookup and launch run per call), and copies
    # the outputs back.
    # the ring's K input copies are views of one contiguous tensor (make_ring): one
    # pinned-host copy in and one out per step, the same bytes as K separate copies
    def whole(views):
        base = views[0]
        n = len(views)
        assert all(v.data_ptr() == base.data_ptr() + k * base.numel() * base.element_size()
                   for k, v in enumerate(views))
        return base.as_strided((n,) + tuple(base.shape), (base.numel(),) + tuple(base.stride()))

    dev_in, dev_out = whole(ins), whole(outs)
    host_in = [torch.empty_like(dev_in, device="cpu").pin_memory()]
    host_in[0].copy_(dev_in)
    host_out = [torch.empty_like(dev_out, device="cpu").pin_memory()]
    ins_all, outs_all = [dev_in], [dev_out]
    side = [stream] + [torch.cuda.Stream() for _ in range(args.streams - 1)]

    def e2e_step():
        for h, t in zip(host_in, ins_all):
            t.copy_(h, non_blocking=True)
        for s_ in side[1:]:
            s_.wait_stream(stream)
        n = run_step(lq, ctx, gauges, ins, ts, outs, vc, side, nrhs=nrhs)
        for s_ in side[1:]:
            stream.wait_stream(s_)
        for h, t in zip(host_out, outs_all):
            h.copy_(t, non_blocking=True)
        return n

    e2e_steps = max(1, args.steps // 2)
    ms_e2e, _, _ = time_steps(torch, e2e_step, e2e_steps, min(args.warmup, 3), stream, dist, device)
    e2e_val = e2e_steps * APPS * 2 * Vh * nrhs * FLOPS_PER_SITE * world / (ms_e2e * 1e-3) / 1e9

    # the same with the step's launches replayed from a CUDA graph (copies still every step)
    def e2e_graph_step():
        for h, t in zip(host_in, ins_all):
            t.copy_(h, non_blocking=True)
        n = step()
        for h, t in zip(host_out, outs_all):
            h.copy_(t, non_blocking=True)
        return n

    ms_e2eg, _, _ = time_steps(torch, e2e_graph_step, e2e_steps, min(args.warmup, 3), stream, dist, device)
    e2e_graph_val = e2e_steps * APPS * 2 * Vh * nrhs * FLOPS_PER_SITE * world / (ms_e2eg * 1e-3) / 1e9

    extra = {}
    if rank == 0 and not args.no_variants:  # same regime as the headline: concurrent launches
        fp64 = ctx.fp64_fma_rate()
        extra["fp64_peak"] = {"gflops": round(fp64, 1), "nominal_gflops": FP64_NOMINAL_GFLOPS,
                              "source": "measured: lq_fp64_fma_rate (16 independent FMA chains per thread, "
                                        "every SM, CUDA events, best of 3)"}
        U_var = U_dev if dims == DIMS else torch.from_numpy(
            synth.gauge_field(DIMS, "near_identity", seed=3, eps=0.3)).cuda()
        extra["variants"] = run_variants(lq, ctx, torch, U_var, l2, stream, args.streams, args.variants, fp64)
    if rank == 0 and not args.no_cg:
        ctx.set_tuning(1)  # the solvers issue one launch at a time
        extra["cg"] = run_cg(lq, ctx, torch, args.cg_maxiter)
        if not args.no_batched_force:
            extra["batched"] = run_batched(lq, ctx, torch)
            extra["multi_rhs_cg"] = run_multi_rhs_cg(lq, ctx, torch)
            extra["force"] = run_force(lq, ctx, torch)
    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "GFLOP/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if prec == "f64" else "f32",
        "data": "synthetic",
        "config": {"workload": f"staggered Dslash, {'x'.join(map(str, dims))} lattice, "
                               + ("links exp(i*0.3*H) on SU(3), " if args.field == "near_identity" else "Haar links, ")
                               + f"{APPS} full-D applications per step" + (f", {nrhs} right-hand sides" if nrhs > 1 else ""),
                   "lattice": "x".join(map(str, dims)), "nrhs": nrhs,
                   "link_storage": f"{prec}/{recon}-real", "vector_storage": vec,
                   "l2": f"inputs larger than L2: ring of {K} device copies of links and vectors "
                         f"({K * Vh * sb / 1e6:.0f} MB) cycled across launches",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "kernel": "k_dslash", "bytes_per_launch": Vh * sb,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
                     "us_per_launch": round(us_per_launch, 3)},
        "e2e": {"value": round(e2e_val, 1), "unit": "GFLOP/s",
                "h2d_bytes_per_step": sum(t.numel() * t.element_size() for t in ins_all),
                "d2h_bytes_per_step": sum(t.numel() * t.element_size() for t in outs_all),
                "path": f"pinned host -> device copies, {2 * APPS} dslash_eo calls through the binding and "
                        f"the C ABI on {args.streams} streams, device -> pinned host copies, every step",
                "graph_replay_value": round(e2e_graph_val, 1)},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    line["config"]["streams"] = args.streams
    line["config"]["tuning"] = "autotuned, throughput mode (lq_set_tuning 2)"
    dkey = f"g={prec}/{recon} v={vec} dims={'x'.join(map(str, dims))} nrhs={nrhs}"
    line["config"]["launch_shape"] = [l for l in ctx.tune_report().splitlines() if dkey in l]
    line.update(extra)
    if rank == 0 and not args.no_cpu:
        fp64_iters = extra.get("cg", {}).get("fp64", {}).get("iters")
        line["cpu_baseline"] = cpu_baseline(DIMS, fp64_cg_iters=fp64_iters)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------ reference arm -----

def run_reference(args):
    """The oracle as it stands, on the host cores: each step is one full-D application (two
    half-Dslash calls) of the FP64 C++ oracle on the benchmark lattice, on every core -- a
    bounded sample of the GPU arm's step (100 applications)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import synth
    from oracle import cxx
    U = synth.gauge_field(DIMS, "near_identity", seed=3, eps=0.3)
    chi = synth.fermion_field(DIMS, 1, seed=2)[0]
    Vh = synth.volume(DIMS) // 2
    nproc = os.cpu_count() or 1
    threads = min(nproc, cxx.max_threads())
    for i in range(args.warmup):
        cxx.dslash_eo(U, cxx.dslash_eo(U, chi, DIMS, 1, threads), DIMS, 0, threads)
    t0 = time.perf_counter()
    for i in range(args.steps):
        cxx.dslash_eo(U, cxx.dslash_eo(U, chi, DIMS, 1, threads), DIMS, 0, threads)
    dt = time.perf_counter() - t0
    value = args.steps * 2 * Vh * FLOPS_PER_SITE / dt / 1e9
    sample = (f"{args.steps} full-D applications (two half-Dslash each, one application per step) on the "
              f"16x16x16x32 lattice, FP64 C++ oracle on {threads} threads")
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1000 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": "staggered Dslash, 16^3x32 lattice, links exp(i*0.3*H) on SU(3)",
                   "lattice": "16x16x16x32", "implementation": "FP64 C++ oracle (OpenMP) on the host"},
        "cpu_baseline": {"value": round(value, 4), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                         "cpu": cpu_model(), "nproc": nproc, "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
