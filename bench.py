"""Throughput benchmark of the D2Q9 BGK stream-and-collide library on GB300.

Default workload (one JSON line on stdout): dense, fully periodic
Taylor-Green vortex, 4096 x 4096 nodes, tau 0.8, peak velocity 0.05, FP32
storage, two-lattice pattern; one "step" = one lbm_step over the whole grid
(gather, moments, BGK, store: every node-update of the hot path).  The metric
is GLUPS = node updates / s (Sec. 4.2.2, P_LUPS), with the bandwidth
roofline of 2 q s_d bytes per node (B_node, Sec. 4.2.2).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--precision f32|f64|f16s] [--pattern two_lattice|aa]
                  [--layout dense|sparse] [--n 4096] [--no-extra]

N > 1 (torchrun, one rank per GPU): every rank runs its own replica of the
workload (the method needs no exchange between independent simulations),
"scaling": "weak"; value = node updates of all ranks / max rank time.

--impl reference times the FP64 CPU oracle (the plain C implementation the
tests check the GPU against) on the host cores, on a bounded sample of the
same workload, and prints the same JSON line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D2Q9 GLUPS and % HBM roofline, dense+sparse, fp64/32/16; adjoint step cost"
BYTES_PER_VALUE = {"f64": 8, "f32": 4, "f16s": 2}
KERNEL_SOURCE = os.path.join(ROOT, "paper_2108_13241_gb300", "csrc", "lbm_kernels.cuh")
PROFILE_DIR = os.path.join(ROOT, "profiles")


def node_bytes(precision: str) -> int:
    """Algorithmic bytes per node update: read and write all q = 9 values."""
    return 2 * 9 * BYTES_PER_VALUE[precision]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_hash() -> str:
    """Hash of the kernel source with comments and white space removed, so
    that a profile stays valid across comment-only edits."""
    with open(KERNEL_SOURCE) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    text = re.sub(r"\s+", "", text)
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def profiled_traffic(name: str):
    """DRAM bytes per launch recorded in profiles/<name>.md by an ncu capture of
    the current kernel source (None when absent or taken on another source)."""
    path = os.path.join(PROFILE_DIR, name + ".md")
    try:
        text = open(path).read()
    except OSError:
        return None
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    t = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not h or not t or h.group(1) != kernel_hash():
        return None
    return float(t.group(1))


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "lbm_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[4:9]))
            except ValueError:
                continue
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["active_mask", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, flags in rows:
            for nm, v in zip(names[1:], flags[1:]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------- workloads

def build_case(workload: str, n: int, precision: str):
    """Solver arguments, initial fields and fluid-node count of a workload."""
    from paper_2108_13241_gb300 import inputs
    tau, U = 0.8, 0.05
    if workload == "tgv":
        rho, u = inputs.taylor_green(n, n, U)
        kw = dict(nx=n, ny=n, tau=tau)
        return kw, rho, u, n * n, "taylor_green_%d" % n
    if workload == "poiseuille":
        fx, rho, u = inputs.poiseuille(n, n, tau, U)
        kw = dict(nx=n, ny=n, tau=tau, force=(fx, 0.0), periodic_y=False)
        return kw, rho, u, n * n, "poiseuille_%d" % n
    if workload.startswith("porous"):
        phi = float(workload[len("porous"):] or 0.5)
        solid, achieved, _ = inputs.porous_discs(n, n, phi, rmin=8, rmax=32)
        kw = dict(nx=n, ny=n, tau=tau, solid=solid, force=(1e-6, 0.0), periodic_y=False)
        nf = int((solid == 0).sum())
        return kw, None, None, nf, "porous_phi%.2f_%d" % (achieved, n)
    raise ValueError(workload)


def time_steps(sim, steps: int, warmup: int, stream):
    import torch
    sim.step(warmup)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    sim.step(steps)
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / 1e3


def run_gpu_arm(args, rank, world, dist):
    import torch
    from paper_2108_13241_gb300 import lbm

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    kw, rho, u, nfluid, wname = build_case(args.workload, args.n, args.precision)
    sim = lbm.LBM(precision=args.precision, layout=args.layout, pattern=args.pattern, **kw)
    dtype = sim.dtype
    rho_h = None if rho is None else torch.as_tensor(rho, dtype=dtype).pin_memory()
    u_h = None if u is None else torch.as_tensor(u, dtype=dtype).pin_memory()
    rho_d = None if rho_h is None else rho_h.to(dev)
    u_d = None if u_h is None else u_h.to(dev)
    sim.init_equilibrium(rho_d, u_d)

    # device-resident timing (value)
    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    sim.step(args.warmup)
    barrier()
    with ClockSampler(dev.index) as clk:
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        sim.step(args.steps)
        end.record(stream)
        end.synchronize()
    barrier()
    t = start.elapsed_time(end) / 1e3
    clocks = clk.summary()
    if dist is not None:
        tt = torch.tensor([t], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    mass, _ = sim.reduce()
    if not np.isfinite(mass):
        raise RuntimeError("simulation diverged")

    # end to end through the public API: pinned host fields -> device, init,
    # K steps, macros, device -> pinned host result
    out_rho = torch.empty((kw["ny"], kw["nx"]), dtype=dtype).pin_memory()
    out_u = torch.empty((2, kw["ny"], kw["nx"]), dtype=dtype).pin_memory()
    barrier()
    t0 = time.perf_counter()
    r_d = None if rho_h is None else rho_h.to(dev, non_blocking=True)
    v_d = None if u_h is None else u_h.to(dev, non_blocking=True)
    sim.init_equilibrium(r_d, v_d)
    sim.step(args.steps)
    r_out, u_out = sim.macros()
    out_rho.copy_(r_out, non_blocking=True)
    out_u.copy_(u_out, non_blocking=True)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    if dist is not None:
        tt = torch.tensor([t_e2e], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_e2e = float(tt.item())
    h2d = (0 if rho_h is None else rho_h.numel() * rho_h.element_size()) + \
          (0 if u_h is None else u_h.numel() * u_h.element_size())
    d2h = out_rho.numel() * out_rho.element_size() + out_u.numel() * out_u.element_size()

    glups = nfluid * args.steps * world / t / 1e9
    step_s = t / args.steps
    algo = node_bytes(args.precision) * nfluid
    peak, peak_kind = peaks()
    achieved = algo / step_s / 1e9
    prof_name = "step_%s_%s_%s_%s" % (args.precision, args.layout, args.pattern, wname)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                "traffic": profiled_traffic(prof_name),
                "algorithmic_bytes_per_launch": algo, "kernel": "k_step (%s)" % prof_name}
    res = {
        "metric": METRIC, "value": round(glups, 3), "unit": "GLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "f32": "f32", "f16s": "f16 storage, f32 compute"}[args.precision],
        "data": "synthetic (seeded Taylor-Green / Poiseuille fields, seeded disc geometries)",
        "config": {"workload": wname, "precision": args.precision, "layout": args.layout,
                   "pattern": args.pattern, "nodes": kw["nx"] * kw["ny"], "fluid_nodes": nfluid,
                   "tau": kw["tau"], "bytes_per_node_update": node_bytes(args.precision),
                   "parallelism": "replicas x%d" % world,
                   "l2": "working set %.0f MB > 129 MB L2, no flush needed" %
                         (2 * 9 * BYTES_PER_VALUE[args.precision] * kw["nx"] * kw["ny"] / 1e6)},
        "roofline": roofline,
        "e2e": {"value": round(nfluid * args.steps * world / t_e2e / 1e9, 3), "unit": "GLUPS",
                "h2d_bytes_per_step": round(h2d / args.steps, 1), "d2h_bytes_per_step": round(d2h / args.steps, 1),
                "what": "pinned host rho,u -> device, lbm_init_equilibrium, K x lbm_step, lbm_macros, "
                        "device -> pinned host rho,u"},
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    sim.close()
    return res


# ---------------------------------------------------------------- CPU oracle

def oracle_glups(n: int, budget_s: float, max_steps: int = 1000000):
    """FP64 CPU oracle (as it stands) on an n x n Taylor-Green box: runs
    steps until budget_s has passed; returns (GLUPS, steps, seconds, cores)."""
    from oracle import oracle as orc
    from paper_2108_13241_gb300 import inputs
    orc.build()
    s = orc.Setup(nx=n, ny=n, tau=0.8)
    mask, _ = orc.link_mask(s)
    rho, u = inputs.taylor_green(n, n, 0.05)
    A = orc.init_equilibrium(s, mask, rho, u)
    B = np.empty_like(A)
    p = s.c()
    import ctypes
    L = orc.lib()
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps:
        L.orc_step(ctypes.byref(p), orc._ptr(mask), None, orc._ptr(A), orc._ptr(B))
        A, B = B, A
        steps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return n * n * steps / dt / 1e9, steps, dt, orc.num_threads()


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference_arm(args):
    """The oracle timed on this machine's host cores: K steps after W warm-up
    steps, each step a full oracle step on an S x S Taylor-Green box, with S
    chosen from a probe so that the whole run takes about two minutes."""
    probe_n = 1024
    g, st, dt, cores = oracle_glups(probe_n, 2.0)
    total_steps = args.steps + args.warmup
    nodes_per_step = max(64 * 64, min(args.n * args.n, int(g * 1e9 * 110.0 / max(total_steps, 1))))
    S = max(64, int(np.sqrt(nodes_per_step)) // 16 * 16)
    from oracle import oracle as orc
    from paper_2108_13241_gb300 import inputs
    import ctypes
    s = orc.Setup(nx=S, ny=S, tau=0.8)
    mask, _ = orc.link_mask(s)
    rho, u = inputs.taylor_green(S, S, 0.05)
    A = orc.init_equilibrium(s, mask, rho, u)
    B = np.empty_like(A)
    p = s.c()
    L = orc.lib()
    for _ in range(args.warmup):
        L.orc_step(ctypes.byref(p), orc._ptr(mask), None, orc._ptr(A), orc._ptr(B))
        A, B = B, A
    t0 = time.perf_counter()
    for _ in range(args.steps):
        L.orc_step(ctypes.byref(p), orc._ptr(mask), None, orc._ptr(A), orc._ptr(B))
        A, B = B, A
    dt = time.perf_counter() - t0
    v = S * S * args.steps / dt / 1e9
    sample = "FP64 oracle, %d x %d periodic Taylor-Green (sample of the %d^2 workload), %d steps" % (
        S, S, args.n, args.steps)
    return {
        "impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": "GLUPS", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": "taylor_green_%d" % args.n, "sample": "%dx%d" % (S, S)},
        "cpu_baseline": {"value": round(v, 5), "unit": "GLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(v, 5), "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def cpu_baseline_leg(n: int):
    g, steps, dt, cores = oracle_glups(n, 12.0)
    return {"value": round(g, 5), "unit": "GLUPS", "cores": cores, "kind": "oracle",
            "sample": "FP64 oracle, %d x %d periodic Taylor-Green, %d steps in %.1f s on %d host threads "
                      "(%d cores in the affinity mask)" % (n, n, steps, dt, cores, cpu_cores())}


# ---------------------------------------------------------------- extra lines

def extra_measurements(args):
    """Other rows of the metric at smaller step counts: precisions, AA, sparse."""
    import torch
    from paper_2108_13241_gb300 import lbm
    out = {}
    peak, _ = peaks()
    stream = torch.cuda.current_stream()
    combos = [("tgv", 4096, "f64", "dense", "two_lattice", 100),
              ("tgv", 4096, "f32", "dense", "aa", 500),
              ("tgv", 4096, "f16s", "dense", "two_lattice", 500),
              ("tgv", 4096, "f16s", "dense", "aa", 500),
              ("poiseuille", 4096, "f32", "dense", "two_lattice", 500),
              ("porous0.5", 4096, "f32", "sparse", "two_lattice", 300),
              ("porous0.5", 4096, "f32", "dense", "two_lattice", 300)]
    for wl, n, prec, layout, pattern, k in combos:
        kw, rho, u, nf, wname = build_case(wl, n, prec)
        sim = lbm.LBM(precision=prec, layout=layout, pattern=pattern, **kw)
        sim.init_equilibrium(None if rho is None else torch.as_tensor(rho, dtype=sim.dtype, device="cuda"),
                             None if u is None else torch.as_tensor(u, dtype=sim.dtype, device="cuda"))
        t = time_steps(sim, k, 10, stream)
        g = nf * k / t / 1e9
        out["%s/%s/%s/%s" % (wname, prec, layout, pattern)] = {
            "GLUPS": round(g, 3), "GBps_algorithmic": round(g * node_bytes(prec), 1),
            "frac_of_measured_hbm": round(g * node_bytes(prec) / peak, 4), "steps": k}
        sim.close()
        del sim
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tgv")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--precision", default="f32", choices=["f64", "f32", "f16s"])
    ap.add_argument("--layout", default="dense", choices=["dense", "sparse"])
    ap.add_argument("--pattern", default="two_lattice", choices=["two_lattice", "aa"])
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference_arm(args)), flush=True)
        return 0

    # the CPU-baseline oracle runs before any CUDA call (no fork after CUDA init)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_leg(1024)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
        dist = tdist
    import __graft_entry__
    __graft_entry__.build()
    res = run_gpu_arm(args, rank, world, dist)
    if cpu is not None:
        res["cpu_baseline"] = cpu
    if rank == 0 and world == 1 and not args.no_extra:
        res["extra"] = extra_measurements(args)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
