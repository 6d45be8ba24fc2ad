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
    """Hash of the step kernel's source -- every section of the kernel file
    before the adjoint kernel, and the step launchers -- with comments and
    white space removed, so that a profile of the step kernel stays valid
    across comment-only edits and edits of the other kernels."""
    with open(KERNEL_SOURCE) as fh:
        full = fh.read()
    rule = "// " + "-" * 61 + " "
    text = full[:full.index(rule + "adjoint kernel")]
    launch = full.index(rule + "launchers")
    end = full.rfind("\n", launch, full.index(" node_blocks(const Geo", launch))
    text += full[launch:end]
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    text = re.sub(r"\s+", "", text)
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def profiled_value(name: str, key: str):
    """A figure ("key: value" line) recorded in profiles/<name>.md by an ncu
    capture of the current kernel source (None when absent or taken on
    another source)."""
    path = os.path.join(PROFILE_DIR, name + ".md")
    try:
        text = open(path).read()
    except OSError:
        return None
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    t = re.search(re.escape(key) + r":\s*([0-9.eE+]+)", text)
    if not h or not t or h.group(1) != kernel_hash():
        return None
    return float(t.group(1))


def profiled_traffic(name: str):
    """DRAM bytes per launch of the profiled kernel (see profiled_value)."""
    return profiled_value(name, "dram_bytes_per_launch")


# FP64 pipe of GB300: 2 FP64 thread instructions per SM per cycle (ncu's
# sm__sass_thread_inst_executed_op_dfma_pred_on.peak_sustained, 304 per cycle
# over the 152 SMs), at the 2070 MHz maximum SM clock
FP64_PER_SM_CYCLE = 2
SM_MAX_HZ = 2070e6


def fp64_alu_roofline(glups: float, sms: int):
    """The FP64 step is bound by the FP64 pipe, not by HBM: its ceiling is the
    pipe's instruction rate over the FP64 instructions one node update issues
    (from the committed ncu capture of the dense FP64 step)."""
    per_node = profiled_value("step_f64_dense_two_lattice_taylor_green_2048", "fp64_thread_instructions_per_node")
    if per_node is None:
        return None
    peak = FP64_PER_SM_CYCLE * sms * SM_MAX_HZ
    ceiling = peak / per_node / 1e9
    return {"bound": "alu", "fp64_inst_per_node": per_node, "peak_fp64_inst_per_s": peak,
            "GLUPS_ceiling": round(ceiling, 3), "frac": round(glups / ceiling, 4)}


KERNEL3_SOURCE = os.path.join(ROOT, "paper_2108_13241_gb300", "csrc", "lbm3.cu")


def kernel3_hash() -> str:
    """Hash of the D3Q19 device code (lbm3.cu before its C-ABI section: the
    kernels, not the host code that builds tables and picks them) without
    comments and white space: a profile figure of the 3-D step is used only
    while it matches."""
    with open(KERNEL3_SOURCE) as fh:
        text = fh.read()
    text = text[:text.index("// " + "-" * 61 + " C ABI")]
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    text = re.sub(r"\s+", "", text)
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def fp64_alu_roofline3(glups: float, sms: int):
    """The FP64 D3Q19 step's FP64-pipe ceiling (FP64 instructions a node from
    the committed capture of the same source), as fp64_alu_roofline."""
    path = os.path.join(PROFILE_DIR, "step_d3q19_taylor_green_128.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    h = re.search(r"lbm3_source_sha256_16:\s*([0-9a-f]+)", text)
    v = re.search(r"fp64_thread_instructions_per_node:\s*([0-9.eE+]+)", text)
    if not h or not v or h.group(1) != kernel3_hash():
        return None
    per_node = float(v.group(1))
    peak = FP64_PER_SM_CYCLE * sms * SM_MAX_HZ
    ceiling = peak / per_node / 1e9
    return {"bound": "alu", "fp64_inst_per_node": per_node, "peak_fp64_inst_per_s": peak,
            "GLUPS_ceiling": round(ceiling, 3), "frac": round(glups / ceiling, 4)}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms."""

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
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
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


class NvmlClocks:
    """SM clock and clock-event reasons read through NVML (the driver's
    libnvidia-ml) at chosen moments: the bench reads them right after the
    timed steps are launched and again before it waits for them, so that a
    timed region shorter than the nvidia-smi sampling period still has
    clock samples taken under load."""

    # nvmlClocksEventReasons bits (nvml.h)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, device_index: int):
        import ctypes
        self.rows = []
        self.ok = False
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            handle = ctypes.c_void_p()
            rc = -1
            try:
                import torch
                p = torch.cuda.get_device_properties(device_index)
                bus = "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
                rc = lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(handle))
            except (AttributeError, RuntimeError):
                rc = -1
            if rc != 0:
                rc = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(device_index), ctypes.byref(handle))
            if rc != 0:
                return
            self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
            self.lib, self.handle, self.ct = lib, handle, ctypes
            self.ok = True
        except (OSError, AttributeError):
            self.ok = False

    def sample(self):
        if not self.ok:
            return
        ct = self.ct
        sm, mx, rs = ct.c_uint(0), ct.c_uint(0), ct.c_ulonglong(0)
        if (self.lib.nvmlDeviceGetClockInfo(self.handle, 1, ct.byref(sm)) == 0 and
                self.lib.nvmlDeviceGetMaxClockInfo(self.handle, 1, ct.byref(mx)) == 0 and
                self.reasons_fn(self.handle, ct.byref(rs)) == 0):
            self.rows.append((float(sm.value), float(mx.value),
                              [nm for bit, nm in self.REASONS.items() if rs.value & bit]))


def merge_clocks(smi: dict, point: "NvmlClocks"):
    """The nvidia-smi sampler's summary joined with the NVML point samples."""
    if not point.rows:
        return smi
    sms = [r[0] for r in point.rows]
    reasons = set(r for row in point.rows for r in row[2])
    out = dict(smi)
    if smi.get("sm_mhz") is None:
        out["sm_mhz"] = statistics.median(sms)
        out["sm_max_mhz"] = max(r[1] for r in point.rows)
        out["reasons"] = sorted(reasons)
        out["samples"] = 0
    else:
        out["reasons"] = sorted(set(smi.get("reasons", [])) | reasons)
    out["nvml_samples_in_timed_region"] = [r[0] for r in point.rows]
    return out


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


def bench_config(args, kw, nfluid, wname, world):
    """The workload's description, the same for both arms."""
    return {"workload": wname, "precision": args.precision, "layout": args.layout,
            "pattern": args.pattern, "nodes": kw["nx"] * kw["ny"], "fluid_nodes": nfluid,
            "tau": kw["tau"], "bytes_per_node_update": node_bytes(args.precision),
            "parallelism": "replicas x%d" % world,
            "l2": "working set %.0f MB > 129 MB L2, no flush needed" %
                  (2 * 9 * BYTES_PER_VALUE[args.precision] * kw["nx"] * kw["ny"] / 1e6)}


def sector_nodes(solid: np.ndarray, precision: str) -> int:
    """Nodes in the 32-byte DRAM sectors (aligned runs of 32 / s nodes along
    x) that hold a fluid node: the bytes any step must move at sector
    granularity on this geometry are 2 q s per such node."""
    seg = 32 // BYTES_PER_VALUE[precision]
    ny, nx = solid.shape
    fl = (solid == 0)[:, : nx // seg * seg].reshape(ny, nx // seg, seg)
    return int(fl.any(axis=2).sum()) * seg


def max_over_ranks(value: float, dist, device) -> float:
    """The largest value over all ranks (every rank gets it)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_glups(nodes_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Node updates of all ranks (one replica each) per second, in 1e9."""
    return nodes_per_rank * steps * world / seconds / 1e9


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
    point = NvmlClocks(dev.index)
    point.sample()  # the first NVML query is slow: take it outside the timed region
    point.rows.clear()
    barrier()
    with ClockSampler(dev.index) as clk:
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        sim.step(args.steps)
        end.record(stream)  # queued before the host samples, so the samples add no device time
        point.sample()      # the steps are queued and running
        point.sample()
        end.synchronize()
    barrier()
    # kernels of the timed sim.step(K): K x launches per step (graph nodes
    # included), plus the step counter's set and advances when graphs replay
    step_launches = sim.step_launches(args.steps)
    t = max_over_ranks(start.elapsed_time(end) / 1e3, dist, dev)
    clocks = merge_clocks(clk.summary(), point)
    mass, _ = sim.reduce()
    if not np.isfinite(mass):
        raise RuntimeError("simulation diverged")

    # end to end through the public API: the initial fields in pinned host
    # memory are read by the init kernel itself (the device maps pinned
    # host memory; on GB300 the reads cross NVLink-C2C while the kernel
    # runs), K steps, and the macros kernel writes (rho, u) straight into
    # pinned host memory; every byte still moves host <-> device inside the
    # timed region
    out_rho = torch.empty((kw["ny"], kw["nx"]), dtype=dtype).pin_memory()
    out_u = torch.empty((2, kw["ny"], kw["nx"]), dtype=dtype).pin_memory()
    barrier()
    t0 = time.perf_counter()
    lbm.lbm_init_equilibrium(sim.ctx, rho_h, u_h)
    sim.step(args.steps)
    lbm.lbm_macros(sim.ctx, out_rho, out_u)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, dev)
    # the fields came back: the same (rho, u) as through device buffers
    r_out, u_out = sim.macros()
    if not (torch.equal(out_rho, r_out.cpu()) and torch.equal(out_u, u_out.cpu())):
        raise RuntimeError("fields written into pinned host memory differ from the device result")
    h2d = (0 if rho_h is None else rho_h.numel() * rho_h.element_size()) + \
          (0 if u_h is None else u_h.numel() * u_h.element_size())
    d2h = out_rho.numel() * out_rho.element_size() + out_u.numel() * out_u.element_size()

    glups = whole_job_glups(nfluid, args.steps, world, t)
    step_s = t / args.steps
    algo = node_bytes(args.precision) * nfluid
    peak, peak_kind = peaks()
    achieved = algo / step_s / 1e9
    prof_name = "step_%s_%s_%s_%s" % (args.precision, args.layout, args.pattern, wname)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                "frac_of_nominal_8000_gbs": round(achieved / 8000.0, 4),
                "traffic": profiled_traffic(prof_name),
                "algorithmic_bytes_per_launch": algo, "kernel": "k_step (%s)" % prof_name}
    if kw.get("solid") is not None and args.pattern == "two_lattice":
        # porous workloads: the geometry's fluid DRAM sectors copied without
        # arithmetic (lbm_sector_copy), what HBM delivers for its pattern
        nbytes, tc = sector_copy_time(sim, args.steps, stream)
        roofline["sector_copy"] = {"bytes_per_copy": nbytes, "GBps": round(nbytes / tc / 1e9, 1),
                                   "frac_of_sector_copy": round(tc / step_s, 4)}
    res = {
        "metric": METRIC, "value": round(glups, 3), "unit": "GLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "f32": "f32", "f16s": "f16 storage, f32 compute"}[args.precision],
        "data": "synthetic (seeded Taylor-Green / Poiseuille fields, seeded disc geometries)",
        "config": bench_config(args, kw, nfluid, wname, world),
        "roofline": roofline,
        "e2e": {"value": round(whole_job_glups(nfluid, args.steps, world, t_e2e), 3), "unit": "GLUPS",
                "h2d_bytes_per_step": round(h2d / args.steps, 1), "d2h_bytes_per_step": round(d2h / args.steps, 1),
                "what": "lbm_init_equilibrium reading rho,u from pinned host memory, K x lbm_step, "
                        "lbm_macros writing rho,u into pinned host memory (NVLink-C2C, no staging copies)"},
        "gpu_launches": step_launches,
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
    kw, _, _, nfluid, wname = build_case(args.workload, args.n, args.precision)
    ref_config = bench_config(args, kw, nfluid, wname, 1)
    sample = "FP64 oracle, %d x %d periodic Taylor-Green (sample of the %d^2 workload), %d steps" % (
        S, S, args.n, args.steps)
    return {
        "impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": "GLUPS", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Taylor-Green / Poiseuille fields, seeded disc geometries)",
        "config": ref_config,
        "cpu_baseline": {"value": round(v, 5), "unit": "GLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(v, 5), "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def cpu_baseline_leg(n: int):
    """The oracle on all host threads (the reported value) and on one thread."""
    from oracle import oracle as orc
    orc.build()
    threads = orc.num_threads()
    orc.set_threads(1)
    g1, steps1, dt1, _ = oracle_glups(n, 4.0)
    orc.set_threads(threads)
    g, steps, dt, cores = oracle_glups(n, 12.0)
    return {"value": round(g, 5), "unit": "GLUPS", "cores": cores, "kind": "oracle",
            "single_thread_value": round(g1, 5),
            "sample": "FP64 oracle, %d x %d periodic Taylor-Green, %d steps in %.1f s on %d host threads "
                      "(%d cores in the affinity mask); one thread: %d steps in %.1f s"
                      % (n, n, steps, dt, cores, cpu_cores(), steps1, dt1)}


# ---------------------------------------------------------------- extra lines

def _timed(sim, k, stream):
    return time_steps(sim, k, 10, stream)


def sector_copy_time(sim, k: int, stream):
    """(bytes, seconds) of one lbm_sector_copy: the geometry's fluid DRAM
    sectors, all nine slots, read and written once, no arithmetic; the mean
    of k back-to-back copies after 5 warm-up ones, CUDA events on the
    library's stream."""
    import torch
    nbytes = sim.sector_copy(5)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    sim.sector_copy(k)
    end.record(stream)
    end.synchronize()
    return nbytes, start.elapsed_time(end) / 1e3 / k


def extra_measurements(args):
    """Other rows of the metric, each with fewer steps: every precision and
    pattern on the dense Taylor-Green box, the Poiseuille channel, the porous
    sweep (phi 0.2 / 0.5 / 0.8, tiled layout, fluid-node GLUPS, with the
    sparse computational efficiency eta_P of Eq. 9 against the same layout on
    the all-fluid box), and the adjoint step cost on the cylinder channel."""
    import torch
    from paper_2108_13241_gb300 import inputs, lbm
    out = {}
    peak, _ = peaks()
    stream = torch.cuda.current_stream()

    def record(key, nf, k, t, prec):
        g = nf * k / t / 1e9
        out[key] = {"GLUPS": round(g, 3), "GBps_algorithmic": round(g * node_bytes(prec), 1),
                    "frac_of_measured_hbm": round(g * node_bytes(prec) / peak, 4), "steps": k}
        return g

    kept = {}

    def run(kw, rho, u, prec, layout, pattern, k):
        sim = lbm.LBM(precision=prec, layout=layout, pattern=pattern, **kw)
        sim.init_equilibrium(None if rho is None else torch.as_tensor(rho, dtype=sim.dtype, device="cuda"),
                             None if u is None else torch.as_tensor(u, dtype=sim.dtype, device="cuda"))
        t = _timed(sim, k, stream)
        kept["nodes"] = sim.tile_map()[1].shape[0] * 256 if layout == "sparse" else None
        sim.close()
        del sim
        torch.cuda.empty_cache()
        return t

    def geometry_copy(kw, prec, layout):
        sim = lbm.LBM(precision=prec, layout=layout, pattern="two_lattice", **kw)
        sim.init_equilibrium(None, None)
        cp = sector_copy_time(sim, 100, stream)
        sim.close()
        del sim
        torch.cuda.empty_cache()
        return cp

    n = 4096
    rho, u = inputs.taylor_green(n, n, 0.05)
    kw = dict(nx=n, ny=n, tau=0.8)
    dense_geom = {}
    for prec, layout, pattern, k in [("f64", "dense", "two_lattice", 100), ("f64", "dense", "aa", 100),
                                     ("f32", "dense", "aa", 500), ("f16s", "dense", "two_lattice", 500),
                                     ("f16s", "dense", "aa", 500), ("f32", "sparse", "two_lattice", 500),
                                     ("f32", "sparse", "aa", 500), ("f16s", "sparse", "aa", 500)]:
        t = run(kw, rho, u, prec, layout, pattern, k)
        key = "taylor_green_%d/%s/%s/%s" % (n, prec, layout, pattern)
        dense_geom[(prec, layout, pattern)] = record(key, n * n, k, t, prec)
        if prec == "f64":
            alu = fp64_alu_roofline(dense_geom[(prec, layout, pattern)],
                                    torch.cuda.get_device_properties(0).multi_processor_count)
            if alu is not None:
                out[key]["alu_roofline"] = alu
    fx, rho_p, u_p = inputs.poiseuille(n, n, 0.8, 0.05)
    t = run(dict(nx=n, ny=n, tau=0.8, force=(fx, 0.0), periodic_y=False), rho_p, u_p, "f32", "dense",
            "two_lattice", 500)
    record("poiseuille_%d/f32/dense/two_lattice" % n, n * n, 500, t, "f32")
    # the same channel with the two-relaxation-time collision (Lambda = 3/16)
    t = run(dict(nx=n, ny=n, tau=0.8, force=(fx, 0.0), periodic_y=False, collision="trt", magic=3.0 / 16.0),
            rho_p, u_p, "f32", "dense", "two_lattice", 500)
    record("poiseuille_%d/f32/dense/two_lattice/trt" % n, n * n, 500, t, "f32")
    for phi in (0.2, 0.5, 0.8):
        copies = {}
        solid, achieved, _ = inputs.porous_discs(n, n, phi, rmin=8, rmax=32)
        nf = int((solid == 0).sum())
        kwp = dict(nx=n, ny=n, tau=0.8, solid=solid, force=(1e-6, 0.0), periodic_y=False)
        combos = [("f32", "sparse", "two_lattice"), ("f32", "sparse", "aa"), ("f32", "dense", "two_lattice")]
        if phi == 0.5:
            combos += [("f16s", "sparse", "aa"), ("f64", "sparse", "two_lattice")]
        for prec, layout, pattern in combos:
            k = 100 if prec == "f64" else 300
            t = run(kwp, None, None, prec, layout, pattern, k)
            key = "porous_phi%.2f_%d/%s/%s/%s" % (achieved, n, prec, layout, pattern)
            g = record(key, nf, k, t, prec)
            if kept["nodes"]:
                out[key]["kept_tile_nodes"] = kept["nodes"]
            # the geometry's own bound at DRAM sector granularity
            sec = sector_nodes(solid, prec)
            out[key]["sector_nodes"] = sec
            out[key]["frac_of_sector_roofline"] = round(g * sec / nf * node_bytes(prec) / peak, 4)
            # against what HBM measurably delivers for this geometry's sector
            # pattern in this layout: the copy of its fluid sectors
            if (prec, layout) not in copies:
                copies[(prec, layout)] = geometry_copy(kwp, prec, layout)
            nbytes, tc = copies[(prec, layout)]
            out[key]["sector_copy"] = {"GBps": round(nbytes / tc / 1e9, 1),
                                       "frac_of_sector_copy": round(tc / (t / k), 4)}
            if layout == "sparse" and (prec, layout, pattern) in dense_geom:
                out["porous_phi%.2f_%d/%s/%s/%s" % (achieved, n, prec, layout, pattern)]["eta_P"] = round(
                    g / dense_geom[(prec, layout, pattern)], 3)
            if prec == "f64":
                # the masked tiled FP64 step issues at least the dense step's
                # FP64 instructions per node, so this ceiling is an upper bound
                alu = fp64_alu_roofline(g, torch.cuda.get_device_properties(0).multi_processor_count)
                if alu is not None:
                    alu["note"] = "FP64 instructions per node of the dense step (a lower bound for this step)"
                    out[key]["alu_roofline"] = alu
        out["porous_phi%.2f_%d/fluid_nodes" % (achieved, n)] = nf
    out["d3q19_taylor_green_256"] = d3q19_rows(peak, stream)
    # eta_P of the paper's two sparse geometries (Sec. 4.2.2) at three porosities
    out["eta_P_sweep"] = porosity_sweep(n, 300, names=("random_r8_256", "array_8x8"), phis=(0.3, 0.5, 0.8))
    out["adjoint_channel_512x256"] = adjoint_cost()
    return out


def d3q19_rows(peak: float, stream, n: int = 256, steps: int = 200):
    """The D3Q19 step (lbm3_*) on an n^3 periodic 3-D Taylor-Green box
    (U 0.05, tau 0.8), FP64, FP32 and FP16-shifted storage, `steps` timed
    steps after 10 warm-up ones: GLUPS, the fraction of the 2 x 19 x s bytes
    per node (304 / 152 / 76 B) at the measured HBM peak, and the relative L2
    error of u against the FP64 run after the same steps; FP32 AA on the same
    box; FP32 on an n^3 porous medium of random spheres (porosity 0.5)."""
    import torch
    from paper_2108_13241_gb300 import inputs, lbm
    rho, u = inputs.taylor_green_3d(n, n, n, 0.05)
    rows = {}
    u64 = None
    for prec in ("f64", "f32", "f16s"):
        sim = lbm.LBM3(n, n, n, 0.8, precision=prec)
        sim.init_equilibrium(rho, u)
        t = time_steps(sim, steps, 10, stream)
        _, v = sim.macros()
        v = v.double()
        sim.close()
        del sim
        torch.cuda.empty_cache()
        g = n ** 3 * steps / t / 1e9
        nb = 2 * 19 * BYTES_PER_VALUE[prec]
        rows[prec] = {"GLUPS": round(g, 3), "bytes_per_node": nb, "GBps_algorithmic": round(g * nb, 1),
                      "frac_of_measured_hbm": round(g * nb / peak, 4), "steps": steps,
                      "finite": bool(torch.isfinite(v).all())}
        if prec == "f64":
            alu = fp64_alu_roofline3(g, torch.cuda.get_device_properties(0).multi_processor_count)
            if alu is not None:
                rows[prec]["alu_roofline"] = alu
        if u64 is None:
            u64 = v
        else:
            rows[prec]["rel_l2_u_vs_f64"] = float(torch.linalg.vector_norm(v - u64) / torch.linalg.vector_norm(u64))
        del v
    # the in-place AA pattern, FP32
    sim = lbm.LBM3(n, n, n, 0.8, precision="f32", pattern="aa")
    sim.init_equilibrium(rho, u)
    t = time_steps(sim, steps, 10, stream)
    sim.close()
    del sim
    torch.cuda.empty_cache()
    g = n ** 3 * steps / t / 1e9
    rows["f32_aa"] = {"GLUPS": round(g, 3), "bytes_per_node": 152, "GBps_algorithmic": round(g * 152, 1),
                      "frac_of_measured_hbm": round(g * 152 / peak, 4), "steps": steps}
    # a porous medium of random overlapping spheres (r 8-16, porosity 0.5),
    # periodic, force along x: the masked step with bounce-back, fluid-node
    # GLUPS, two-lattice and AA, FP32; the library's own choice (AA: the node
    # list; two lattices: the dense grid) and, for comparison, the other one
    solid, phi = inputs.porous_spheres_3d(n, 0.5)
    # nodes of the 32-byte sectors (8 FP32 nodes along x) that hold fluid:
    # at sector granularity a step moves 152 B per such node
    sec = sector_nodes(solid.reshape(-1, n), "f32")
    for pattern in ("two_lattice", "aa"):
        for mode in ("auto", "never" if pattern == "aa" else "always"):
            sim = lbm.LBM3(n, n, n, 0.8, solid=solid, force=(1e-6, 0.0, 0.0), precision="f32", pattern=pattern,
                           node_list=mode)
            nf, nl = sim.fluid_nodes, sim.list_nodes
            sim.init_equilibrium(None, None)
            t = time_steps(sim, steps, 10, stream)
            sim.close()
            del sim
            torch.cuda.empty_cache()
            g = nf * steps / t / 1e9
            key = "porous_spheres_phi%.2f/f32/%s" % (phi, pattern) + {"auto": "", "never": "/dense_grid",
                                                                        "always": "/node_list"}[mode]
            rows[key] = {"GLUPS": round(g, 3), "fluid_nodes": nf, "listed_nodes": nl,
                         "GBps_algorithmic": round(g * 152, 1), "frac_of_measured_hbm": round(g * 152 / peak, 4),
                         "sector_nodes": sec, "frac_of_sector_roofline": round(g * sec / nf * 152 / peak, 4),
                         "steps": steps}
    return rows


def d3q19_large(peak: float, stream, n: int = 1024, steps: int = 20, pattern: str = "two_lattice"):
    """The D3Q19 FP32 step on a large box from rest -- 1024^3 two-lattice
    (1.07e9 nodes, 163 GB) or 1280^3 AA (2.1e9 nodes, one 159 GB lattice),
    64-bit slot offsets: the working sets the GPU's memory allows, timed
    like the other rows."""
    import torch
    from paper_2108_13241_gb300 import lbm
    sim = lbm.LBM3(n, n, n, 0.8, precision="f32", pattern=pattern)
    sim.init_equilibrium(None, None)
    t = time_steps(sim, steps, 5, stream)
    gb = sim.workspace.numel() / 1e9
    sim.close()
    del sim
    torch.cuda.empty_cache()
    g = n ** 3 * steps / t / 1e9
    return {"GLUPS": round(g, 3), "pattern": pattern, "workspace_GB": round(gb, 1),
            "GBps_algorithmic": round(g * 152, 1), "frac_of_measured_hbm": round(g * 152 / peak, 4), "steps": steps}


def porosity_sweep(n: int = 4096, steps: int = 300, names=None, phis=None):
    """Sparse computational efficiency eta_P (Eq. 9) over porosity, Sec. 4.2.2's
    sweep: random discs r in [8, 256] (phi 0.1 .. 0.9), the regular 8 x 8 disc
    array (phi 0.3 .. 0.9) and the r in [8, 32] discs of the porous workload
    (phi 0.1 .. 0.9); FP32, two-lattice, periodic x, walls y, F = (1e-6, 0).
    Each geometry runs in the tiled layout (only tiles with fluid stored) and
    in the dense layout with the per-node link mask (the paper's bitmask-node
    comparison); eta_P divides each by the same layout on the all-fluid box
    with the same sides.  GLUPS count fluid nodes only.  names / phis select
    generators and porosities (default: all of them)."""
    import torch
    from paper_2108_13241_gb300 import inputs, lbm
    stream = torch.cuda.current_stream()
    peak, _ = peaks()
    base = dict(nx=n, ny=n, tau=0.8, force=(1e-6, 0.0), periodic_y=False)

    def glups(solid, layout):
        sim = lbm.LBM(precision="f32", layout=layout, pattern="two_lattice", solid=solid, **base)
        nf = sim.fluid_nodes
        sim.init_equilibrium(None, None)
        t = time_steps(sim, steps, 10, stream)
        tiles = sim.tile_map()[1].shape[0] if layout == "sparse" else None
        copy = sector_copy_time(sim, steps, stream) if solid is not None else None
        sim.close()
        del sim
        torch.cuda.empty_cache()
        return nf * steps / t / 1e9, nf, tiles, (None if copy is None else (copy[0] / copy[1] / 1e9,
                                                                            copy[1] / (t / steps)))

    ref = {lay: glups(None, lay)[0] for lay in ("sparse", "dense")}
    res = {"all_fluid": {lay: round(g, 3) for lay, g in ref.items()}}
    gens = [("random_r8_256", [round(0.1 * k, 1) for k in range(1, 10)],
             lambda phi: inputs.porous_discs(n, n, phi, rmin=8, rmax=256)[:2]),
            ("array_8x8", [round(0.1 * k, 1) for k in range(3, 10)],
             lambda phi: inputs.circle_array(n, n, phi, 8)[:2]),
            ("random_r8_32", [round(0.1 * k, 1) for k in range(1, 10)],
             lambda phi: inputs.porous_discs(n, n, phi, rmin=8, rmax=32)[:2])]
    for name, gen_phis, gen in gens:
        if names is not None and name not in names:
            continue
        rows = []
        for phi in (gen_phis if phis is None else phis):
            solid, achieved = gen(phi)
            row = {"phi": round(achieved, 4)}
            for lay in ("sparse", "dense"):
                g, nf, tiles, cp = glups(solid, lay)
                row[lay] = {"GLUPS": round(g, 3), "eta_P": round(g / ref[lay], 3),
                            "frac_of_measured_hbm": round(g * node_bytes("f32") / peak, 4)}
                if cp is not None:
                    row[lay]["sector_copy_GBps"] = round(cp[0], 1)
                    row[lay]["frac_of_sector_copy"] = round(cp[1], 4)
                if tiles is not None:
                    row["kept_tiles"] = int(tiles)
                row[lay]["frac_of_sector_roofline"] = round(
                    g * sector_nodes(solid, "f32") / nf * node_bytes("f32") / peak, 4)
            row["fluid_nodes"] = int(nf)
            rows.append(row)
        res[name] = rows
    return {"sweep": "porosity", "n": n, "steps": steps, "precision": "f32", "results": res}


def channel_runs(steps: int = 1_000_000):
    """The paper's channel validation (Sec. 4.1.2): 4096 x 512 nodes, walls
    south/north, nu = 0.25 (tau = 1.25), pressure outlet rho = 1 on the east
    side; chan_v: velocity inlet u_x = 0.1 on the west side, initial rho = 1;
    chan_p: pressure inlet rho = 1.016, initial rho = 1.008; initial u = 0;
    FP32 (the paper's precision), 10^6 steps.  Reports the velocity profile at
    x = 15 R (R = 256, half the channel height): its maximum (the paper
    prints 0.158 for chan_v and 0.160 for chan_p) and its deviation from the
    best-fitting parabola vanishing at the half-way walls."""
    import torch
    from paper_2108_13241_gb300 import lbm
    nx, ny, R = 4096, 512, 256
    stream = torch.cuda.current_stream()
    out = {}
    for name, inlet, rho0 in (("chan_v", ("velocity", (0.1, 0.0)), 1.0), ("chan_p", ("pressure", 1.016), 1.008)):
        sim = lbm.LBM(nx=nx, ny=ny, tau=1.25, periodic_x=False, periodic_y=False, precision="f32",
                      open={"west": inlet, "east": ("pressure", 1.0)})
        sim.init_equilibrium(torch.full((ny, nx), rho0, dtype=torch.float32, device="cuda"), None)
        t = time_steps(sim, steps, 0, stream)
        rho, u = sim.macros()
        prof = u[0][:, 15 * R].double().cpu().numpy()
        y = np.arange(ny) + 0.5
        shape = y * (ny - y) / (ny * ny / 4.0)
        amp = float(prof @ shape / (shape @ shape))
        out[name] = {"v_max": round(float(prof.max()), 5), "paper_v_max": 0.158 if name == "chan_v" else 0.160,
                     "parabola_v_max": round(amp, 5),
                     "max_dev_from_parabola_rel": round(float(np.abs(prof - amp * shape).max() / amp), 5),
                     "rho_inlet_mean": round(float(rho[:, 0].double().mean()), 6),
                     "GLUPS": round(nx * ny * steps / t / 1e9, 3), "seconds": round(t, 2), "steps": steps}
        sim.close()
        del sim
        torch.cuda.empty_cache()
    return {"sweep": "channels", "results": out}


def adjoint_cost(nx=512, ny=256, T=2000, K=45, count=12, rmin=6, rmax=12):
    """Cost of one adjoint step relative to one forward step on the
    differentiable channel (default: 512 x 256, 12 cylinders, FP32,
    T = 2000, checkpoint every 45): backward wall time (recompute + adjoint)
    / T over plain forward step time."""
    import torch
    from paper_2108_13241_gb300 import autograd as ag, inputs, lbm
    solid, _ = inputs.channel_cylinders(nx, ny, count=count, rmin=rmin, rmax=rmax, clearance=2)
    F = np.zeros((2, ny, nx), np.float32)
    F[0] = 1e-5
    ut = torch.as_tensor(inputs.target_velocity(nx, ny, solid), dtype=torch.float32, device="cuda")
    sim = lbm.LBM(nx, ny, 0.8, solid=solid, periodic_y=False, precision="f32")
    Ft = torch.as_tensor(F, device="cuda")
    sim.set_force(Ft)
    stream = torch.cuda.current_stream()
    t_step = time_steps(sim, T, 20, stream) / T
    fl = torch.as_tensor(solid == 0, device="cuda")
    for _ in range(2):  # the first pass warms the allocator (checkpoint buffers)
        sim.init_equilibrium(None, None)
        Fg = Ft.clone().requires_grad_(True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        rho, u = ag.simulate(sim, T, None, Fg, K=K)
        loss = (((u - ut) ** 2).sum(0) * fl).sum() / fl.sum()
        ev[1].record(stream)
        loss.backward()
        ev[2].record(stream)
        ev[2].synchronize()
    t_fwd = ev[0].elapsed_time(ev[1]) / 1e3
    t_bwd = ev[1].elapsed_time(ev[2]) / 1e3
    nf = int((solid == 0).sum())
    # the adjoint kernel's share of a backward step: one recompute step is
    # the rest; algorithmic bytes of k_adjoint: 33 FP32 values per node
    t_adj = max(t_bwd / T - t_step, 1e-12)
    return {"forward_step_us": round(t_step * 1e6, 2),
            "checkpointed_forward_step_us": round(t_fwd / T * 1e6, 2),
            "backward_step_us": round(t_bwd / T * 1e6, 2),
            "adjoint_over_forward": round(t_bwd / T / t_step, 3),
            "adjoint_kernel_GBps_algorithmic": round(nf * 33 * 4 / t_adj / 1e9, 1),
            "grad_finite": bool(torch.isfinite(Fg.grad).all().item())}


def _accuracy_runs(cases, steps, precisions, stream, pattern="aa"):
    """For each case: GLUPS of each precision and the relative L2 norm of u
    over fluid nodes against the FP64 GPU run of the same case."""
    import torch
    from paper_2108_13241_gb300 import lbm
    res = {}
    for name, kw, r0, u0, nf, fl, layout in cases:
        ref_u = None
        for prec in ("f64",) + tuple(precisions):
            sim = lbm.LBM(precision=prec, layout=layout, pattern=pattern, **kw)
            sim.init_equilibrium(None if r0 is None else torch.as_tensor(r0, dtype=sim.dtype, device="cuda"),
                                 None if u0 is None else torch.as_tensor(u0, dtype=sim.dtype, device="cuda"))
            torch.cuda.synchronize()
            start = torch.cuda.Event(enable_timing=True)
            end = torch.cuda.Event(enable_timing=True)
            start.record(stream)
            sim.step(steps)
            end.record(stream)
            end.synchronize()
            t = start.elapsed_time(end) / 1e3
            _, uu = sim.macros()
            uu = uu.double()
            if fl is not None:
                uu = uu * fl
            entry = {"GLUPS": round(nf * steps / t / 1e9, 3), "layout": layout, "pattern": pattern}
            if ref_u is None:
                ref_u = uu
            else:
                entry["rel_l2_u_vs_f64"] = float(torch.linalg.vector_norm(uu - ref_u) /
                                                 torch.linalg.vector_norm(ref_u))
            res["%s/%s" % (name, prec)] = entry
            sim.close()
            del sim, uu
            torch.cuda.empty_cache()
    return res


def precision_sweep(n: int = 8192, steps: int = 5000):
    """Precision sweep: dense Taylor-Green (U 0.05) and the porous medium
    (phi 0.3, same disc generator, F = 1e-6) at n^2, FP64 vs FP32 vs FP16s
    storage, `steps` steps each, in the in-place AA pattern; plus the dense
    Taylor-Green and Poiseuille boxes at 1024^2 .. 4096^2 after 1000 steps,
    two-lattice.  Errors are relative L2 norms
    of u over fluid nodes against the FP64 GPU run (itself pinned to the CPU
    oracle on the smaller configurations), reported beside GLUPS."""
    import torch
    from paper_2108_13241_gb300 import inputs
    stream = torch.cuda.current_stream()
    rho, u = inputs.taylor_green(n, n, 0.05)
    solid, achieved, _ = inputs.porous_discs(n, n, 0.3, rmin=8, rmax=32)
    big = [("taylor_green_%d" % n, dict(nx=n, ny=n, tau=0.8), rho, u, n * n, None, "dense"),
           ("porous_phi%.2f_%d" % (achieved, n),
            dict(nx=n, ny=n, tau=0.8, solid=solid, force=(1e-6, 0.0), periodic_y=False),
            None, None, int((solid == 0).sum()), torch.as_tensor(solid == 0, device="cuda"), "sparse")]
    del rho, u
    res = {"steps_%d" % steps: _accuracy_runs(big, steps, ("f32", "f16s"), stream)}
    small = []
    for m in (1024, 2048, 4096):
        r, v = inputs.taylor_green(m, m, 0.05)
        small.append(("taylor_green_%d" % m, dict(nx=m, ny=m, tau=0.8), r, v, m * m, None, "dense"))
        fx, r, v = inputs.poiseuille(m, m, 0.8, 0.05)
        small.append(("poiseuille_%d" % m, dict(nx=m, ny=m, tau=0.8, force=(fx, 0.0), periodic_y=False),
                      r, v, m * m, None, "dense"))
    res["steps_1000"] = _accuracy_runs(small, 1000, ("f32", "f16s"), stream, pattern="two_lattice")
    return {"sweep": "precision", "results": res}


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
    ap.add_argument("--sweep", action="store_true",
                    help="run the 8192^2 FP64/FP32/FP16s precision sweep instead of the benchmark")
    ap.add_argument("--porosity-sweep", action="store_true",
                    help="run the 4096^2 eta_P sweep over porosity instead of the benchmark")
    ap.add_argument("--channels", action="store_true",
                    help="run the paper's two channel flows (4096 x 512, 10^6 steps) instead of the benchmark")
    ap.add_argument("--adjoint", action="store_true",
                    help="run the adjoint cost on the 512 x 256 channel and on a 2048 x 2048 one")
    ap.add_argument("--d3q19", action="store_true",
                    help="run the D3Q19 step on an n^3 3-D Taylor-Green box and an n^3 porous medium of "
                         "spheres (n = --n, default 256 here), plus a 1024^3 two-lattice and a 1280^3 AA box "
                         "from rest unless --n is given")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.d3q19:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        n = 256 if args.n == 4096 else args.n
        res = {"sweep": "d3q19", "n": n, "results": d3q19_rows(peaks()[0], torch.cuda.current_stream(), n)}
        if args.n == 4096:
            # the large boxes (163 / 159 GB) only in the default form of this mode
            res["rest_1024"] = d3q19_large(peaks()[0], torch.cuda.current_stream())
            res["rest_1280_aa"] = d3q19_large(peaks()[0], torch.cuda.current_stream(), n=1280, pattern="aa")
        print(json.dumps(res), flush=True)
        return 0
    if args.sweep or args.porosity_sweep or args.channels or args.adjoint:
        import __graft_entry__
        __graft_entry__.build()
        if args.sweep:
            res = precision_sweep()
        elif args.porosity_sweep:
            res = porosity_sweep()
        elif args.channels:
            res = channel_runs()
        else:
            res = {"sweep": "adjoint", "results": {
                "channel_512x256_T2000_K45": adjoint_cost(),
                "channel_2048x2048_T40_K8": adjoint_cost(2048, 2048, 40, 8, count=96, rmin=12, rmax=24)}}
        print(json.dumps(res), flush=True)
        return 0

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
