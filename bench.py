"""Benchmark of the matrix-free p-Laplacian Jacobian action and Newton-CG solve on one GB300.

Workload: 3D p-Laplacian p=3 on a 64^3 hex lattice with seeded jitter, order 3 (7,189,057 DOFs),
4^3 Gauss points per element, linearised at the seeded smooth state, FP64.  One timed step is one
partially assembled Jacobian action y = J(u) v in FP64 (Eq. 2), the headline `value`, graded
against the measured FP64 fused multiply-add rate.  Measured in the same run and reported beside
it: the FP32 action (the operator the mixed-precision CG applies) with its HBM roofline, the
double-float action, the FP64 residual, the FP64 action end to end through host buffers, and the
full Newton-CG solves (FP64 and mixed precision, to 1e-8 relative residual).

Prints one JSON line.  ``--impl reference`` times the oracle (plain FP64 C on the host cores) on
a bounded sample of the same workload instead.  Under torchrun (N > 1) the ranks split one problem
by the subdomain restriction P: each holds a 64^3-element z-slab of a 64 x 64 x 64N lattice (weak
scaling), and a step is the split FP64 Jacobian action, whose interface planes the neighbours
exchange (NCCL; ``--backend gloo`` stages them through host memory); timing is the max over
ranks and the value counts the DOFs of the whole lattice.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Jacobian action GDOF/s; Newton solve time to 1e-8 rel residual, FP64 vs mixed"
WORKLOAD = "3d_p3_k3_64"
# Newton modes (name, inner precision); fp64 last, the others are timed against it
NEWTON_MODES = (("mixed", -32), ("mixed_fp32_cg", 32), ("double_float", 48), ("fp64", 64))


# ------------------------------------------------------------------------------------------------
# distributed helpers (host logic; tested on CPU with gloo)
# ------------------------------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        if device is not None and getattr(device, "type", "cpu") == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def aggregate(units_per_rank: float, seconds_per_rank: float, world: int, device=None) -> tuple[float, float]:
    """Whole-job throughput: units of all ranks / max time over ranks (weak scaling)."""
    t = max_over_ranks(seconds_per_rank, device)
    return units_per_rank * world / t, t


# ------------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2])); power.append(float(f[3]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() in ("active", "1", "0x1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ------------------------------------------------------------------------------------------------
# roofline bookkeeping
# ------------------------------------------------------------------------------------------------
def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


FP64_NOMINAL_TFLOPS = 1.25   # nominal dense FP64 rate of the GB300 (context only)
FP64_PEAK_FILE = os.path.join(ROOT, "profiles", "fp64_peak.json")


def fp64_peak() -> dict:
    """The FP64 rate the FP64 kernels are graded against: the committed measurement of this GPU
    model's FMA rate (written by ``bench.py --suite fp64-peak``), else the nominal figure."""
    if os.path.exists(FP64_PEAK_FILE):
        d = json.load(open(FP64_PEAK_FILE))
        return {"tflops": float(d["tflops_best"]), "source": "measured (profiles/fp64_peak.json)"}
    return {"tflops": FP64_NOMINAL_TFLOPS, "source": "nominal"}


def jv_algorithmic_flops(dim: int, n_e: int, d1: int, q1: int) -> float:
    """Flops of one partially assembled J v: per element, interpolation plus collocated gradient
    in both directions (4 d D1^(d+1) multiply-adds) and the symmetric d x d matvec per point."""
    return 2.0 * n_e * (4 * dim * d1 ** (dim + 1) + dim * dim * q1 ** dim)


def residual_algorithmic_flops(dim: int, n_e: int, d1: int, q1: int) -> float:
    """Flops of one residual R(u): the same contractions as J v (4 d D1^(d+1) multiply-adds per
    element) plus, per point, M g (d^2 multiply-adds), g . M g / (w det J) (d + 1) and the flux
    kappa M g (d multiplies); the power kappa = (eps^2 + sigma)^((p-2)/2) is not counted."""
    per_point = 2 * dim * dim + 2 * (dim + 1) + dim
    return 2.0 * n_e * 4 * dim * d1 ** (dim + 1) + n_e * q1 ** dim * per_point


def jv_algorithmic_bytes(n_l: int, n_e: int, nq_per_elem: int, nl_per_elem: int, word: int) -> int:
    """Bytes a partially assembled J v must move: read v and write y (N_L words each), read the
    6 symmetric tangent entries per quadrature point, read the element index (4 B per E-vector
    entry)."""
    return 2 * word * n_l + 6 * word * n_e * nq_per_elem + 4 * n_e * nl_per_elem


def kernel_source_hash() -> str:
    """Hash of the sources that define the Jacobian kernels: the kernel headers and the device
    parameter blocks of internal.h (the host context that follows them does not enter)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2506_00746_gb300", "csrc")
    for f in ("element_kernels.cuh", "jv_tile.cuh", "res_tile.cuh", "tma.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    internal = open(os.path.join(csrc, "internal.h"), "rb").read()
    h.update(internal.split(b"// The context.")[0])
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str) -> tuple[float | None, str | None]:
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was taken on the
    current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None, None
    d = json.load(open(path))
    e = d.get(kernel)
    if not e or e.get("kernel_source_hash") != kernel_source_hash():
        return None, None
    return float(e["dram_bytes_per_launch"]), e.get("summary")


# ------------------------------------------------------------------------------------------------
# the GPU arm
# ------------------------------------------------------------------------------------------------
def run_gpu(args) -> dict | None:
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2506_00746_gb300 import Operator
    from paper_2506_00746_gb300 import abi
    from paper_2506_00746_gb300 import inputs as I

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=dev)
    w = I.WORKLOADS[args.workload]
    V = I.lattice_vertices(w.dim, w.n, seed=w.mesh_seed)
    op = Operator(w.dim, w.n, w.order, V, p=w.p, eps=w.eps)
    nl, ne = op.n_dofs, op.n_elements
    nq = (w.order + 1) ** w.dim
    u0 = torch.from_numpy(I.smooth_field(w.dim, w.n, w.order, seed=w.state_seed)).to(dev)
    v64 = torch.from_numpy(I.uniform_vector(nl, seed=w.dir_seed)).to(dev)
    v32 = v64.float()
    y32 = torch.empty_like(v32)
    y64 = torch.empty_like(v64)
    op.linearize(u0)
    stream = torch.cuda.current_stream()

    def timed(fn, steps, warmup):
        """K calls between barriers and synchronisations, CUDA events on the launching stream."""
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        barrier(dev)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = op.launch_count()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(dev)
        return e0.elapsed_time(e1) / 1e3, op.launch_count() - l0

    def call_median(fn, calls):
        """Median of `calls` individually event-timed calls (ms)."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(calls)]
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in ev)

    def kernel_ms(fn, calls):
        """Per-kernel average durations (ms) from the library's own events around each launch."""
        op.prof_enable(True)
        op.prof_reset()
        for _ in range(calls):
            fn()
        prof = op.prof_read()
        op.prof_enable(False)
        return {k: ms / n for k, (n, ms) in prof.items() if n > 0}

    ncalls = max(50, args.steps)

    # ---- headline: FP64 partially assembled Jacobian action, device-resident inputs ----
    jv64 = lambda: op.jacobian_action(v64, precision=64, out=y64)
    clk = ClockSampler(local).start()
    t_dev, launches = timed(jv64, args.steps, args.warmup)
    clocks = clk.stop()
    value, t_max = aggregate(nl * args.steps / 1e9, t_dev, world, dev)
    med64 = call_median(jv64, ncalls)
    k64 = kernel_ms(jv64, ncalls)
    t_main64 = k64.get("jv_pa_f64", float("nan")) / 1e3
    t_fix64 = k64.get("fixup", 0.0) / 1e3
    y64_host = y64.cpu().numpy() if rank == 0 else None

    # ---- the FP32 action (inner operator of the mixed-precision CG): HBM roofline ----
    jv32 = lambda: op.jacobian_action(v32, precision=32, out=y32)
    t32, l32 = timed(jv32, ncalls, args.warmup)
    med32 = call_median(jv32, ncalls)
    k32 = kernel_ms(jv32, ncalls)
    t_main32 = k32.get("jv_pa_f32", float("nan")) / 1e3
    t_fix32 = k32.get("fixup", 0.0) / 1e3
    y32_host = y32.double().cpu().numpy() if rank == 0 else None

    # ---- other operators of the path ----
    jvdf = lambda: op.jacobian_action(v64, precision=48, out=y64)
    jvdf()                       # splits the FP64 tangent into word pairs (once per linearisation)
    tdf, _ = timed(jvdf, ncalls, 3)
    ydf_host = y64.cpu().numpy() if rank == 0 else None
    jvcg = lambda: op.jacobian_action(v64, precision=-32, out=y64)
    tcg, _ = timed(jvcg, ncalls, 3)
    r = torch.empty_like(u0)
    res = lambda: op.residual(u0, out=r)
    tres, _ = timed(res, ncalls, 3)
    kres = kernel_ms(res, 10)
    t_res_main = kres.get("residual", float("nan")) / 1e3
    r_host = r.cpu().numpy() if rank == 0 else None
    # linearisation at the same state: the tangent (FP64 and FP32 copies) and the Jacobi diagonal
    lin = lambda: op.linearize(u0)
    tlin, _ = timed(lin, 10, 2)
    klin = kernel_ms(lin, 5)
    f64peak = fp64_peak()
    live_best, live_med = abi.fe_measure_fp64_peak(10)

    # ---- end to end through the C ABI with host buffers (copies inside the timed region) ----
    vh = v64.cpu().pin_memory()
    yh = torch.empty_like(vh).pin_memory()
    for _ in range(3):
        op.jacobian_action_host(vh, yh, precision=64)
    torch.cuda.synchronize()
    barrier(dev)
    ne2e = max(5, args.steps)
    t0 = time.perf_counter()
    for _ in range(ne2e):
        op.jacobian_action_host(vh, yh, precision=64)
    t_e2e = time.perf_counter() - t0
    e2e_value, _ = aggregate(nl * ne2e / 1e9, t_e2e, world, dev)

    # ---- Newton solves: FP64 and mixed precision to 1e-8 ----
    newton = {}
    if not args.no_newton:
        # mixed: FP32 J v inside an FP64 CG; mixed_fp32_cg: FP32 J v and FP32 CG vectors with
        # compensated inner products; double_float: double-float J v inside an FP64 CG; fp64:
        # everything FP64
        for name, prec in NEWTON_MODES:
            u = u0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = op.newton_solve(u, rtol=1e-8, inner_precision=prec, max_newton=args.max_newton,
                                  raise_on_error=False)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            newton[name] = {"time_s": round(max_over_ranks(wall, dev), 4), "status": rep["status"],
                            "newton_iters": rep["newton_iters"], "cg_iters": rep["cg_iters"],
                            "rel_residual": rep["rel"], "cg_time_s": round(rep["cg_ms"] / 1e3, 4),
                            "kernel_launches": rep["launches"]}
            if name == "mixed":
                u_mixed_host = u.cpu().numpy() if rank == 0 else None
        for name, _ in NEWTON_MODES[:-1]:
            if "fp64" in newton and name in newton:
                newton[f"speedup_{name}_vs_fp64"] = round(newton["fp64"]["time_s"] / newton[name]["time_s"], 3)
        # the same solves with Eisenstat-Walker choice 2 inner tolerances (forcing 1)
        ew = {}
        for name, prec in NEWTON_MODES:
            u = u0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = op.newton_solve(u, rtol=1e-8, inner_precision=prec, max_newton=args.max_newton, forcing=1,
                                  raise_on_error=False)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            ew[name] = {"time_s": round(max_over_ranks(wall, dev), 4), "status": rep["status"],
                        "newton_iters": rep["newton_iters"], "cg_iters": rep["cg_iters"],
                        "rel_residual": rep["rel"]}
        for name, _ in NEWTON_MODES[:-1]:
            ew[f"speedup_{name}_vs_fp64"] = round(ew["fp64"]["time_s"] / ew[name]["time_s"], 3)
        newton["eisenstat_walker"] = ew
        newton["small_cases"] = small_newton_cases(Operator, I)
    else:
        u_mixed_host = None

    if rank != 0:
        op.close()
        return None

    peaks = measured_peaks()
    flops64 = jv_algorithmic_flops(w.dim, ne, w.order + 1, w.order + 1)
    achieved64 = flops64 / t_main64 / 1e12
    k64name = "k_jv_tile<4,2,double,double>"
    traffic64, traffic64_src = profiled_traffic(k64name)
    bytes64 = jv_algorithmic_bytes(nl, ne, nq, nq, 8)
    bytes32 = jv_algorithmic_bytes(nl, ne, nq, nq, 4)
    k32name = "k_jv_tile2<4,2,float>"
    traffic32, traffic32_src = profiled_traffic(k32name)
    traffic_fix32, _ = profiled_traffic("k_fixup<float,float>")
    flops_res = residual_algorithmic_flops(w.dim, ne, w.order + 1, w.order + 1)
    traffic_res, traffic_res_src = profiled_traffic("k_res_tile<4,2,1,0>")
    out = {
        "metric": METRIC,
        "value": round(value, 4),
        "unit": "GDOF/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_max / args.steps * 1e3, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded jittered lattice, seeded smooth state, seeded U[-1,1] direction)",
        "config": {"workload": f"{args.workload}: 3D p-Laplacian p=3, 64^3 hex, order 3, 4^3 Gauss points, "
                               f"{nl} DOFs; step = one FP64 partially assembled J(u) v",
                   "n_dofs": nl, "n_elements": ne, "order": w.order, "p": w.p,
                   "l2": "inputs larger than L2 (FP64 tangent %.0f MB + index/vectors)" % (6 * 8 * ne * nq / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   # the library's default tile edge of 3D order k (elements per CTA = tile^3)
                   "tile": {1: 4, 2: 3, 3: 2, 4: 2, 5: 2, 6: 1}[w.order]},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": {"bound": "fp64", "achieved": round(achieved64, 4), "peak": round(f64peak["tflops"], 4),
                     "unit": "TFLOP/s", "frac": round(achieved64 / f64peak["tflops"], 4), "traffic": traffic64,
                     "kernel": k64name, "peak_source": f64peak["source"],
                     "peak_live_best_tflops": round(live_best, 4), "peak_live_median_tflops": round(live_med, 4),
                     "algorithmic_flops_per_launch": flops64, "algorithmic_bytes_per_launch": bytes64,
                     "kernel_ms": round(t_main64 * 1e3, 5), "fixup_ms": round(t_fix64 * 1e3, 5),
                     "hbm_frac": round(bytes64 / t_main64 / 1e9 / peaks["hbm_gbs"], 4),
                     "action_frac": round(flops64 / (t_dev / args.steps) / 1e12 / f64peak["tflops"], 4),
                     "call_ms_median": round(med64, 5), "traffic_summary": traffic64_src},
        "e2e": {"value": round(e2e_value, 4), "unit": "GDOF/s", "h2d_bytes_per_step": 8 * nl,
                "d2h_bytes_per_step": 8 * nl},
        "jv_f32": {"gdofs": round(nl * ncalls / t32 / 1e9, 4), "ms_per_action": round(t32 / ncalls * 1e3, 5),
                   "call_ms_median": round(med32, 5), "launches_per_action": l32 / ncalls,
                   "roofline": {"bound": "hbm", "unit": "GB/s", "peak": peaks["hbm_gbs"],
                                "peak_source": peaks["source"], "kernel": k32name,
                                "algorithmic_bytes_per_launch": bytes32,
                                "kernel_ms": round(t_main32 * 1e3, 5), "fixup_ms": round(t_fix32 * 1e3, 5),
                                "kernel_achieved": round(bytes32 / t_main32 / 1e9, 1),
                                "kernel_frac": round(bytes32 / t_main32 / 1e9 / peaks["hbm_gbs"], 4),
                                "action_frac": round(bytes32 / (t32 / ncalls) / 1e9 / peaks["hbm_gbs"], 4),
                                "traffic": traffic32, "fixup_traffic": traffic_fix32,
                                "action_traffic_ratio": (round((traffic32 + traffic_fix32) / bytes32, 4)
                                                         if traffic32 and traffic_fix32 else None),
                                "traffic_summary": traffic32_src}},
        "jv_double_float_gdofs": round(nl * ncalls / tdf / 1e9, 4),
        "jv_cg_mixed_gdofs": round(nl * ncalls / tcg / 1e9, 4),
        "residual_f64": {"gdofs": round(nl * ncalls / tres / 1e9, 4), "kernel_ms": round(t_res_main * 1e3, 5),
                         "algorithmic_flops": flops_res,
                         "fp64_frac": round(flops_res / t_res_main / 1e12 / f64peak["tflops"], 4),
                         "traffic": traffic_res, "traffic_summary": traffic_res_src,
                         "linearize_ms": round(tlin / 10 * 1e3, 5),
                         "linearize_kernel_ms": {k: round(v, 5) for k, v in klin.items()}},
        "newton": newton,
        "kernel_ms": {"f64": {k: round(v, 5) for k, v in k64.items()},
                      "f32": {k: round(v, 5) for k, v in k32.items()}},
    }
    op.close()
    if not args.no_cpu_baseline:
        gpu = {"r": r_host, "jv_f64": y64_host, "jv_f32": y32_host, "jv_double_float": ydf_host,
               "newton_mixed_u": u_mixed_host}
        out["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_seconds, gpu)
    return out


def run_split(args) -> dict | None:
    """N > 1: one problem split across the ranks by the subdomain restriction P (weak scaling).
    Every rank holds a z-slab of 64^3 order-3 elements of the lattice 64 x 64 x 64N (each slab
    the 64^3 workload's jittered cube, shifted to z in [rank, rank + 1], its interface planes
    unjittered so that neighbours agree); one step is the split FP64 Jacobian action: the local
    action, then one exchange of the two interface planes with the neighbours."""
    import torch
    import torch.distributed as dist

    from paper_2506_00746_gb300 import Operator
    from paper_2506_00746_gb300 import dist as D
    from paper_2506_00746_gb300 import inputs as I

    world, rank, local = dist_env()
    ndev = torch.cuda.device_count()
    torch.cuda.set_device(local % ndev)
    dev = torch.device("cuda", local % ndev)
    if not dist.is_initialized():
        if args.backend == "nccl":
            dist.init_process_group("nccl", device_id=dev)
        else:
            dist.init_process_group("gloo")
    staging = args.backend != "nccl"
    w = I.WORKLOADS[args.workload]
    part = D.SlabPartition(w.n, w.order, world, nz=w.n * world)
    V = I.lattice_vertices(3, w.n, seed=w.mesh_seed + rank).copy()
    V[:, 2] += rank
    op = Operator(3, part.elements(rank), w.order, V, p=w.p, eps=w.eps, natural_faces=part.natural_faces(rank))
    be = D.LibraryBackend(op)
    comm = D.TorchComm(rank, world, staging=staging)
    solver = D.SlabSolver(part, rank, be, comm)
    u0 = torch.from_numpy(I.smooth_field(3, w.n, w.order, seed=w.state_seed)).to(dev)
    v = torch.from_numpy(I.uniform_vector(op.n_dofs, seed=w.dir_seed + rank)).to(dev)
    # the shared planes must agree: take the lower neighbour's top plane
    pl = part.plane
    lo, _ = comm.exchange(v[:pl].clone(), v[-pl:].clone())
    if lo is not None:
        v[:pl] = lo
    be.linearize(u0)
    y = be.zeros()
    stream = torch.cuda.current_stream()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        barrier(dev if args.backend == "nccl" else None)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = op.launch_count()
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        barrier(dev if args.backend == "nccl" else None)
        # the exchange synchronises the host (gloo staging): take the larger of device and wall time
        return max(e0.elapsed_time(e1) / 1e3, wall if staging else 0.0), op.launch_count() - l0

    jv64 = lambda: solver.jv(v, y, 64)
    clk = ClockSampler(local % ndev).start()
    t_dev, launches = timed(jv64, args.steps, args.warmup)
    clocks = clk.stop()
    t_max = max_over_ranks(t_dev, dev if args.backend == "nccl" else None)
    value = part.n_dofs * args.steps / t_max / 1e9
    y32 = be.zeros()
    jv32 = lambda: solver.jv(v, y32, -32)
    t32, _ = timed(jv32, args.steps, 3)
    t32 = max_over_ranks(t32, dev if args.backend == "nccl" else None)
    # end to end: the rank's slice from pinned host memory, the split action, the result back
    vh = v.cpu().pin_memory()
    yh = torch.empty_like(vh).pin_memory()
    vd = torch.empty_like(v)

    def e2e():
        vd.copy_(vh, non_blocking=True)
        solver.jv(vd, y, 64)
        yh.copy_(y, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    for _ in range(3):
        e2e()
    barrier(dev if args.backend == "nccl" else None)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e()
    t_e2e = max_over_ranks(time.perf_counter() - t0, dev if args.backend == "nccl" else None)
    newton = {}
    if not args.no_newton:
        for name, prec in (("mixed", -32), ("fp64", 64)):
            u = u0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = solver.newton(u, rtol=1e-8, precision=prec, max_newton=args.max_newton)
            torch.cuda.synchronize()
            newton[name] = {"time_s": round(max_over_ranks(time.perf_counter() - t0,
                                                           dev if args.backend == "nccl" else None), 4),
                            "status": rep["status"], "newton_iters": rep["newton_iters"],
                            "cg_iters": rep["cg_iters"], "rel_residual": rep["rel"]}
    op.close()
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": round(value, 4), "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_max / args.steps * 1e3, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (each rank: the seeded jittered 64^3 lattice shifted in z, seeded state and direction)",
        "config": {"workload": f"{args.workload} per rank: 3D p-Laplacian p={w.p:g}, {w.n} x {w.n} x {w.n * world} hex "
                               f"lattice split in {world} z-slabs, order {w.order}, {part.n_dofs} DOFs; step = one "
                               "split FP64 J(u) v (local action + one interface exchange)",
                   "n_dofs": part.n_dofs, "parallelism": f"subdomain split P over {world} ranks ({args.backend})",
                   "l2": "FP64 tangent %.0f MB per rank" % (6 * 8 * w.n ** 3 * (w.order + 1) ** 3 / 1e6)},
        "gpu_launches": int(launches), "clocks": clocks,
        "jv_mixed_gdofs": round(part.n_dofs * args.steps / t32 / 1e9, 4),
        "e2e": {"value": round(part.n_dofs * args.steps / t_e2e / 1e9, 4), "unit": "GDOF/s",
                "h2d_bytes_per_step": 8 * op.n_dofs * world, "d2h_bytes_per_step": 8 * op.n_dofs * world},
        "newton": newton,
        "exchange_bytes_per_step": 2 * 8 * pl * 2 * (world - 1),
    }


def small_newton_cases(Operator, I) -> dict:
    """Newton solves of the small configurations whose oracle Newton the CPU baseline also times:
    the 2D 16x16 order-2 problem and the 3D 16^3 order-2 problem, FP64 and mixed."""
    import torch
    out = {}
    for key in ("2d_p3_k2_16x16", "3d_p3_k2_16"):
        wk = I.WORKLOADS[key]
        opk = Operator(wk.dim, wk.n, wk.order, I.lattice_vertices(wk.dim, wk.n, seed=wk.mesh_seed), p=wk.p,
                       eps=wk.eps)
        uk = torch.from_numpy(I.smooth_field(wk.dim, wk.n, wk.order, seed=wk.state_seed)).cuda()
        small = {}
        for name, prec in (("mixed", -32), ("fp64", 64)):
            uu = uk.clone()
            opk.newton_solve(uu, rtol=1e-8, inner_precision=prec)        # warm-up (graph creation)
            uu = uk.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = opk.newton_solve(uu, rtol=1e-8, inner_precision=prec, raise_on_error=False)
            torch.cuda.synchronize()
            small[name] = {"time_s": round(time.perf_counter() - t0, 5), "status": rep["status"],
                           "newton_iters": rep["newton_iters"], "cg_iters": rep["cg_iters"]}
        opk.close()
        out[key] = small
    return out


# ------------------------------------------------------------------------------------------------
# measurement suites beside the headline: the order sweep and the design-sensitivity case
# ------------------------------------------------------------------------------------------------
def _event_time(fn, steps: int, warmup: int) -> float:
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / steps


def _newton_modes(op, u0, max_newton: int) -> dict:
    import torch
    out = {}
    for name, prec in NEWTON_MODES:
        u = u0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = op.newton_solve(u, rtol=1e-8, inner_precision=prec, max_newton=max_newton, raise_on_error=False)
        torch.cuda.synchronize()
        out[name] = {"time_s": round(time.perf_counter() - t0, 4), "status": rep["status"],
                     "newton_iters": rep["newton_iters"], "cg_iters": rep["cg_iters"],
                     "rel_residual": rep["rel"]}
    for name, _ in NEWTON_MODES[:-1]:
        out[f"speedup_{name}_vs_fp64"] = round(out["fp64"]["time_s"] / out[name]["time_s"], 3)
    return out


def run_sweep(args) -> dict:
    """3D p=3, orders 1..6 on meshes of about 8M DOFs (k n ~ 200): FP32 / FP64 J v, FP64 residual
    and the three Newton modes per order."""
    import torch

    from paper_2506_00746_gb300 import Operator
    from paper_2506_00746_gb300 import inputs as I
    torch.cuda.set_device(0)
    peaks = measured_peaks()
    f64 = fp64_peak()
    orders = [int(k) for k in args.orders.split(",")]
    rows = []
    clk = ClockSampler(0).start()
    for k in orders:
        w = I.sweep_workload(k)
        V = I.lattice_vertices(3, w.n, seed=w.mesh_seed)
        op = Operator(3, w.n, k, V, p=w.p, eps=w.eps)
        nl, ne, nq = op.n_dofs, op.n_elements, (k + 1) ** 3
        u0 = torch.from_numpy(I.smooth_field(3, w.n, k, seed=w.state_seed)).cuda()
        v64 = torch.from_numpy(I.uniform_vector(nl, seed=w.dir_seed)).cuda()
        v32 = v64.float()
        y32, y64 = torch.empty_like(v32), torch.empty_like(v64)
        op.linearize(u0)
        t32 = _event_time(lambda: op.jacobian_action(v32, precision=32, out=y32), 30, 3)
        op.prof_enable(True); op.prof_reset()
        for _ in range(10):
            op.jacobian_action(v32, precision=32, out=y32)
        prof = op.prof_read(); op.prof_enable(False)
        kn, kms = prof.get("jv_pa_f32", (1, float("nan")))
        t_main = kms / 1e3 / max(kn, 1)
        t64 = _event_time(lambda: op.jacobian_action(v64, precision=64, out=y64), 5, 2)
        tdf = _event_time(lambda: op.jacobian_action(v64, precision=48, out=y64), 10, 2)
        r = torch.empty_like(u0)
        tres = _event_time(lambda: op.residual(u0, out=r), 3, 1)
        b32 = jv_algorithmic_bytes(nl, ne, nq, nq, 4)
        fl = jv_algorithmic_flops(3, ne, k + 1, k + 1)
        row = {"order": k, "n": w.n, "n_dofs": nl, "n_elements": ne,
               "jv_f32_gdofs": round(nl / t32 / 1e9, 3), "jv_f32_ms": round(t32 * 1e3, 4),
               "jv_f32_main_kernel_ms": round(t_main * 1e3, 4),
               "jv_f32_hbm_frac": round(b32 / t_main / 1e9 / peaks["hbm_gbs"], 4),
               "jv_f64_gdofs": round(nl / t64 / 1e9, 3),
               "jv_f64_fp64_frac": round(fl / t64 / 1e12 / f64["tflops"], 4),
               "jv_double_float_gdofs": round(nl / tdf / 1e9, 3),
               "residual_f64_gdofs": round(nl / tres / 1e9, 3)}
        if not args.no_newton:
            row["newton"] = _newton_modes(op, u0, args.max_newton)
        rows.append(row)
        op.close()
        del u0, v64, v32, y32, y64
        torch.cuda.empty_cache()
    clocks = clk.stop()
    return {"suite": "sweep", "workload": "3D p-Laplacian p=3, orders %s, k n ~ 200 (about 8M DOFs)" % args.orders,
            "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_source": peaks["source"],
            "fp64_peak_tflops": f64["tflops"], "fp64_peak_source": f64["source"],
            "jv_f32_hbm_frac_note": "algorithmic bytes (v, y, 6 tangent words per point, 4 B index per "
                                    "E-vector entry) / main kernel time, fix-up excluded",
            "clocks": clocks, "orders": rows}


def run_design(args) -> dict:
    """Design sensitivity on 48^3 order 2: kappa(rho) = 1e-3 + rho^3 times the p=3 flux; Newton,
    the adjoint gradient of the compliance through the autograd function, and central differences
    on 20 seeded directions."""
    import numpy as np
    import torch

    from paper_2506_00746_gb300 import ComplianceFn, Operator
    from paper_2506_00746_gb300 import inputs as I
    torch.cuda.set_device(0)
    w = I.WORKLOADS["3d_design_k2_48"]
    V = I.lattice_vertices(3, w.n, seed=w.mesh_seed)
    rho0 = I.design_field(3, w.n, seed=3)
    op = Operator(3, w.n, w.order, V, p=w.p, eps=w.eps, rho=rho0)
    u0 = torch.from_numpy(I.smooth_field(3, w.n, w.order, seed=w.state_seed)).cuda()
    kw = {"rtol": 1e-12, "cg_rtol": 1e-8}
    rho = torch.from_numpy(rho0).cuda().requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c = ComplianceFn.apply(rho, op, u0, kw)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    c.backward()
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    g = rho.grad.detach().clone()
    rng = np.random.default_rng(4)
    h = 1e-5
    errs, t_fd = [], 0.0
    for _ in range(args.fd_dirs):
        d = torch.from_numpy(rng.standard_normal(op.n_elements)).cuda()
        t0 = time.perf_counter()
        with torch.no_grad():
            cp = ComplianceFn.apply(rho.detach() + h * d, op, u0, kw).item()
            cm = ComplianceFn.apply(rho.detach() - h * d, op, u0, kw).item()
        t_fd += time.perf_counter() - t0
        fd = (cp - cm) / (2 * h)
        gd = torch.dot(g, d).item()
        errs.append(abs(fd - gd) / abs(gd))
    out = {"suite": "design", "workload": "3d_design_k2_48: 48^3 hex, order 2, p=3, kappa = 1e-3 + rho^3, "
                                          "rho seeded U[0,1] per element, compliance F^T u, FP64",
           "n_dofs": op.n_dofs, "n_elements": op.n_elements, "compliance": c.item(),
           "forward_newton_s": round(t_fwd, 4), "adjoint_backward_s": round(t_bwd, 4),
           "fd_directions": args.fd_dirs, "fd_step": h, "fd_rel_err_max": max(errs),
           "fd_rel_err_median": float(np.median(errs)), "fd_time_s": round(t_fd, 3)}
    # the same Newton solve by the FP64 GPU path and by the mixed-precision one, to 1e-8
    for name, prec in (("fp64", 64), ("mixed", -32)):
        op.set_design(torch.from_numpy(rho0).cuda())
        u = u0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = op.newton_solve(u, rtol=1e-8, inner_precision=prec, raise_on_error=False)
        torch.cuda.synchronize()
        out[f"newton_{name}"] = {"time_s": round(time.perf_counter() - t0, 4), "status": rep["status"],
                                 "newton_iters": rep["newton_iters"], "cg_iters": rep["cg_iters"], "rel": rep["rel"]}
    op.close()
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = design_cpu_baseline(w, V, rho0)
    return out


def design_cpu_baseline(w, V, rho0) -> dict:
    """The oracle's Newton solve of the design case on the host cores (assembled sparse Jacobian,
    Jacobi-preconditioned scipy CG to 1e-4 per step, the GPU's line search), to 1e-8."""
    import oracle as O
    from paper_2506_00746_gb300 import inputs as I
    cores = O.set_threads(os.cpu_count() or 1)
    P = O.Problem(3, w.n, w.order, V, p=w.p, eps=w.eps, rho=rho0)
    its: list = []
    t0 = time.perf_counter()
    _, hist = O.newton(P, I.smooth_field(3, w.n, w.order, seed=w.state_seed), rtol=1e-8, linear="cg", cg_iters=its)
    return {"kind": "oracle", "cores": cores, "newton_time_s": round(time.perf_counter() - t0, 3),
            "newton_iters": len(hist) - 1, "cg_iters": int(sum(its)), "rel_residual": float(hist[-1] / hist[0]),
            "sample": "the whole 48^3 order-2 design problem"}


def run_batched(args) -> dict:
    """64 independent instances (p ~ U[2.5,4], n in [8,40], orders 1-4, seed 5): the batched FP32
    J v (autotuned: persistent launch or one launch per variant) against the same instances'
    single-instance actions one after another, the batched action under each work policy, and the
    lock-step batched Newton (FP32 CG, FP64 outer) against per-instance solves."""
    import torch

    from paper_2506_00746_gb300 import Batch, Operator
    from paper_2506_00746_gb300 import inputs as I
    torch.cuda.set_device(0)
    peaks = measured_peaks()
    ws = I.batched_instances(64, seed=5)
    inst = [{"vertices": I.lattice_vertices(3, w.n, seed=w.mesh_seed), "n": w.n, "order": w.order, "p": w.p}
            for w in ws]
    cache = os.path.join(ROOT, "paper_2506_00746_gb300", "_build", "tune_cache.json")
    t0 = time.perf_counter()
    B = Batch(inst, tune=True, tune_cache=cache)
    t_create = time.perf_counter() - t0
    us = [I.smooth_field(3, w.n, w.order, seed=w.state_seed) for w in ws]
    u0 = B.concat(us)
    B.linearize(u0)
    v = B.concat([I.uniform_vector(n, seed=w.dir_seed) for n, w in zip(B.n_dofs, ws)], torch.float32)
    y = torch.empty_like(v)
    total_dofs = sum(B.n_dofs)
    bytes_alg = sum(jv_algorithmic_bytes(n, w.n ** 3, (w.order + 1) ** 3, (w.order + 1) ** 3, 4)
                    for n, w in zip(B.n_dofs, ws))
    clk = ClockSampler(0).start()
    l0 = B.shape()["launches"]
    t_b = _event_time(lambda: B.jacobian_action(v, out=y), args.steps, args.warmup)
    launches = (B.shape()["launches"] - l0) / (args.steps + args.warmup)
    # the same action captured once in a CUDA graph and replayed
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph):
        B.jacobian_action(v, out=y)
    t_graph = _event_time(graph.replay, args.steps, args.warmup)
    # the same instances one after another through their own single-instance operators
    ops = [Operator(3, d["n"], d["order"], d["vertices"], p=d["p"]) for d in inst]
    vs, ys = [], []
    for i, op in enumerate(ops):
        op.linearize(torch.from_numpy(us[i]).cuda())
        vs.append(B.split(v)[i].clone())
        ys.append(torch.empty_like(vs[-1]))

    def seq():
        for op, vi, yi in zip(ops, vs, ys):
            op.jacobian_action(vi, precision=32, out=yi)
    t_s = _event_time(seq, max(5, args.steps // 4), 3)
    # the batched action under each work policy at the tuned tile edges (0-2: persistent launch at
    # its default grid, 3: one launch per variant)
    tiles = [next((t for t, w in zip(B.tiles, ws) if w.order == k), 0) for k in (1, 2, 3, 4)]
    policy_ms = {}
    for pol in (0, 1, 2, 3):
        Bp = Batch(inst, tune=False, tiles=tiles, policy=pol)
        Bp.linearize(u0)
        policy_ms[pol] = round(_event_time(lambda: Bp.jacobian_action(v, out=y), args.steps, args.warmup) * 1e3, 4)
        Bp.close()
    clocks = clk.stop()
    out = {"suite": "batched", "workload": "64 instances, p ~ U[2.5,4], n in [8,40], orders 1-4 (seed 5), "
                                          "%d DOFs in total" % total_dofs,
           "n_instances": len(ws), "n_dofs_total": total_dofs,
           "orders": {k: sum(w.order == k for w in ws) for k in (1, 2, 3, 4)},
           "tiles_by_order": {k: next((t for t, w in zip(B.tiles, ws) if w.order == k), None) for k in (1, 2, 3, 4)},
           "launch": B.shape(), "create_and_tune_s": round(t_create, 3),
           "batched_jv_ms": round(t_b * 1e3, 4), "batched_jv_gdofs": round(total_dofs / t_b / 1e9, 3),
           "batched_jv_launches_per_step": launches,
           "batched_jv_graph_ms": round(t_graph * 1e3, 4),
           "batched_jv_hbm_frac": round(bytes_alg / t_b / 1e9 / peaks["hbm_gbs"], 4),
           "sequential_jv_ms": round(t_s * 1e3, 4), "sequential_jv_gdofs": round(total_dofs / t_s / 1e9, 3),
           "sequential_jv_launches_per_step": 2 * len(ws),
           "batching_speedup_jv": round(t_s / t_b, 3), "jv_ms_by_policy": policy_ms, "clocks": clocks,
           "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_source": peaks["source"]}
    if not args.no_newton:
        u = u0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps, tot = B.newton_solve(u, rtol=1e-8, raise_on_error=False)
        torch.cuda.synchronize()
        t_bn = time.perf_counter() - t0
        t_sn, it_s, ok_s = 0.0, 0, 0
        for i, op in enumerate(ops):
            ui = torch.from_numpy(us[i]).cuda()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = op.newton_solve(ui, rtol=1e-8, inner_precision=32, raise_on_error=False)
            torch.cuda.synchronize()
            t_sn += time.perf_counter() - t0
            it_s += r["cg_iters"]
            ok_s += r["status"] == "FE_OK"
        out["newton"] = {"batched_s": round(t_bn, 4), "batched_status": tot["status"],
                         "batched_converged": sum(r["status"] == "FE_OK" for r in reps),
                         "batched_max_newton_steps": tot["newton_iters"], "batched_cg_iters": tot["cg_iters"],
                         "batched_max_rel_residual": max(r["rel"] for r in reps),
                         "batched_launches": tot["launches"],
                         "sequential_s": round(t_sn, 4), "sequential_converged": ok_s, "sequential_cg_iters": it_s,
                         "batching_speedup_newton": round(t_sn / t_bn, 3)}
    for op in ops:
        op.close()
    B.close()
    return out


def run_element_ad(args) -> dict:
    """Element tangent matrices K_e (Eq. 3) on hexahedra of orders 1-3, formed by the hand-coded
    tangent (HND), quadrature-point AD (RES) and element-level AD (ELM): time per element."""
    import torch

    from paper_2506_00746_gb300 import Operator
    from paper_2506_00746_gb300 import inputs as I
    torch.cuda.set_device(0)
    rows = []
    for k, n in ((1, 48), (2, 32), (3, 24)):
        V = I.lattice_vertices(3, n, seed=0)
        op = Operator(3, n, k, V, p=3.0)
        u = torch.from_numpy(I.smooth_field(3, n, k, seed=1)).cuda()
        ne, nl = op.n_elements, (k + 1) ** 3
        nc = 8
        # flops of each implementation (multiply-add = 2): point gradients + tangent, then
        # sum_q G^T (T G); ELM: ceil(nl / 8) passes of the dual B and B^T (9 components each)
        f_res = nl * 6 * nl + nl * nl * (18 + 6 * nl)
        f_elm = -(-nl // nc) * (2 * nl * nl * 3 * 2 * (nc + 1))
        row = {"order": k, "n": n, "elements": ne, "nl": nl, "flop_res_per_elem": f_res,
               "flop_elm_per_elem": f_elm}
        for m in ("hnd", "res", "elm"):
            t = _event_time(lambda: op.element_matrices(u, m), 3, 1)
            row[f"{m}_us_per_elem"] = round(t / ne * 1e6, 5)
        row["elm_over_res"] = round(row["elm_us_per_elem"] / row["res_us_per_elem"], 3)
        row["res_over_hnd"] = round(row["res_us_per_elem"] / row["hnd_us_per_elem"], 3)
        rows.append(row)
        op.close()
        torch.cuda.empty_cache()
    return {"suite": "element-ad", "note": "dense element tangents; one CTA loops over elements", "orders": rows}


def run_fp64_peak(args) -> dict:
    """The FP64 fused multiply-add rate of this GPU (fe_measure_fp64_peak: independent FMA chains on
    every SM, CUDA events), with the SM clocks sampled while it runs."""
    import torch

    from paper_2506_00746_gb300 import abi
    torch.cuda.set_device(0)
    clk = ClockSampler(0).start()
    runs = [abi.fe_measure_fp64_peak(args.reps) for _ in range(5)]
    clocks = clk.stop()
    best = max(b for b, _ in runs)
    out = {"suite": "fp64-peak", "gpu": torch.cuda.get_device_name(0), "tflops_best": round(best, 4),
            "tflops_median_per_run": [round(m, 4) for _, m in runs], "reps_per_run": args.reps,
            "sm_count": torch.cuda.get_device_properties(0).multi_processor_count, "clocks": clocks,
            "fma_per_clk_per_sm": (round(best * 1e12 / 2 / torch.cuda.get_device_properties(0).multi_processor_count
                                         / (clocks["sm_mhz"] * 1e6), 3) if clocks.get("sm_mhz") else None),
            "method": "16 independent FP64 FMA chains per thread, 256-thread CTAs, every SM filled to its "
                      "occupancy, 4096 iterations per launch; 2 untimed launches, then `reps` timed ones",
           "command": "python bench.py --suite fp64-peak --reps %d" % args.reps}
    if args.save:
        os.makedirs(os.path.dirname(os.path.abspath(args.save)), exist_ok=True)
        with open(args.save, "w") as f:
            json.dump(out, f, indent=1)
    return out


def run_jv_small(args) -> dict:
    """A few Jacobian actions of one 3D p=3 instance (the small cases the ncu captures use): n
    elements per direction, order, precision 64 / 32 / -32, `reps` actions after linearising at
    the seeded smooth state."""
    import torch

    from paper_2506_00746_gb300 import Operator
    from paper_2506_00746_gb300 import inputs as I
    torch.cuda.set_device(0)
    V = I.lattice_vertices(3, args.n, seed=0)
    op = Operator(3, args.n, args.order, V, p=3.0)
    u = torch.from_numpy(I.smooth_field(3, args.n, args.order, seed=1)).cuda()
    op.linearize(u)
    v = torch.from_numpy(I.uniform_vector(op.n_dofs, seed=2)).cuda()
    if args.precision == 32:
        v = v.float()
    for _ in range(args.reps):
        y = op.jacobian_action(v, precision=args.precision)
    torch.cuda.synchronize()
    out = {"suite": "jv", "n": args.n, "order": args.order, "precision": args.precision, "reps": args.reps,
           "n_dofs": op.n_dofs, "norm": float(y.double().norm())}
    op.close()
    return out


def run_residual_small(args) -> dict:
    """`reps` FP64 residual evaluations R(u) of one 3D p=3 instance at the seeded smooth state (the
    small case of the residual-kernel captures)."""
    import torch

    from paper_2506_00746_gb300 import Operator
    from paper_2506_00746_gb300 import inputs as I
    torch.cuda.set_device(0)
    V = I.lattice_vertices(3, args.n, seed=0)
    op = Operator(3, args.n, args.order, V, p=3.0)
    u = torch.from_numpy(I.smooth_field(3, args.n, args.order, seed=1)).cuda()
    for _ in range(args.reps):
        r = op.residual(u)
    torch.cuda.synchronize()
    out = {"suite": "residual", "n": args.n, "order": args.order, "reps": args.reps, "n_dofs": op.n_dofs,
           "norm": float(r.norm())}
    op.close()
    return out


def run_cg_small(args) -> dict:
    """`reps` Jacobi-preconditioned CG iterations (fe_cg_solve, precision as given) on one 3D p=3
    instance linearised at the seeded smooth state, with the load vector as right-hand side and an
    unreachable tolerance (the small case of the CG-kernel captures)."""
    import torch

    from paper_2506_00746_gb300 import Operator
    from paper_2506_00746_gb300 import inputs as I
    from paper_2506_00746_gb300.abi import FeodError
    torch.cuda.set_device(0)
    V = I.lattice_vertices(3, args.n, seed=0)
    op = Operator(3, args.n, args.order, V, p=3.0)
    u = torch.from_numpy(I.smooth_field(3, args.n, args.order, seed=1)).cuda()
    op.linearize(u)
    F = op.load_vector()
    try:
        op.cg_solve(F, rtol=1e-30, max_iter=args.reps, precision=args.precision)
        status = "FE_OK"
    except FeodError as e:
        status = str(e).split("(")[1].split(")")[0] if "(" in str(e) else str(e)
    torch.cuda.synchronize()
    out = {"suite": "cg", "n": args.n, "order": args.order, "precision": args.precision, "iterations": args.reps,
           "n_dofs": op.n_dofs, "status": status}
    op.close()
    return out


def run_batch_subset(args) -> dict:
    """A few batched Jacobian actions on the first `instances` of the 64-instance set (no tuning:
    largest tile edges, largest instances first)."""
    import torch

    from paper_2506_00746_gb300 import Batch
    from paper_2506_00746_gb300 import inputs as I
    torch.cuda.set_device(0)
    ws = I.batched_instances(64, seed=5)[:args.instances]
    inst = [{"vertices": I.lattice_vertices(3, w.n, seed=w.mesh_seed), "n": w.n, "order": w.order, "p": w.p}
            for w in ws]
    B = Batch(inst, tune=False, policy=2)
    B.linearize(B.concat([I.smooth_field(3, w.n, w.order, seed=w.state_seed) for w in ws]))
    v = B.concat([I.uniform_vector(n, seed=w.dir_seed) for n, w in zip(B.n_dofs, ws)], torch.float32)
    for _ in range(args.reps):
        y = B.jacobian_action(v)
    torch.cuda.synchronize()
    out = {"suite": "batch-subset", "instances": args.instances, "n_dofs": sum(B.n_dofs), "launch": B.shape(),
           "norm": float(y.double().norm())}
    B.close()
    return out


# ------------------------------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline / reference arm)
# ------------------------------------------------------------------------------------------------
def cpu_baseline(workload: str, budget_s: float = 12.0, gpu: dict | None = None) -> dict:
    """The oracle on the host cores: its FP64 J v and R (element by element, OpenMP over element
    colours) on the workload -- the whole vector when that fits the budget, else a bounded sample
    of the elements, scaled to GDOF/s of a whole action -- and the Newton solves of the small
    configurations.  With the GPU's results of the same inputs (`gpu`), the relative 2-norm
    error of each against the oracle's whole-vector result, and the oracle's residual of the
    GPU's mixed-precision Newton solution."""
    import numpy as np

    import oracle as O
    from paper_2506_00746_gb300 import inputs as I
    w = I.WORKLOADS[workload]
    V = I.lattice_vertices(w.dim, w.n, seed=w.mesh_seed)
    P = O.Problem(w.dim, w.n, w.order, V, p=w.p, eps=w.eps)
    u = I.smooth_field(w.dim, w.n, w.order, seed=w.state_seed)
    v = I.uniform_vector(P.n_dofs, seed=w.dir_seed)
    cores = O.set_threads(os.cpu_count() or 1)

    def sample(fn, share):
        """(elements timed, seconds): a probe on 1/512 of the elements, then as many as the
        budget share allows (all of them when they fit)."""
        m = max(1, P.n_elems // 512)
        t0 = time.perf_counter()
        fn(m)
        dt = time.perf_counter() - t0
        m = int(min(P.n_elems, max(m, m * share * budget_s / max(dt, 1e-6))))
        t0 = time.perf_counter()
        fn(m)
        return m, time.perf_counter() - t0

    m, dt = sample(lambda mm: O.jv_partial(P, u, v, 0, mm), 0.4)
    value = P.n_dofs * (m / P.n_elems) / dt / 1e9
    mr, dtr = sample(lambda mm: O.residual_partial(P, u, 0, mm), 0.2)
    out = {"value": round(value, 6), "unit": "GDOF/s", "cores": cores, "kind": "oracle",
           "sample": f"element-by-element FP64 J(u) v over the first {m} of {P.n_elems} elements "
                     f"({dt:.1f} s), scaled by the element fraction",
           "residual_gdofs": round(P.n_dofs * (mr / P.n_elems) / dtr / 1e9, 6),
           "residual_sample": f"FP64 R(u) over the first {mr} of {P.n_elems} elements ({dtr:.1f} s), scaled likewise"}
    if gpu is not None:
        # the oracle's whole-vector results (Dirichlet convention included) against the GPU's on
        # the same inputs
        y_ref = O.jv(P, u, v)
        r_ref = O.residual(P, u)
        v32 = v.astype(np.float32).astype(np.float64)
        y_ref32 = O.jv(P, u, v32)
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        err = {}
        if gpu.get("r") is not None:
            err["residual_f64"] = rel(gpu["r"], r_ref)
        if gpu.get("jv_f64") is not None:
            err["jv_f64"] = rel(gpu["jv_f64"], y_ref)
        if gpu.get("jv_double_float") is not None:
            err["jv_double_float"] = rel(gpu["jv_double_float"], y_ref)
        if gpu.get("jv_f32") is not None:
            err["jv_f32"] = rel(gpu["jv_f32"], y_ref32)
        if gpu.get("newton_mixed_u") is not None:
            err["newton_mixed_oracle_rel_residual"] = float(
                np.linalg.norm(O.residual(P, gpu["newton_mixed_u"])) / np.linalg.norm(r_ref))
        out["err_vs_oracle"] = err
        out["err_note"] = ("relative 2-norm over the whole vector; FP32 J v against the oracle's J v of the "
                           "FP32-rounded direction; tolerances 1e-12 (FP64, double-float) and 1e-5 (FP32)")
    # Newton solves of the small configurations: 2D 16x16 order 2 (sparse direct inner solves)
    # and 3D 16^3 order 2 (Jacobi-preconditioned CG inner solves to 1e-4, as the GPU's)
    newton = {}
    for key, linear in (("2d_p3_k2_16x16", "direct"), ("3d_p3_k2_16", "cg")):
        wk = I.WORKLOADS[key]
        Pk = O.Problem(wk.dim, wk.n, wk.order, I.lattice_vertices(wk.dim, wk.n, seed=wk.mesh_seed), p=wk.p,
                       eps=wk.eps)
        uk = I.smooth_field(wk.dim, wk.n, wk.order, seed=wk.state_seed)
        its: list = []
        t0 = time.perf_counter()
        _, hist = O.newton(Pk, uk, rtol=1e-8, linear=linear, cg_iters=its)
        newton[key] = {"time_s": round(time.perf_counter() - t0, 4), "linear_solver": linear,
                       "newton_iters": len(hist) - 1, "cg_iters": int(sum(its)) if its else None,
                       "rel_residual": float(hist[-1] / hist[0])}
    out["newton"] = newton
    out["newton_note"] = ("the 64^3 order-3 oracle Newton is impractical on the host cores; the 48^3 design "
                          "case's oracle solve is timed by the design suite")
    return out


def run_reference(args) -> dict | None:
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    import numpy as np

    import oracle as O
    from paper_2506_00746_gb300 import inputs as I
    w = I.WORKLOADS[args.workload]
    V = I.lattice_vertices(w.dim, w.n, seed=w.mesh_seed)
    P = O.Problem(w.dim, w.n, w.order, V, p=w.p, eps=w.eps)
    u = I.smooth_field(w.dim, w.n, w.order, seed=w.state_seed)
    v = I.uniform_vector(P.n_dofs, seed=w.dir_seed)
    cores = O.set_threads(os.cpu_count() or 1)
    y = np.zeros(P.n_dofs)
    # each step is the oracle J v over a bounded element sample, sized so that the whole run
    # (warm-up and timed steps) takes about two minutes (at most 1.5 s per step)
    per_step = min(1.5, 120.0 / max(args.steps + args.warmup, 1))
    m = max(1, P.n_elems // 1024)
    t0 = time.perf_counter()
    O.jv_partial(P, u, v, 0, m, y)
    dt = time.perf_counter() - t0
    m = int(min(P.n_elems, max(m, m * per_step / max(dt, 1e-6))))
    for _ in range(args.warmup):
        O.jv_partial(P, u, v, 0, m, y)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.jv_partial(P, u, v, 0, m, y)
    dt = time.perf_counter() - t0
    value = P.n_dofs * (m / P.n_elems) * args.steps / dt / 1e9
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "GDOF/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: same workload as the GPU arm; each step is the oracle "
                                   f"J(u) v over {m} of {P.n_elems} elements, scaled by the element fraction"},
            "cpu_baseline": {"value": round(value, 6), "unit": "GDOF/s", "cores": cores, "kind": "oracle",
                             "sample": f"first {m} of {P.n_elems} elements per step"},
            "e2e": {"value": round(value, 6), "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-newton", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--max-newton", type=int, default=50)
    ap.add_argument("--suite", choices=["headline", "sweep", "design", "batched", "element-ad", "jv", "residual",
                                        "batch-subset",
                                        "fp64-peak", "cg"],
                    default="headline",
                    help="headline (the benchmark line), sweep (orders 1-6), design (adjoint case), batched "
                         "(64 instances in one persistent launch); jv, residual and batch-subset run the small cases "
                         "of the ncu captures")
    ap.add_argument("--n", type=int, default=48)
    ap.add_argument("--order", type=int, default=3)
    ap.add_argument("--precision", type=int, default=32)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--instances", type=int, default=24)
    ap.add_argument("--orders", default="1,2,3,4,5,6")
    ap.add_argument("--fd-dirs", type=int, default=20)
    ap.add_argument("--backend", choices=["nccl", "gloo"], default="nccl",
                    help="N > 1: interface exchange and sums over ranks through NCCL (device buffers) or gloo "
                         "(host copies; ranks may then share a GPU)")
    ap.add_argument("--save", default=None,
                    help="fp64-peak: also write the result to this JSON file (profiles/fp64_peak.json is the "
                         "committed copy the FP64 rooflines read)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.suite != "headline" and args.impl == "gpu":
        out = {"sweep": run_sweep, "design": run_design, "batched": run_batched, "element-ad": run_element_ad,
               "jv": run_jv_small, "residual": run_residual_small, "fp64-peak": run_fp64_peak, "cg": run_cg_small,
               "batch-subset": run_batch_subset}[args.suite](args)
    elif args.impl == "reference":
        out = run_reference(args)
    else:
        out = run_split(args) if dist_env()[0] > 1 else run_gpu(args)
    if out is not None:
        print(json.dumps(out), flush=True)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
