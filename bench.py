"""Benchmark of the matrix-free p-Laplacian Jacobian action and Newton-CG solve on one GB300.

Workload: 3D p-Laplacian p=3 on a 64^3 hex lattice with seeded jitter, order 3 (7,189,057 DOFs),
4^3 Gauss points per element, linearised at the seeded smooth state.  One timed step is one
partially assembled Jacobian action y = J(u) v in FP32 (the operator the mixed-precision CG
applies); the FP64 action, the FP64 residual and the full Newton-CG solves (FP64 and mixed
precision, to 1e-8 relative residual) are measured in the same run and reported beside it.

Prints one JSON line.  ``--impl reference`` times the oracle (plain FP64 C on the host cores) on
a bounded sample of the same workload instead.  Under torchrun every rank runs an independent
replica on its own GPU (the single-GPU problem does not exchange data); timing is the max over
ranks and the value sums the work of all ranks.
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
    for f in ("element_kernels.cuh", "jv_tile.cuh", "tma.cuh"):
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

    # ---- headline: FP32 Jacobian action, device-resident inputs ----
    jv32 = lambda: op.jacobian_action(v32, precision=32, out=y32)
    clk = ClockSampler(local).start()
    t_dev, launches = timed(jv32, args.steps, args.warmup)
    clocks = clk.stop()
    value, t_max = aggregate(nl * args.steps / 1e9, t_dev, world, dev)

    # ---- per-kernel durations over the same kind of timed region (library CUDA events) ----
    op.prof_enable(True)
    op.prof_reset()
    for _ in range(args.steps):
        jv32()
    prof = op.prof_read()
    op.prof_enable(False)
    main_n, main_ms = prof.get("jv_pa_f32", (1, float("nan")))
    fix_n, fix_ms = prof.get("fixup", (0, 0.0))
    t_main = main_ms / 1e3 / max(main_n, 1)
    t_fix = fix_ms / 1e3 / max(fix_n, 1) if fix_n else 0.0

    # ---- other operators of the path ----
    jv64 = lambda: op.jacobian_action(v64, precision=64, out=y64)
    t64, _ = timed(jv64, max(3, args.steps // 20), 2)
    n64 = max(3, args.steps // 20)
    # double-float operator (FP32 word pairs): the first call splits the FP64 tangent, untimed
    jvdf = lambda: op.jacobian_action(v64, precision=48, out=y64)
    jvdf()
    tdf, _ = timed(jvdf, max(3, args.steps // 10), 2)
    ndf = max(3, args.steps // 10)
    jvcg = lambda: op.jacobian_action(v64, precision=-32, out=y64)
    tcg, _ = timed(jvcg, args.steps, 3)
    r = torch.empty_like(u0)
    res = lambda: op.residual(u0, out=r)
    nres = max(3, args.steps // 20)
    tres, _ = timed(res, nres, 2)

    # ---- end to end through the C ABI with host buffers (copies inside the timed region) ----
    vh = v32.cpu().pin_memory()
    yh = torch.empty_like(vh).pin_memory()
    for _ in range(3):
        op.jacobian_action_host(vh, yh, precision=32)
    torch.cuda.synchronize()
    barrier(dev)
    ne2e = max(5, args.steps // 4)
    t0 = time.perf_counter()
    for _ in range(ne2e):
        op.jacobian_action_host(vh, yh, precision=32)
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
        # the small 2D configuration (16x16 quads, order 2), FP64 and mixed, beside the oracle's
        w2 = I.WORKLOADS["2d_p3_k2_16x16"]
        op2 = Operator(2, w2.n, w2.order, I.lattice_vertices(2, w2.n, seed=w2.mesh_seed), p=w2.p, eps=w2.eps)
        u2 = torch.from_numpy(I.smooth_field(2, w2.n, w2.order, seed=w2.state_seed)).cuda()
        small = {}
        for name, prec in (("mixed", -32), ("fp64", 64)):
            uu = u2.clone()
            op2.newton_solve(uu, rtol=1e-8, inner_precision=prec)        # warm-up (graph creation)
            uu = u2.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = op2.newton_solve(uu, rtol=1e-8, inner_precision=prec, raise_on_error=False)
            torch.cuda.synchronize()
            small[name] = {"time_s": round(time.perf_counter() - t0, 5), "status": rep["status"],
                           "newton_iters": rep["newton_iters"], "cg_iters": rep["cg_iters"]}
        op2.close()
        newton["2d_16x16_order2"] = small

    if rank != 0:
        op.close()
        return None

    peaks = measured_peaks()
    bytes_alg = jv_algorithmic_bytes(nl, ne, nq, nq, 4)
    achieved = bytes_alg / t_main / 1e9
    kname = "k_jv_tile2<4,2,float>"
    traffic, traffic_src = profiled_traffic(kname)
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
        "dtype": "f32",
        "data": "synthetic (seeded jittered lattice, seeded smooth state, seeded U[-1,1] direction)",
        "config": {"workload": f"{args.workload}: 3D p-Laplacian p=3, 64^3 hex, order 3, 4^3 Gauss points, "
                               f"{nl} DOFs; step = one FP32 partially assembled J(u) v",
                   "n_dofs": nl, "n_elements": ne, "order": w.order, "p": w.p,
                   "l2": "inputs larger than L2 (FP32 tangent %.0f MB + index/vectors)" % (6 * 4 * ne * nq / 1e6),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   # the library's default tile edge of 3D order k (elements per CTA = tile^3)
                   "tile": {1: 4, 2: 3, 3: 2, 4: 2, 5: 2, 6: 1}[w.order]},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                     "kernel": kname, "peak_source": peaks["source"],
                     "algorithmic_bytes_per_launch": bytes_alg,
                     "kernel_ms": round(t_main * 1e3, 5), "fixup_ms": round(t_fix * 1e3, 5),
                     "traffic_summary": traffic_src},
        "e2e": {"value": round(e2e_value, 4), "unit": "GDOF/s", "h2d_bytes_per_step": 4 * nl,
                "d2h_bytes_per_step": 4 * nl},
        "jv_f64_gdofs": round(nl * n64 / t64 / 1e9, 4),
        "jv_double_float_gdofs": round(nl * ndf / tdf / 1e9, 4),
        "jv_cg_mixed_gdofs": round(nl * args.steps / tcg / 1e9, 4),
        "residual_f64_gdofs": round(nl * nres / tres / 1e9, 4),
        "newton": newton,
        "kernel_ms": {k: round(ms / max(n, 1), 5) for k, (n, ms) in prof.items()},
    }
    op.close()
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_seconds)
    return out


# ------------------------------------------------------------------------------------------------
# measurement suites beside the headline: the order sweep and the design-sensitivity case
# ------------------------------------------------------------------------------------------------
FP64_PEAK_TFLOPS = 1.25   # nominal dense FP64 rate of the GB300 (no measured FP64 peak is recorded)


def jv_algorithmic_flops(dim: int, n_e: int, d1: int, q1: int) -> float:
    """Flops of one partially assembled J v: per element, interpolation plus collocated gradient
    in both directions (4 d D1^(d+1) multiply-adds) and the symmetric d x d matvec per point."""
    return 2.0 * n_e * (4 * dim * d1 ** (dim + 1) + dim * dim * q1 ** dim)


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
               "jv_f64_fp64_frac": round(fl / t64 / 1e12 / FP64_PEAK_TFLOPS, 4),
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
            "fp64_peak_tflops": FP64_PEAK_TFLOPS, "fp64_peak_source": "nominal",
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
    op.close()
    return out


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
def cpu_baseline(workload: str, budget_s: float = 12.0) -> dict:
    """Oracle J v (element by element, FP64, OpenMP over element colours) on a bounded sample of
    the elements of the workload, scaled to GDOF/s of a whole action."""
    import numpy as np

    import oracle as O
    from paper_2506_00746_gb300 import inputs as I
    w = I.WORKLOADS[workload]
    V = I.lattice_vertices(w.dim, w.n, seed=w.mesh_seed)
    P = O.Problem(w.dim, w.n, w.order, V, p=w.p, eps=w.eps)
    u = I.smooth_field(w.dim, w.n, w.order, seed=w.state_seed)
    v = I.uniform_vector(P.n_dofs, seed=w.dir_seed)
    cores = O.set_threads(os.cpu_count() or 1)
    y = np.zeros(P.n_dofs)
    m = max(1, P.n_elems // 512)
    t0 = time.perf_counter()
    O.jv_partial(P, u, v, 0, m, y)
    dt = time.perf_counter() - t0
    m = int(min(P.n_elems, max(m, m * budget_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    O.jv_partial(P, u, v, 0, m, y)
    dt = time.perf_counter() - t0
    value = P.n_dofs * (m / P.n_elems) / dt / 1e9
    # the residual on a sample timed the same way (half the budget)
    r = np.zeros(P.n_dofs)
    mr = max(1, P.n_elems // 512)
    t0 = time.perf_counter()
    O.residual_partial(P, u, 0, mr, r)
    dtr = time.perf_counter() - t0
    mr = int(min(P.n_elems, max(mr, mr * 0.5 * budget_s / max(dtr, 1e-6))))
    t0 = time.perf_counter()
    O.residual_partial(P, u, 0, mr, r)
    dtr = time.perf_counter() - t0
    # the small 2D configuration's Newton solve (sparse direct inner solves), whole
    w2 = I.WORKLOADS["2d_p3_k2_16x16"]
    P2 = O.Problem(w2.dim, w2.n, w2.order, I.lattice_vertices(w2.dim, w2.n, seed=w2.mesh_seed), p=w2.p, eps=w2.eps)
    u2 = I.smooth_field(w2.dim, w2.n, w2.order, seed=w2.state_seed)
    t0 = time.perf_counter()
    O.newton(P2, u2, rtol=1e-8)
    dtn = time.perf_counter() - t0
    return {"value": round(value, 6), "unit": "GDOF/s", "cores": cores, "kind": "oracle",
            "sample": f"element-by-element FP64 J(u) v over the first {m} of {P.n_elems} elements "
                      f"({dt:.1f} s), scaled by the element fraction",
            "residual_gdofs": round(P.n_dofs * (mr / P.n_elems) / dtr / 1e9, 6),
            "residual_sample": f"FP64 R(u) over the first {mr} elements ({dtr:.1f} s), scaled likewise",
            "newton_2d_16x16_s": round(dtn, 4)}


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
    ap.add_argument("--suite", choices=["headline", "sweep", "design", "batched", "element-ad", "jv", "batch-subset"],
                    default="headline",
                    help="headline (the benchmark line), sweep (orders 1-6), design (adjoint case), batched "
                         "(64 instances in one persistent launch); jv and batch-subset run the small cases "
                         "of the ncu captures")
    ap.add_argument("--n", type=int, default=48)
    ap.add_argument("--order", type=int, default=3)
    ap.add_argument("--precision", type=int, default=32)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--instances", type=int, default=24)
    ap.add_argument("--orders", default="1,2,3,4,5,6")
    ap.add_argument("--fd-dirs", type=int, default=20)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.suite != "headline" and args.impl == "gpu":
        out = {"sweep": run_sweep, "design": run_design, "batched": run_batched, "element-ad": run_element_ad,
               "jv": run_jv_small,
               "batch-subset": run_batch_subset}[args.suite](args)
    else:
        out = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if out is not None:
        print(json.dumps(out), flush=True)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
