#!/usr/bin/env python3
"""Benchmark of the SpMV format sweep (and the solves built on it) on GB300.

One step = one SpMV of every (matrix, value type, format) of the sweep:
  * 27-point 3D stencil on 100^3 (n = 1,000,000, nnz = 26,463,592);
  * power-law random matrix, n = 2,000,000, row lengths Pareto(tail 1.5) with
    mean 16 and cap 20,000, uniform columns, N(0,1) values (nnz = 32.0M);
  x {FP64, FP32} x {CSR (kernel chosen from row statistics), ELL, COO, HYB},
int32 indices.  ELL of
the power-law matrix does not fit (20,000 x 2M padded slots) and is reported
as rejected, as the library does.

value = algorithmic bytes of all SpMVs of the job / device time (GB/s), the
byte model being CSR (V+4) nnz + 4 (n+1) + 2 V n, ELL (V+4) k n + 2 V n,
COO (V+8) nnz + 2 V n, HYB (V+4) k n + (V+8) nnz_coo + 2 V n (x read once,
y written once).  Every matrix is larger than the 129 MB L2 and the step
cycles through 14 matrices, so nothing stays cached between timed steps.

--impl reference times the CPU oracle (its plain index-order FP64 CSR SpMV,
OpenMP over rows on every host core) on the same workload and metric.  Multi-GPU (torchrun): independent
replicas, one per GPU, no collective on the data path (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMV GB/s and CG solve time vs HBM roofline; batched solves/s; p50/p99 latency"
WORKLOAD = ("spmv_format_sweep: 27-point 3D stencil 100^3 (n=1,000,000, nnz=26,463,592) and power-law "
            "n=2,000,000 (Pareto tail 1.5, mean 16, max 20,000 nnz/row, nnz=32,000,000); "
            "CSR (kernel chosen from row statistics: row-block for the stencil, nnz-split for the power-law)/ELL/COO/HYB x FP64/FP32 values, int32 indices")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def algorithmic_bytes(fmt: str, V: int, n: int, ncols: int, nnz: int, ell_w: int = 0, coo_nnz: int = 0) -> int:
    """Bytes an SpMV must move at least once: stored entries, row pointers
    (CSR), x read once and y written once."""
    vec = V * ncols + V * n
    if fmt == "csr":
        return (V + 4) * nnz + 4 * (n + 1) + vec
    if fmt == "ell":
        return (V + 4) * ell_w * n + vec
    if fmt == "coo":
        return (V + 8) * nnz + vec
    if fmt == "hyb":
        return (V + 4) * ell_w * n + (V + 8) * coo_nnz + vec
    raise ValueError(fmt)


def paper_intensity(fmt: str, V: int) -> float:
    """The paper's simplified arithmetic intensity (Section 6.3): 2 flops per
    nonzero over 1 value + 1 index (CSR) or 1 value + 2 indices (COO)."""
    return 2.0 / ((V + 4) if fmt == "csr" else (V + 8))


def _src_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = ["paper_2103_10116_gb300/csrc/spmv.cu", "paper_2103_10116_gb300/csrc/dev_common.cuh",
                  "paper_2103_10116_gb300/csrc/kstate.cuh"]


def _traffic(key: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
    the committed ncu capture table profiles/dram_traffic.json, if the kernel
    sources still hash to the ones the capture was taken with; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            tab = json.load(f)
    except (OSError, ValueError):
        return None
    if tab.get("kernel_source_hash") != _src_hash(KERNEL_SOURCES):
        return None
    ent = tab.get("entries", {}).get(key)
    return int(ent["read"]) + int(ent["write"]) if ent else None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"spx_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() in ("active", "1"):
                        reasons.add(nm)
        except Exception:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def build_workload(only: str = ""):
    """The two sweep matrices (only those an --only filter can match)."""
    from paper_2103_10116_gb300 import synth
    gens = {"stencil27_100": lambda: synth.stencil3d_27pt(100), "powerlaw_2m": lambda: synth.powerlaw(2_000_000)}
    return {k: f() for k, f in gens.items() if not only or k in only or "/" not in only and only in k}


def _floor_key(entry_name: str) -> str:
    """'powerlaw_2m/csr/f64' -> 'powerlaw_2m/f64' (the gather floor depends on pattern and value type)."""
    parts = entry_name.split("/")
    return f"{parts[0]}/{parts[-1]}"


def max_over_ranks(elapsed_ms: float, dist=None, device=None) -> float:
    """The job's time is the slowest replica's: all-reduce MAX, then a barrier.
    Replicas share no data; this is the only collective and it sits outside the
    timed region."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(elapsed_ms)
    import torch
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_value(bytes_per_step: int, steps: int, world: int, elapsed_ms: float) -> float:
    """Whole-job GB/s: every replica moves bytes_per_step per step."""
    return bytes_per_step * steps * world / (elapsed_ms * 1e-3) / 1e9


def run_gpu(args):
    import torch
    from paper_2103_10116_gb300 import spx

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    spx.load()
    stream = torch.cuda.Stream(device=dev)
    ctx = spx.spx_ctx_create(local, stream)

    mats = build_workload(args.only)
    entries = []  # (name, fmt, V, handle, x, y, bytes, launches, x_host, y_host)
    rejected = []
    for mname, (rp, col, val) in mats.items():
        n = rp.shape[0] - 1
        nnz = col.shape[0]
        rp_d = torch.from_numpy(rp).to(dev)
        col_d = torch.from_numpy(col).to(dev)
        val_d = torch.from_numpy(val).to(dev)
        xs = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, n)).to(dev)
        for tdt, V in ((torch.float64, 8), (torch.float32, 4)):
            vv = val_d.to(tdt)
            x = xs.to(tdt)
            for fmt in ("csr", "ell", "coo", "hyb"):
                if args.only and args.only not in f"{mname}/{fmt}/{'f64' if V == 8 else 'f32'}":
                    continue
                try:
                    with torch.cuda.stream(stream):
                        A = spx.spx_matrix_create(ctx, fmt, rp_d, col_d, vv)
                except spx.SpxError as e:
                    if e.status == spx.SPX_ERR_TOO_LARGE:
                        rejected.append(f"{mname}/{fmt}/{'f64' if V == 8 else 'f32'}")
                        continue
                    raise
                info = spx.spx_matrix_get_info(A)
                b = algorithmic_bytes(fmt, V, n, n, nnz, info["ell_width"], info["coo_nnz"])
                launches = 2 if (fmt == "hyb" and info["coo_nnz"] > 0 and info["ell_width"] > 0) else 1
                y = torch.empty(n, dtype=tdt, device=dev)
                xh = x.cpu().pin_memory()
                yh = torch.empty(n, dtype=tdt).pin_memory()
                entries.append(dict(name=f"{mname}/{fmt}/{'f64' if V == 8 else 'f32'}", fmt=fmt, V=V, A=A, x=x, y=y,
                                    bytes=b, launches=launches, xh=xh, yh=yh, n=n, nnz=nnz))
        del rp_d, col_d, val_d
    torch.cuda.synchronize()

    def step(evs=None):
        for i, e in enumerate(entries):
            if evs is not None:
                evs[i][0].record(stream)
            spx.spx_spmv(ctx, e["A"], e["x"], e["y"])
            if evs is not None:
                evs[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in entries]
           for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0.record(stream)
    for s in range(args.steps):
        step(evs[s])
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed_ms = max_over_ranks(t0.elapsed_time(t1), dist, dev)
    per_entry_ms = [statistics.mean(evs[s][i][0].elapsed_time(evs[s][i][1]) for s in range(args.steps))
                    for i in range(len(entries))]
    bytes_step = sum(e["bytes"] for e in entries)
    value = job_value(bytes_step, args.steps, world, elapsed_ms)

    # end to end through the public API with host buffers (copies inside the timed region)
    for e in entries:
        spx.spx_spmv_host(ctx, e["A"], e["xh"], e["yh"])
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        t = time.perf_counter()
        for e in entries:
            spx.spx_spmv_host(ctx, e["A"], e["xh"], e["yh"])
        e2e_ms.append((time.perf_counter() - t) * 1e3)
    e2e_step_ms = statistics.median(e2e_ms)
    h2d = sum(e["n"] * e["V"] for e in entries)
    d2h = sum(e["n"] * e["V"] for e in entries)

    peak, peak_src = _peaks()
    secondary = {}
    solves = None
    if not args.no_solve:
        secondary["small_case"] = small_case_secondary(spx, ctx, stream, dev)
        solves = solve_secondary(spx, ctx, stream, dev, peak)
    if not args.no_solve:
        secondary["fixed_iterations"] = fixed_iter_secondary(spx, ctx, stream, dev)
        secondary["vendor_csr_context"] = vendor_secondary(mats, dev)
        secondary["jacobi"] = jacobi_secondary(spx, ctx, stream, dev)
    if args.batched:
        secondary["batched"] = batched_secondary(spx, ctx, stream, dev)
    floors = gather_floor(spx, ctx, stream, mats, dev)
    if args.serve_seconds > 0:
        # random gathers of x per second on the power-law pattern (32 M uniform columns), FP32
        pl = mats.get("powerlaw_2m")
        rate = pl[1].shape[0] / (floors["powerlaw_2m/f32"] * 1e-6) if pl is not None else None
        secondary["serving"] = serving_secondary(spx, ctx, dev, seconds=args.serve_seconds, gather_rate=rate)
    # the roofline is reported for one kernel: the single-launch sweep entry
    # (HYB launches two) with the largest device time per step
    single = [i for i, e in enumerate(entries) if e["launches"] == 1] or list(range(len(entries)))
    dom = max(single, key=lambda i: per_entry_ms[i])
    de = entries[dom]
    achieved = de["bytes"] / (per_entry_ms[dom] * 1e-3) / 1e9
    traffic = _traffic(de["name"])
    result = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(elapsed_ms / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64,f32",
        "data": "synthetic",
        "config": {
            "workload": WORKLOAD,
            "spmvs_per_step": len(entries),
            "rejected": rejected,
            "l2": "inputs larger than L2: every matrix exceeds the 129 MB L2 and a step cycles through all of them",
            "roofline_kernel": "the single-kernel sweep entry with the largest device time per step",
            "parallelism": "replicas" if world > 1 else "single GPU",
            "per_spmv": {e["name"]: {"us": round(per_entry_ms[i] * 1e3, 1),
                                     "GB_s": round(e["bytes"] / (per_entry_ms[i] * 1e-3) / 1e9, 1),
                                     "frac_of_peak": round(e["bytes"] / (per_entry_ms[i] * 1e-3) / 1e9 / peak, 3)}
                         for i, e in enumerate(entries)},
            "gather_floor_us": floors,
        },
        "roofline": {"bound": "hbm", "kernel": de["name"], "achieved": round(achieved, 1), "peak": peak,
                     "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured" else "fallback",
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                     "algorithmic_bytes_per_launch": de["bytes"],
                     "gather_floor_us": floors.get(_floor_key(de["name"])),
                     "time_over_gather_floor": round(per_entry_ms[dom] * 1e3 / floors[_floor_key(de["name"])], 2)
                     if floors.get(_floor_key(de["name"])) else None},
        "e2e": {"value": round(bytes_step / (e2e_step_ms * 1e-3) / 1e9, 1), "unit": "GB/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": sum(e["launches"] for e in entries) * args.steps,
        "clocks": clk,
        "secondary": secondary,
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        result["cpu_baseline"] = cpu_baseline(mats, budget_s=args.cpu_seconds)
    if solves is not None:  # the Krylov solve times, the metric's second half, as the line's last key
        result["solves"] = solves
    for e in entries:
        spx.spx_matrix_destroy(e["A"])
    spx.spx_ctx_destroy(ctx)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.destroy_process_group()


def solve_bytes_per_iter(solver: str, fmt_bytes: int, n: int, m: int = 30, V: int = 8) -> int:
    """Algorithmic bytes of one FP64 iteration in this library's fused form:
    SpMV stream (fmt_bytes: matrix + gathered vector + result) plus the vector
    kernels.  CG: SpMV (+p re-read for p.q), x/r update (4 reads, 2 writes),
    p update (2 reads, 1 write).  BiCGSTAB: two SpMVs (+ dot operands), p, s,
    x/r updates.  GMRES(m), averaged over a cycle: SpMV + one Gram-Schmidt
    pass (the j+1 basis vectors read for the dots and again for the update, w
    read and written) + normalisation; a reorthogonalisation pass is extra
    work, not counted.  V: bytes per vector element (8 FP64, 4 FP32)."""
    if solver == "cg":
        return fmt_bytes + V * n + 6 * V * n + 3 * V * n
    if solver == "bicgstab":
        return 2 * fmt_bytes + 2 * V * n + 4 * V * n + 3 * V * n + 8 * V * n
    if solver == "cgs":  # v = A p (+r^), q/w/x (3 reads, 3 writes), A w, r (3 reads, 1 write), u/p (3 reads, 2 writes)
        return 2 * fmt_bytes + V * n + 6 * V * n + 4 * V * n + 5 * V * n
    jbar = (m + 1) / 2.0
    return int(fmt_bytes + 2 * (jbar + 1) * V * n + 2 * V * n + 2 * V * n)


def small_case_secondary(spx, ctx, stream, dev, reps: int = 50):
    """The small configuration (latency-bound, reported in microseconds): the 2D
    5-point Laplacian on a 64 x 64 grid (n = 4096, 20,224 nonzeros), FP64 CSR,
    b = A x* with x* ~ U[-1, 1]: one SpMV (median of `reps` CUDA-event timings)
    and unpreconditioned CG to relative residual 1e-10."""
    import torch
    from paper_2103_10116_gb300 import synth
    rp, col, val = synth.laplace2d_5pt(64)
    n = rp.shape[0] - 1
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    out = {"n": n, "nnz": int(col.shape[0])}
    with torch.cuda.stream(stream):
        A = spx.spx_matrix_create(ctx, "csr", t(rp), t(col), t(val))
        xs = t(np.random.default_rng(0).uniform(-1, 1, n))
        b = torch.empty_like(xs)
        for _ in range(3):
            spx.spx_spmv(ctx, A, xs, b)
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            spx.spx_spmv(ctx, A, xs, b)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        out["spmv_us"] = round(statistics.median(ts), 2)
        x = torch.zeros_like(xs)
        spx.spx_solve(ctx, A, b, x, "cg", 1e-10, 10000)  # warm-up
        x.zero_()
        si = spx.spx_solve(ctx, A, b, x, "cg", 1e-10, 10000)
        out["cg"] = {"solve_ms": round(si.time_ms, 3), "iterations": si.iterations, "status": si.status_name,
                     "relres_true": si.relres_true,
                     "err_vs_xstar": float(torch.linalg.norm(x - xs) / torch.linalg.norm(xs))}
        spx.spx_matrix_destroy(A)
    return out


def solve_secondary(spx, ctx, stream, dev, peak, fmt="csr"):
    """Krylov solves to relative residual 1e-10 with b = A x*, x* ~ U[-1,1]
    (solve_ms: the median of three timed solves after a warm-up):
    CG on the 128^3 7-point Poisson matrix; BiCGSTAB and GMRES(30) on the
    128^3 upwind convection-diffusion matrix (Peclet 10).  FP64 and FP32
    inner iterations inside FP64 refinement ("mixed").  Storage `fmt`."""
    import torch
    from paper_2103_10116_gb300 import synth
    out = {}
    cd = synth.convdiff3d_upwind(128)
    cases = [("cg_poisson128", synth.laplace3d_7pt(128), "cg"),
             ("bicgstab_convdiff128", cd, "bicgstab"),
             ("cgs_convdiff128", cd, "cgs"),
             ("gmres30_convdiff128", cd, "gmres")]
    for name, (rp, col, val), solver in cases:
        n = rp.shape[0] - 1
        res = {"n": n, "nnz": int(col.shape[0]), "tol": 1e-10, "format": fmt}
        with torch.cuda.stream(stream):
            A = spx.spx_matrix_create(ctx, fmt, torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev),
                                      torch.from_numpy(val).to(dev), flags=spx.SPX_MIXED_SHADOW)
            info = spx.spx_matrix_get_info(A)
            xs = torch.from_numpy(np.random.default_rng(3).uniform(-1, 1, n)).to(dev)
            b = torch.empty(n, dtype=torch.float64, device=dev)
            spx.spx_spmv(ctx, A, xs, b)
            fmt_bytes = algorithmic_bytes(fmt, 8, n, n, col.shape[0], info["ell_width"], info["coo_nnz"])
            for prec in ("f64", "mixed"):
                x = torch.zeros(n, dtype=torch.float64, device=dev)
                spx.spx_solve(ctx, A, b, x, solver, 1e-10, 20000, restart=30, precision=prec)  # warm-up
                times = []
                for _ in range(3):  # the median of three timed solves
                    x.zero_()
                    torch.cuda.synchronize()
                    si = spx.spx_solve(ctx, A, b, x, solver, 1e-10, 20000, restart=30, precision=prec)
                    times.append(si.time_ms)
                t_ms = statistics.median(times)
                err = float(torch.linalg.norm(x - xs) / torch.linalg.norm(xs))
                r = {"solve_ms": round(t_ms, 2), "iterations": si.iterations, "status": si.status_name,
                     "relres_true": si.relres_true, "err_vs_xstar": err, "restarts": si.restarts}
                if prec == "f64" and si.iterations > 0:
                    bpi = solve_bytes_per_iter(solver, fmt_bytes, n)
                    gbs = bpi * si.iterations / (t_ms * 1e-3) / 1e9
                    r.update({"bytes_per_iter": bpi, "achieved_GB_s": round(gbs, 1),
                              "frac_of_hbm_peak": round(gbs / peak, 3),
                              "roofline_ms": round(bpi * si.iterations / (peak * 1e9) * 1e3, 2)})
                res[prec] = r
            spx.spx_matrix_destroy(A)
        out[name] = res
    return out


def jacobi_secondary(spx, ctx, stream, dev, max_iter: int = 20000):
    """Jacobi (M = diag A) and block-Jacobi (blocks of 8 rows; FP64 inverses,
    and adaptive storage with FP32 copies of well-conditioned blocks)
    preconditioning against the plain solvers on 128^3 matrices: the 7-point Poisson matrix
    scaled symmetrically, S A S with s_i = exp(U[-2, 2]) (CG); the upwind
    convection-diffusion matrix (Peclet 10) with rows scaled by exp(U[-3, 3])
    (BiCGSTAB, CGS, GMRES(30)); and the stress variant with cell Peclet
    number 10 (Peclet 10 * 129), unscaled, where the constant diagonal leaves
    Jacobi nothing to do and the blocks hold the strong upwind couplings along
    x.  b = A x*, tol 1e-10, FP64, CSR.  solve_ms: the median of up to three
    solves after one that builds the preconditioner (first_solve_ms); solves
    from a matrix's second on replay CUDA graphs."""
    import torch
    from paper_2103_10116_gb300 import synth
    rng = np.random.default_rng(21)

    def scaled(rp, col, val, rs, cs):
        rows = np.repeat(np.arange(rp.shape[0] - 1), np.diff(rp))
        return rp, col, val * rs[rows] * cs[col]

    rp, col, val = synth.laplace3d_7pt(128)
    sp = np.exp(rng.uniform(-2.0, 2.0, size=rp.shape[0] - 1))
    poisson = scaled(rp, col, val, sp, sp)
    rp, col, val = synth.convdiff3d_upwind(128)
    cdiff = scaled(rp, col, val, np.exp(rng.uniform(-3.0, 3.0, size=rp.shape[0] - 1)), np.ones(rp.shape[0] - 1))
    stress = synth.convdiff3d_upwind(128, peclet=10.0 * 129)
    out = {}
    for name, (rp, col, val), solvers in (("poisson128_sym_scaled", poisson, ("cg",)),
                                          ("convdiff128_row_scaled", cdiff, ("bicgstab", "cgs", "gmres")),
                                          ("convdiff128_cell_peclet10", stress, ("bicgstab", "cgs", "gmres"))):
        n = rp.shape[0] - 1
        with torch.cuda.stream(stream):
            A = spx.spx_matrix_create(ctx, "csr", torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev),
                                      torch.from_numpy(val).to(dev))
            xs = torch.from_numpy(np.random.default_rng(3).uniform(-1, 1, n)).to(dev)
            b = torch.empty(n, dtype=torch.float64, device=dev)
            spx.spx_spmv(ctx, A, xs, b)
            res = {}
            for solver in solvers:
                for pc, tag in ((None, ""), ("jacobi", "_jacobi"), ("block_jacobi", "_block8"),
                                ("adaptive_block_jacobi", "_block8_adaptive")):
                    x = torch.zeros(n, dtype=torch.float64, device=dev)
                    first = spx.spx_solve(ctx, A, b, x, solver, 1e-10, max_iter, restart=30, precond=pc,
                                          block_size=8)  # builds M^-1
                    times = []
                    for _ in range(3 if first.time_ms < 1000 else 1):  # median of up to three timed solves
                        x.zero_()
                        si = spx.spx_solve(ctx, A, b, x, solver, 1e-10, max_iter, restart=30, precond=pc,
                                           block_size=8)
                        times.append(si.time_ms)
                    res[f"{solver}{tag}"] = {
                        "solve_ms": round(statistics.median(times), 2), "first_solve_ms": round(first.time_ms, 2),
                        "iterations": si.iterations, "status": si.status_name, "relres_true": si.relres_true}
            spx.spx_matrix_destroy(A)
        out[name] = res
    return out


def solver_flops_per_iter(solver: str, n: int, nnz: int, m: int = 30) -> float:
    """Floating-point operations of one iteration (an FMA counts 2): SpMVs
    2 nnz each, dot products and vector updates 2n per FMA each.  GMRES(m):
    one Gram-Schmidt pass (dots and update over the j+1 basis vectors),
    the norm and the scaling, averaged over a cycle."""
    if solver == "cg":       # A p; p.q, r.r; x, r, p updates
        return 2 * nnz + 10 * n
    if solver == "bicgstab":  # A p, A s; r^.v, s.s, t.s, t.t, r.r, r^.r; p (2 FMA), s, x (2), r
        return 4 * nnz + 24 * n
    if solver == "cgs":       # A p, A w; r^.v, r.r, r^.r; q, w (add), x, r, u, p (2 FMA)
        return 4 * nnz + 19 * n
    jbar = (m - 1) / 2.0
    return 2 * nnz + 4 * (jbar + 1) * n + 3 * n


def fixed_iter_secondary(spx, ctx, stream, dev, iters: int = 1000):
    """The solver throughput protocol of Section 6.4: each Krylov solver runs
    exactly `iters` iterations after a warm-up, with COO SpMV, reported in
    GFLOP/s (solver_flops_per_iter).  Matrix: the 128^3 7-point Poisson
    matrix (SPD, so every solver is defined on it), FP64 and FP32."""
    import torch
    from paper_2103_10116_gb300 import synth
    rp, col, val = synth.laplace3d_7pt(128)
    n, nnz = rp.shape[0] - 1, int(col.shape[0])
    out = {"matrix": "7-point Poisson 128^3", "n": n, "nnz": nnz, "format": "coo", "iterations": iters}
    for tdt, name in ((torch.float64, "f64"), (torch.float32, "f32")):
        with torch.cuda.stream(stream):
            A = spx.spx_matrix_create(ctx, "coo", torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev),
                                      torch.from_numpy(val).to(dev).to(tdt))
            b = torch.from_numpy(np.random.default_rng(6).uniform(-1, 1, n)).to(dev).to(tdt)
            res = {}
            for solver in ("cg", "bicgstab", "cgs", "gmres"):
                x = torch.zeros(n, dtype=tdt, device=dev)
                spx.spx_solve_fixed(ctx, A, b, x, solver, 30, restart=30, precision=name)  # warm-up
                times = []
                for _ in range(3):  # the median of three timed runs
                    x.zero_()
                    torch.cuda.synchronize()
                    si = spx.spx_solve_fixed(ctx, A, b, x, solver, iters, restart=30, precision=name)
                    times.append(si.time_ms)
                t_ms = statistics.median(times)
                fl = solver_flops_per_iter(solver, n, nnz) * si.iterations
                res[solver] = {"ms": round(t_ms, 2), "iterations": si.iterations,
                               "gflops": round(fl / (t_ms * 1e-3) / 1e9, 1)}
            spx.spx_matrix_destroy(A)
        out[name] = res
    return out


def gather_floor(spx, ctx, stream, mats, dev, steps: int = 10):
    """Per matrix and value type: the time of the gather-only probe
    (spx_probe_gather: stream the column indices, gather x at each), the
    floor any SpMV kernel has on that sparsity pattern.  L2 is flushed (a
    256 MB write) before every launch, as the sweep leaves it cold."""
    import torch
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    out = {}
    for mname, (rp, col, val) in mats.items():
        n = rp.shape[0] - 1
        col_d = torch.from_numpy(col).to(dev)
        for tdt, tag in ((torch.float64, "f64"), (torch.float32, "f32")):
            x = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, n)).to(dev).to(tdt)
            o = torch.zeros(1, dtype=tdt, device=dev)
            ts = []
            with torch.cuda.stream(stream):
                for k in range(steps + 2):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    spx.spx_probe_gather(ctx, col_d, x, o)
                    e1.record(stream)
                    e1.synchronize()
                    if k >= 2:
                        ts.append(e0.elapsed_time(e1))
            out[f"{mname}/{tag}"] = round(statistics.median(ts) * 1e3, 1)
        del col_d
    return out


def vendor_secondary(mats, dev, steps: int = 10):
    """Context only (never on the library's path): PyTorch's CSR
    matrix-vector product, which calls the vendor sparse library, on the
    sweep's CSR matrices, timed with CUDA events like the sweep (median over
    `steps` after 3 warm-ups, a 256 MB buffer written between launches so that
    L2 starts cold)."""
    import torch
    out = {"library": "torch.sparse CSR matvec (cuSPARSE)", "torch": torch.__version__}
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for mname, (rp, col, val) in mats.items():
        n, nnz = rp.shape[0] - 1, int(col.shape[0])
        for tdt, V, tag in ((torch.float64, 8, "f64"), (torch.float32, 4, "f32")):
            try:
                A = torch.sparse_csr_tensor(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev),
                                            torch.from_numpy(val).to(dev).to(tdt), size=(n, n))
                x = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, n)).to(dev).to(tdt)
                for _ in range(3):
                    torch.mv(A, x)
                ts = []
                for _ in range(steps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    torch.mv(A, x)
                    e1.record()
                    e1.synchronize()
                    ts.append(e0.elapsed_time(e1))
                ms = statistics.median(ts)
                b = algorithmic_bytes("csr", V, n, n, nnz)
                out[f"{mname}/csr/{tag}"] = {"us": round(ms * 1e3, 1), "GB_s": round(b / (ms * 1e-3) / 1e9, 1)}
                del A
            except Exception as e:  # a torch build without the sparse path: report, do not fail the bench
                out[f"{mname}/csr/{tag}"] = {"unavailable": str(e).splitlines()[0][:120]}
    return out


def batched_secondary(spx, ctx, stream, dev, plain_sample=4096):
    """4096 SPD systems, n_i ~ U{100..10000}, 2D 5-point Laplacian of the
    ragged n_i-row grid plus a diagonal shift ~ U[0.01, 1], b_i = A_i x*_i:
    one persistent batched CG launch (FP64, and FP32 inner + FP64 refinement)
    to 1e-10, against the plain per-system FP64 path (spx_solve per system on
    resident matrices, every system timed once after a warm-up solve of each;
    a smaller `plain_sample` times the first systems and scales to the batch)."""
    import scipy.sparse as sp
    import torch
    from paper_2103_10116_gb300 import synth
    nsys = 4096
    ro, no, rp, col, val = synth.batch_ragged_laplace(nsys, 100, 10000, seed=4)
    xs = np.random.default_rng(5).uniform(-1, 1, int(ro[-1]))
    b = np.empty_like(xs)
    for s in range(nsys):
        r0, r1 = int(ro[s]), int(ro[s + 1])
        A = sp.csr_matrix((val[no[s]:no[s + 1]], col[no[s]:no[s + 1]], rp[r0 + s:r1 + s + 1]), shape=(r1 - r0,) * 2)
        b[r0:r1] = A @ xs[r0:r1]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    out = {"systems": nsys, "rows": int(ro[-1]), "nnz": int(no[-1]), "tol": 1e-10}
    with torch.cuda.stream(stream):
        B = spx.spx_batch_create(ctx, ro, no, t(rp), t(col), t(val), flags=spx.SPX_MIXED_SHADOW)
        bd, xsd = t(b), t(xs)
        for prec in ("f64", "mixed"):
            chosen = spx.spx_batch_tune(ctx, B, "cg", prec)
            x = torch.zeros_like(bd)
            spx.spx_batch_solve(ctx, B, bd, x, nsys, "cg", 1e-10, 20000, precision=prec)  # warm-up + graph
            x.zero_()
            els = []
            for _ in range(3):  # the median of three timed batch solves
                x.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                infos = spx.spx_batch_solve(ctx, B, bd, x, nsys, "cg", 1e-10, 20000, precision=prec)
                els.append(time.perf_counter() - t0)
            el = statistics.median(els)
            conv = sum(1 for i in infos if i.status == spx.SPX_CONVERGED)
            err = float(torch.linalg.norm(x - xsd) / torch.linalg.norm(xsd))
            out[prec] = {"solve_ms": round(el * 1e3, 2), "solves_per_s": round(nsys / el, 1), "converged": conv,
                         "threads_per_system": chosen, "err_vs_xstar": err,
                         "max_relres": max(i.relres_true for i in infos)}
            if prec == "f64":
                # bytes per CG iteration of system s: its CSR arrays (12 nnz + 4 (n + 1)) and the
                # global vectors (q written and read, x and r read and written: 48 n); p lives in
                # shared memory.  Most of it is served from L2 while a block works on its system.
                its = np.array([i.iterations for i in infos], dtype=np.float64)
                ns, nzs = np.diff(ro).astype(np.float64), np.diff(no).astype(np.float64)
                tot_b = float(np.sum(its * (12 * nzs + 4 * (ns + 1) + 48 * ns)))
                gbs = tot_b / el / 1e9
                peak, _ = _peaks()
                out[prec].update({"iterations_total": int(its.sum()), "bytes_total": int(tot_b),
                                  "bytes_per_solve": int(tot_b / nsys), "achieved_GB_s": round(gbs, 1),
                                  "frac_of_hbm_peak": round(gbs / peak, 3),
                                  "note": "algorithmic bytes of every iteration (matrix + global vectors); "
                                          "most iterations re-read a system that sits in L2, so the fraction "
                                          "can exceed what HBM alone could serve"})
        spx.spx_batch_destroy(B)
        # the plain per-system FP64 path: matrices resident, one spx_solve per system
        el = 0.0
        plain_sample = min(plain_sample, nsys)
        for s in range(plain_sample):
            r0, r1 = int(ro[s]), int(ro[s + 1])
            A = spx.spx_matrix_create(ctx, "csr", t(rp[r0 + s:r1 + s + 1]), t(col[no[s]:no[s + 1]]),
                                      t(val[no[s]:no[s + 1]]))
            x = torch.zeros(r1 - r0, dtype=torch.float64, device=dev)
            bs = t(b[r0:r1])
            spx.spx_solve(ctx, A, bs, x, "cg", 1e-10, 20000)  # warm-up
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            spx.spx_solve(ctx, A, bs, x, "cg", 1e-10, 20000)
            el += time.perf_counter() - t0
            spx.spx_matrix_destroy(A)
        rows_sample = int(ro[plain_sample])
        est = el * (int(ro[-1]) / rows_sample)
        out["plain_per_system_f64"] = {"systems_timed": plain_sample, "timed_ms": round(el * 1e3, 2),
                                       "batch_ms": round(est * 1e3, 1), "solves_per_s": round(nsys / est, 1),
                                       "how": "measured over every system" if plain_sample == nsys else
                                              "the first systems, scaled to the batch by rows"}
        out["speedup_f64_vs_plain"] = round(est * 1e3 / out["f64"]["solve_ms"], 1)
        out["speedup_mixed_vs_plain"] = round(est * 1e3 / out["mixed"]["solve_ms"], 1)
    return out


def plain_serial_f64(spx, ctx, make, count, tol, budget_s=8.0):
    """The plain per-system FP64 path on the first requests of the trace, one
    at a time: upload the operator (host CSR), solve in FP64, read x back."""
    import torch
    t0 = time.perf_counter()
    done = 0
    for i in range(count):
        _, (rp, col, val, b), solver, _ = make(i)
        A = spx.spx_matrix_create(ctx, "csr", torch.from_numpy(rp), torch.from_numpy(col), torch.from_numpy(val))
        try:
            bd = torch.from_numpy(b).cuda()
            xd = torch.zeros_like(bd)
            spx.spx_solve(ctx, A, bd, xd, solver=solver, tol=tol, max_iter=100000, precision="f64")
            xd.cpu()
        finally:
            spx.spx_matrix_destroy(A)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return {"sample_requests": done, "sample_s": round(el, 2), "solves_per_s": round(done / el, 1)}


def family_columns(j, m, v, row, diag, n: int, nnz: int):
    """The column indices of the size-n member of synth.DiagDomFamily from its
    per-entry draws (torch tensors on any device; the same integers as
    DiagDomFamily.matrix)."""
    import torch
    j, m, r = j[:nnz], m[:nnz], row[:nnz]
    lo = torch.div(j * (n - 1), m, rounding_mode="floor")
    w = torch.div((j + 1) * (n - 1), m, rounding_mode="floor") - lo
    c = lo + torch.minimum((v[:nnz] * w).long(), w - 1)
    c += (c >= r).long()
    return torch.where(diag[:nnz], r, c).int()


def _host_bytes_cap():
    """Host memory the serving replay may hold in request payloads: a quarter of
    what the machine has available, at most 24 GB."""
    try:
        with open("/proc/meminfo") as f:
            avail = next(int(ln.split()[1]) * 1024 for ln in f if ln.startswith("MemAvailable:"))
    except Exception:
        avail = 32 << 30
    return float(min(24 << 30, avail // 4))


def serving_secondary(spx, ctx, dev, seconds: float = 10.0, rate: float = 2000.0, slots: int = 16, gather_rate=None,
                      batch_rows=None, plain=True):
    """Poisson arrivals (rate req/s for `seconds`) of solve requests whose sizes
    are drawn continuously from log-U[1e3, 1e6] rows, 50/50 from two families:
    3D 7-point stencils (k = round(n^(1/3)), n := k^3, CG) and diagonally
    dominant random rows with 8-32 nonzeros at exactly the drawn size
    (BiCGSTAB; synth.DiagDomFamily); tolerance 1e-8, FP32 inner iterations +
    FP64 refinement; admission by device footprint (90% of free memory).
    Operators come from pinned host memory and are uploaded per request; those
    of at most batch_rows rows go to the batch lanes (None: the server default,
    0: none).  Payloads are built in arrival order by a producer thread (the
    random family's columns and every right-hand side are formed on the GPU and
    copied to pinned host memory) and submitted when due, with a bound on the
    host bytes held; latency counts from each request's arrival time."""
    import collections
    import threading

    import torch
    from paper_2103_10116_gb300 import synth
    from paper_2103_10116_gb300.serving import Server, latency_stats, poisson_trace, replay_lazy
    rng = np.random.default_rng(5)
    trace = poisson_trace(rate, seconds, seed=5)
    N = trace.shape[0]
    drawn = np.rint(np.exp(rng.uniform(np.log(1e3), np.log(1e6), size=N))).astype(np.int64)
    stencil_fam = rng.random(N) < 0.5
    ks = np.rint(np.cbrt(drawn)).astype(np.int64)
    rows = np.where(stencil_fam, ks ** 3, drawn)
    F = synth.DiagDomFamily(1_000_000, seed=7)
    # request payloads live in pinned host memory, as a serving front end's receive buffers would
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    f_rp, f_val = pin(F.rp), pin(F.val)
    gstream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(gstream):
        d_row = torch.from_numpy(F.row).to(dev)
        d_j = torch.from_numpy(F.j).to(dev)
        d_m = torch.from_numpy(F.m).to(dev)
        d_v = torch.from_numpy(F.v).to(dev)
        d_diag = torch.from_numpy(F.diag).to(dev)
    stencils = {}

    def build(i):
        n = int(rows[i])
        with torch.cuda.stream(gstream):
            g = torch.Generator(device=dev)
            g.manual_seed(10_000 + i)
            bh = torch.empty(n, dtype=torch.float64, pin_memory=True)
            bh.copy_(torch.rand(n, generator=g, device=dev, dtype=torch.float64).mul_(2.0).sub_(1.0),
                     non_blocking=True)
            if stencil_fam[i]:
                k = int(ks[i])
                if k not in stencils:
                    stencils[k] = tuple(pin(a) for a in synth.laplace3d_7pt(k))
                rp, col, val = stencils[k]
                nbytes = 16 * n
            else:
                nnz = int(F.rp[n])
                colh = torch.empty(nnz, dtype=torch.int32, pin_memory=True)
                colh.copy_(family_columns(d_j, d_m, d_v, d_row, d_diag, n, nnz), non_blocking=True)
                rp, val = f_rp[: n + 1], f_val[:nnz]
                nbytes = 16 * n + 4 * nnz
            gstream.synchronize()
            col = col if stencil_fam[i] else colh.numpy()
        # the numpy views keep the pinned buffers alive until the server is done with them
        return ("host", (rp, col, val, bh.numpy()), "cg" if stencil_fam[i] else "bicgstab", nbytes)

    cap = _host_bytes_cap()
    ready = collections.OrderedDict()
    cv = threading.Condition()
    state = {"next": 0, "bytes": 0.0, "stop": False, "err": None}

    def producer():  # builds payloads in arrival order, at most `cap` host bytes ahead
        try:
            while True:
                with cv:
                    cv.wait_for(lambda: state["stop"] or state["bytes"] < cap / 2)
                    if state["stop"] or state["next"] >= N:
                        return
                    i = state["next"]
                    state["next"] += 1
                item = build(i)
                with cv:
                    ready[i] = item
                    state["bytes"] += item[3]
                    cv.notify_all()
        except Exception as e:  # reported by make()
            with cv:
                state["err"] = e
                cv.notify_all()

    def make(i):
        with cv:
            cv.wait_for(lambda: i in ready or state["err"] is not None)
            if state["err"] is not None:
                raise state["err"]
            item = ready.pop(i)
            state["bytes"] -= item[3]
            cv.notify_all()
        return item

    prod = threading.Thread(target=producer, daemon=True)
    prod.start()
    with cv:  # a head start: the first second of arrivals built before the clock starts
        cv.wait_for(lambda: state["next"] >= min(N, int(rate)) or state["bytes"] >= cap / 2 or state["err"])
    srv = Server(ctx, 0, max_slots=slots, batch_rows=batch_rows, keep_x=False)
    try:
        eff_rows = spx.spx_server_set_batching(srv.h, -1)
        cl_rows = spx.spx_server_set_cluster_rows(srv.h, -1)
        wall, ids, delays = replay_lazy(srv, trace, make, max_pending_bytes=cap / 2, tol=1e-8, precision="mixed")
        res = [srv.results[i] for i in ids]
    finally:
        srv.close()
        with cv:
            state["stop"] = True
            cv.notify_all()
        prod.join()
    st = latency_stats(res, delays)
    conv = sum(1 for r in res if r["info"].status == spx.SPX_CONVERGED and r["error"] == 0)
    peak, _ = _peaks()
    # the offered load at the HBM roofline: every request's FP32 inner iterations and FP64 outer
    # residuals at their algorithmic bytes
    nnz_of = np.where(stencil_fam, 7 * rows - 6 * ks ** 2, F.rp[np.minimum(rows, F.n_max)])
    # and the same with each request's random gathers of x at the rate the gather probe measures
    # (one L2 request each: the random family's columns are uniform over the matrix)
    roof_i, floor_i = [], []
    for i, r in enumerate(res):
        n, nnz, solver = int(rows[i]), int(nnz_of[i]), "cg" if stencil_fam[i] else "bicgstab"
        inner = solve_bytes_per_iter(solver, algorithmic_bytes("csr", 4, n, n, nnz), n, V=4)
        outer = algorithmic_bytes("csr", 8, n, n, nnz) + 5 * 8 * n
        t_hbm = (r["info"].inner_iterations * inner + max(1, r["info"].restarts) * outer) / (peak * 1e9)
        roof_i.append(t_hbm)
        products = r["info"].inner_iterations * (1 if solver == "cg" else 2) + max(1, r["info"].restarts)
        t_gather = products * nnz / gather_rate if (gather_rate and not stencil_fam[i]) else 0.0
        floor_i.append(max(t_hbm, t_gather))
    roof = float(sum(roof_i))
    floor = float(sum(floor_i))

    def phases(sel):
        if not sel:
            return None
        out = {"requests": len(sel)}
        for ph in ("upload_ms", "setup_ms", "solve_ms", "download_ms"):
            v = np.array([r[ph] for r in sel])
            out[ph] = {"p50": round(float(np.percentile(v, 50)), 3), "p90": round(float(np.percentile(v, 90)), 3),
                       "sum_s": round(float(v.sum()) / 1e3, 2)}
        return out

    slot_res = [r for r in res if not r["batched"]]
    # where the time goes, by size: the requests' own solve phases against their roofline time
    buckets = {}
    for lo, hi in ((1e3, 2.5e4), (2.5e4, 1e5), (1e5, 3e5), (3e5, 1.01e6)):
        sel = [i for i in range(len(res)) if lo <= rows[i] < hi]
        if not sel:
            continue
        roof_ms = [roof_i[i] * 1e3 for i in sel]
        solve_ms = [res[i]["solve_ms"] for i in sel]
        buckets[f"{int(lo)}-{int(hi)}"] = {
            "requests": len(sel), "batched": int(sum(1 for i in sel if res[i]["batched"])),
            "one_cluster": int(sum(1 for i in sel if res[i]["route"] == "cluster")),
            "roofline_s": round(sum(roof_ms) / 1e3, 2),
            "floor_s": round(sum(floor_i[i] for i in sel), 2), "solve_phase_s": round(sum(solve_ms) / 1e3, 2),
            "upload_phase_s": round(sum(res[i]["upload_ms"] for i in sel) / 1e3, 2),
            "setup_phase_s": round(sum(res[i]["setup_ms"] for i in sel) / 1e3, 2)}
    bad = [{"request": i, "rows": int(rows[i]), "family": "stencil" if stencil_fam[i] else "random",
            "batched": bool(r["batched"]), "error": r["error"], "status": r["info"].status_name,
            "iterations": r["info"].iterations, "restarts": r["info"].restarts, "relres": r["info"].relres_true}
           for i, r in enumerate(res) if r["info"].status != spx.SPX_CONVERGED or r["error"] != 0]
    st.update({"requests": len(res), "converged": conv, "not_converged": bad[:12],
               "arrival_rate_per_s": rate, "window_s": seconds,
               "wall_s": round(wall, 2), "solves_per_s": round(len(res) / wall, 1), "slots": slots,
               "batch_rows": int(eff_rows), "batched_requests": int(sum(1 for r in res if r["batched"])),
               "sizes": "log-uniform rows in [1e3, 1e6], exact per request (stencils: the nearest k^3)",
               "distinct_sizes": int(np.unique(rows).size),
               "offered_gpu_s_at_roofline": round(roof, 2),
               "rho_at_roofline": round(roof / seconds, 3),
               "capacity_solves_per_s_at_roofline": round(len(res) / roof, 1),
               "achieved_frac_of_roofline_capacity": round(roof / wall, 3),
               "offered_gpu_s_at_floor": round(floor, 2),
               "floor": "per request the larger of its HBM roofline time and its random gathers of x at the "
                        "gather probe's rate on the power-law pattern (random family only)",
               "achieved_frac_of_floor_capacity": round(floor / wall, 3),
               "cluster_rows": int(cl_rows),
               "one_cluster_requests": int(sum(1 for r in res if r["route"] == "cluster")),
               "client_delay_ms_p50": round(float(np.percentile(delays, 50)), 3),
               "host_bytes_cap": int(cap),
               "by_size": buckets,
               "phases_slot_route": phases([r for r in slot_res if r["route"] == "slot"]),
               "phases_cluster_route": phases([r for r in slot_res if r["route"] == "cluster"]),
               "phases_batch_route": phases([r for r in res if r["batched"]])})
    if plain:
        st["plain_per_system_f64"] = plain_serial_f64(spx, ctx, build, min(400, N), 1e-8)
        st["speedup_vs_plain_f64"] = round(st["solves_per_s"] / st["plain_per_system_f64"]["solves_per_s"], 2)
    return st


def _cpu_spmv_rate(fn, mats, budget_s):
    """GB/s (CSR FP64 byte model) of fn over whole-matrix SpMVs of the sweep
    matrices, repeated until about budget_s seconds have passed."""
    tot_b, tot_t, reps = 0, 0.0, 0
    xs = {k: np.random.default_rng(1).uniform(-1, 1, v[0].shape[0] - 1) for k, v in mats.items()}
    t_start = time.perf_counter()
    while time.perf_counter() - t_start < budget_s or reps == 0:
        for name, (rp, col, val) in mats.items():
            n = rp.shape[0] - 1
            t = time.perf_counter()
            fn(rp, col, val, xs[name])
            tot_t += time.perf_counter() - t
            tot_b += algorithmic_bytes("csr", 8, n, n, col.shape[0])
        reps += 1
    return tot_b / tot_t / 1e9, reps, tot_t


def cpu_baseline(mats, budget_s=15.0):
    """The CPU oracle's plain FP64 CSR SpMV (the literal index-order loop), on a
    bounded sample of the same workload: whole-matrix SpMVs of both sweep
    matrices, repeated for about budget_s / 2 seconds on all host cores (the
    OpenMP build: rows shared among threads) and as long on one core."""
    import oracle
    oracle.spmv_csr_plain_omp(*mats[next(iter(mats))], np.zeros(mats[next(iter(mats))][0].shape[0] - 1))  # build
    v_all, reps_all, t_all = _cpu_spmv_rate(oracle.spmv_csr_plain_omp, mats, budget_s / 2)
    v_one, reps_one, t_one = _cpu_spmv_rate(oracle.spmv_csr_plain, mats, budget_s / 2)
    cores = oracle.omp_threads()
    return {"value": round(v_all, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{reps_all} x (FP64 CSR SpMV of the 27-point 100^3 and power-law 2M matrices), "
                      f"{t_all:.1f} s on {cores} threads (OpenMP over rows, plain index-order sums)",
            "single_core": {"value": round(v_one, 3), "unit": "GB/s", "cores": 1,
                            "sample": f"{reps_one} x the same SpMVs, {t_one:.1f} s on one thread"}}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    import oracle
    mats = build_workload()
    xs = {k: np.random.default_rng(1).uniform(-1, 1, v[0].shape[0] - 1) for k, v in mats.items()}

    def step():
        b = 0
        for name, (rp, col, val) in mats.items():
            oracle.spmv_csr_plain_omp(rp, col, val, xs[name])
            n = rp.shape[0] - 1
            b += algorithmic_bytes("csr", 8, n, n, col.shape[0])
        return b

    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    tot = 0
    for _ in range(args.steps):
        tot += step()
    el = time.perf_counter() - t
    v = tot / el / 1e9
    cores = oracle.omp_threads()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (reference step: FP64 CSR SpMV of both matrices by the CPU oracle)"},
        "cpu_baseline": {"value": round(v, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": f"per step: one FP64 CSR SpMV of each sweep matrix (the oracle's plain "
                                   f"index-order loop, OpenMP over rows on {cores} threads)"},
        "e2e": {"value": round(v, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="spx", choices=["spx", "reference"])
    ap.add_argument("--no-solve", action="store_true", help="skip the CG solve-time section")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--only", default="", help="run only sweep entries whose name contains this, "
                                                 "e.g. stencil27_100/ell/f64 (for profiling)")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="0 disables the serving run")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "spx":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
