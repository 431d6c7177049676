#!/usr/bin/env python3
"""Benchmark: MLUPS of the fused collide-stream step on one GB300.

Workload (one "step" = one time level of the whole hot path: pull-stream,
moments, Hermite equilibrium, relaxation, store, FP64 diagnostics):
standing shear wave on a periodic 4096 x 4096 grid, D2Q36 Gauss-Hermite
product set (Lax-Wendroff streaming), third-order equilibrium, FP32 deviation
storage, Kn = 0.1, u_y = 1e-3 sin x + 1e-3 sin y sin x.  The on-lattice D2Q37
set on the same grid is measured alongside (per-quadrature metric).

Prints ONE JSON line (rank 0).  Under torchrun (N > 1) every rank runs its
own independent instance (weak scaling, no data-path collective); the time is
the max over ranks and the value the cell updates of all ranks per second.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores instead.
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS (million lattice-cell updates per second), fused collide-stream step"
WORKLOAD = "standing shear wave 4096x4096, D2Q36-GH (Lax-Wendroff), N=3, FP32 deviations, Kn=0.1"


def reduce_max_ms(ms, dist, device):
    """The job's time: the slowest rank's (all-reduce MAX over ranks; ms itself at N = 1)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(cells_per_rank, world, steps, ms):
    """Whole-job MLUPS of a weak-scaling run: every rank's cell updates over the job's time."""
    return cells_per_rank * world * steps / (ms / 1e3) / 1e6


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        smax = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.samples)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_digest():
    """Digest of the kernel sources' code (comments and blank space removed), so that an
    ncu traffic record stays tied to the code it was taken on."""
    h = hashlib.sha256()
    for f in ("lb_kernels.cuh", "lb_device.h", "velocity_sets.h"):
        with open(os.path.join(ROOT, "paper_0908_4520_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(quad):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    ent = rec.get(quad)
    if not ent or ent.get("kernel_digest") != kernel_digest():
        return None
    return ent.get("dram_bytes_per_full_launch")


# ----------------------------------------------------------------------------- GPU arm

def workload_name(args):
    if (args.n == 4096 and args.quad == "D2Q36-GH" and args.n_eq == 3 and args.precision == "f32"
            and args.scheme == "second_order" and args.streaming == "lax_wendroff"):
        return WORKLOAD
    scheme = ", first-order scheme (Eq. slb)" if args.scheme == "first_order" else ""
    scheme += ", second-order upwind streaming" if args.streaming == "upwind2" else ""
    return (f"standing shear wave {args.n}x{args.n}, {args.quad}, N={args.n_eq}, {args.precision} deviations, "
            f"Kn={args.kn}{scheme}")


def kernel_label(args, tma):
    st = {"f32": "float", "f64": "double", "f16": "__half", "bf16": "__nv_bfloat16"}[args.precision]
    if tma == 2:
        return f"lb_tma_step_kernel<{args.quad}, {args.n_eq}, {st}, upwind=0, kStep, store_staged=1>"
    if tma:
        return f"lb_tma_step_kernel<{args.quad}, {args.n_eq}, {st}>"
    return f"lb_fused_kernel<{args.quad}, {args.n_eq}, {st}, kStep>"


def dvm_crosscheck(capi, Lattice, args, n=256, t_end=6.0):
    """Same-quadrature cross-check (Sec. 3.2): the lattice run of the benchmark's set on an
    n x n subgrid (free wave u_y = 1e-3 sin x) against the GPU DVM with the same 1-D
    Gauss-Hermite rule; max |A_LB - A_DVM| / U0 over t in [0, t_end]."""
    import numpy as np

    nodes = {"D2Q16-GH": 4, "D2Q36-GH": 6, "D2Q64-GH": 8}.get(args.quad)
    if nodes is None:
        return None
    u0 = 1e-3
    L = Lattice(args.quad, args.n_eq, n, n, args.kn, precision="f32", diag_capacity=1 << 14)
    L.init_shear_wave(u0)
    dt, tau = L.info["dt"], L.info["tau"]
    L.step(int(t_end / dt))
    rec = L.diagnostics()
    L.close()
    dt_dvm = 0.5 * (2 * np.pi / n) / float(np.max(np.abs(np.polynomial.hermite_e.hermegauss(nodes)[0])))
    nd = int(t_end / dt_dvm) + 2
    A, _ = capi.lb_dvm_run([tau], nodes, n, u0, nd)
    td = dt_dvm * np.arange(nd + 1)
    diff = float(np.max(np.abs(rec["amp"] - np.interp(rec["t"], td, A[0]))) / u0)
    return {"grid": f"{n}x{n}", "kn": args.kn, "t_end": t_end, "max_abs_amp_diff_over_u0": round(diff, 7),
            "dvm": f"GPU DVM, {nodes}-point Gauss-Hermite rule, nx {n}, cfl 0.5, FP64",
            "lb": f"{args.quad} N={args.n_eq}, FP32"}


def time_quadrature(torch, Lattice, quad, nx, ny, steps, warmup, kn, n_eq=3, precision="f32",
                    scheme="second_order", streaming="lax_wendroff", step_kernel="auto"):
    stream = torch.cuda.Stream()
    if not quad.endswith("-GH"):
        streaming = "lax_wendroff"  # on-lattice sets stream by the exact shift
        step_kernel = "auto" if step_kernel == "tma_store" else step_kernel
    L = Lattice(quad, n_eq, nx, ny, kn, precision=precision, stream=stream.cuda_stream, scheme=scheme,
                streaming=streaming, step_kernel=step_kernel)
    L.init_shear_wave(1e-3, 1e-3)
    L.step(warmup)
    L.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = L.launches
    return L, stream, ev0, ev1, n0


def error_vs_oracle(Lattice, args, futs):
    """Error of the benchmark's configuration against the FP64 oracle at the benchmark's run
    length: the GPU lattice nx x nx in the benchmark's launch configuration, started from the
    y-independent wave u_y = 1e-3 sin x (u1 = 0), so that every row equals the oracle's
    nx x 1 run.  Relative L2 of u_y and sigma_xy over sampled rows, the amplitude A(n) at
    every level, and the decay rate (the library's FP64 fit on the GPU records, the oracle's
    fit on its own, same window)."""
    import numpy as np

    out = {}
    for quad, fut in futs.items():
        L = Lattice(quad, args.n_eq, args.n, args.n, args.kn, precision=args.precision, scheme=args.scheme,
                    streaming=args.streaming if quad.endswith("-GH") else "lax_wendroff",
                    diag_capacity=args.check_steps + 8)
        L.init_shear_wave(1e-3, 0.0)
        L.step(args.check_steps)
        rec = L.diagnostics()
        m = L.moments()
        t_fit = min(5.0 * L.info["tau"], rec["t"][-1] / 4.0)
        try:
            rate = L.fit_decay(t_fit)[0]
        except Exception:
            rate = float("nan")
        L.close()
        o = fut.result()
        rows = slice(0, args.n, max(1, args.n // 64))
        uy, sxy = m["uy"][rows], m["sxy"][rows]
        ub = np.broadcast_to(o["uy"], uy.shape)
        sb = np.broadcast_to(o["sxy"], sxy.shape)
        out[quad] = {
            "uy_rel_l2": float(np.linalg.norm(uy - ub) / np.linalg.norm(ub)),
            "sxy_rel_l2": float(np.linalg.norm(sxy - sb) / np.linalg.norm(sb)),
            "sxy_err_over_uy_norm": float(np.linalg.norm(sxy - sb) / np.linalg.norm(ub)),
            "amp_max_err_rel": float(np.max(np.abs(rec["amp"] - o["amp"])) / np.max(np.abs(o["amp"]))),
            "decay_rate_rel_err": float(abs(rate / o["rate"] - 1.0)),
            "decay_rate": rate, "decay_rate_oracle": o["rate"],
        }
    return {"per_quadrature": out, "steps": args.check_steps, "u0": 1e-3, "u1": 0.0,
            "grid": f"{args.n}x{args.n} on the GPU (the benchmark's launch configuration), {args.n}x1 in the "
                    f"FP64 oracle; rows sampled every {max(1, args.n // 64)}",
            "fit": "minus the least-squares slope of ln|A(n)| for t >= min(5 tau, t_end / 4) while |A| >= 1e-4 |A0|"}


def run_gpu(args):
    import torch

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    # the oracle runs that the error check compares with start first, in spawned processes,
    # and overlap the GPU measurement
    check_pool, check_futs = None, {}
    if rank == 0 and args.check_steps > 0:
        quads = [q for q in (args.quad, args.also) if q]
        check_pool = _spawn_pool(len(quads))
        check_futs = {q: check_pool.submit(_oracle_rows_job, q, args.n_eq, args.n, args.kn, 1e-3, args.check_steps,
                                           args.scheme, args.streaming) for q in quads}
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl")
    import __graft_entry__

    __graft_entry__.build()
    import numpy as np

    from paper_0908_4520_gb300 import Lattice, capi

    nx = ny = args.n
    ncell = nx * ny
    results = {}
    sampler = ClockSampler(local)
    main_ms = None
    launches = 0
    for quad in (args.quad, args.also):
        if not quad:
            continue
        L, stream, ev0, ev1, n0 = time_quadrature(torch, Lattice, quad, nx, ny, args.steps, args.warmup, args.kn,
                                                  args.n_eq, args.precision, args.scheme, args.streaming,
                                                  args.step_kernel)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if quad == args.quad:
            sampler.start()
            time.sleep(0.3)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            L.step(args.steps)
            ev1.record(stream)
        torch.cuda.synchronize()
        if quad == args.quad:
            sampler.stop()
        ms = reduce_max_ms(ev0.elapsed_time(ev1), dist, "cuda")
        if quad == args.quad:
            launches = L.launches - n0
        rec = L.diagnostics(4)
        ok = bool(np.all(rec["flags"] == 0))
        info = L.info
        bpc = info["bytes_per_cell_update"]
        per_launch_s = ms / 1e3 / args.steps
        results[quad] = {
            "ms_per_step": ms / args.steps,
            "mlups": weak_value(ncell, world, args.steps, ms),
            "algorithmic_bytes_per_cell": bpc,
            "achieved_gbs": bpc * ncell / per_launch_s / 1e9,
            "finite": ok,
        }
        if quad == args.quad:
            main_ms = ms
            main_L = L
            main_tma = int(info["tma_staged"])
        else:
            L.close()

    # end-to-end through the C-ABI with host buffers: fields in, one record out per step, u_y back
    L = main_L
    e2e = None
    if True:  # every rank: the job's end-to-end time is the slowest rank's
        x = 2 * np.pi * np.arange(nx) / nx
        y = 2 * np.pi * np.arange(ny) / ny
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        uy_h = pin(1e-3 * np.sin(x)[None, :] + 1e-3 * np.sin(y)[:, None] * np.sin(x)[None, :])
        rho_h = pin(np.ones((ny, nx)))
        ux_h = pin(np.zeros((ny, nx)))
        out_h = torch.empty((ny, nx), dtype=torch.float64).pin_memory()
        import ctypes

        dptr = lambda t: ctypes.cast(t.data_ptr(), ctypes.POINTER(ctypes.c_double))
        e2e_steps = args.e2e_steps or args.steps
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        rec = capi.lb_diag()
        t0 = time.perf_counter()
        capi.check(capi.lib.lb_init_fields(L.h, dptr(rho_h), dptr(ux_h), dptr(uy_h), None), L.h)
        # every level's record is read on the host while the next two levels run (a host
        # hiccup shorter than two levels leaves the GPU busy)
        for n in range(1, e2e_steps + 1):
            capi.lb_step(L.h, 1)
            if n >= 2:
                capi.lb_diagnostics_at(L.h, n - 2, rec)
        for n in range(max(0, e2e_steps - 1), e2e_steps + 1):
            capi.lb_diagnostics_at(L.h, n, rec)
        capi.check(capi.lib.lb_moments(L.h, None, None, dptr(out_h), None, None), L.h)
        t1 = time.perf_counter()
        el = reduce_max_ms((t1 - t0) * 1e3, dist, "cuda") / 1e3
        h2d = world * 3 * 8 * ncell / e2e_steps  # all ranks' copies
        d2h = world * (64 * (e2e_steps + 1) + 8 * ncell) / e2e_steps
        e2e = {"value": weak_value(ncell, world, e2e_steps, el * 1e3), "unit": "MLUPS", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": e2e_steps,
               "note": "timed: one solve through the C-ABI: lb_init_fields from pinned host rho/ux/uy, then "
                       "the same number of levels as the device-timed run, every level's diagnostics record "
                       "read on the host (lb_diagnostics_at, while the next two levels run), then the u_y field "
                       "read back; bytes amortised per step"}
    L.close()
    errors = error_vs_oracle(Lattice, args, check_futs) if check_futs else None
    if check_pool:
        check_pool.shutdown()
    dvm = dvm_crosscheck(capi, Lattice, args) if rank == 0 else None

    if dist:
        dist.barrier()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    main = results[args.quad]
    peak, peak_kind = peaks()
    bpc = main["algorithmic_bytes_per_cell"]
    achieved = main["achieved_gbs"]
    traffic = ncu_traffic(args.quad)
    # the oracle on the host cores: at N = 1 only (rank 0), a reported baseline
    cpu = cpu_baseline(args) if not args.no_cpu and world == 1 else None
    line = {
        "metric": METRIC,
        "value": round(main["mlups"], 2),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(main_ms / args.steps, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": args.precision,
        "data": "synthetic (analytic shear-wave initial condition, seeded; no dataset)",
        "config": {"workload": workload_name(args), "quadrature": args.quad, "n_eq": args.n_eq, "nx": nx, "ny": ny,
                   "kn": args.kn, "u0": 1e-3, "u1": 1e-3,
                   "storage": ("f32 deviation f - w rho0" if args.precision == "f32" else
                               f"{args.precision} deviation / power-of-two scale, stochastic rounding"),
                   "diagnostics": "every step (fused)",
                   "l2": "inputs larger than L2: two population buffers of %.2f GB each" % (bpc / 2 * ncell / 1e9),
                   "parallelism": f"independent instance per GPU x{world}"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs", "kernel": kernel_label(args, main_tma),
                     "algorithmic_bytes_per_launch": bpc * ncell},
        "per_quadrature": {q: {k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()}
                           | {"roofline_frac": round(r["achieved_gbs"] / peak, 4)} for q, r in results.items()},
        "e2e": e2e,
        "error_vs_oracle": errors,
        "dvm_crosscheck": dvm,
        "gpu_launches": launches,
        "clocks": sampler.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- oracle (CPU) legs
# Every oracle computation of the bench runs in spawned worker processes (never in the
# process that drives the GPU): the timed CPU baselines, the reference arm, and the
# oracle runs the GPU results are compared with.

def _spawn_ctx():
    import multiprocessing as mp

    return mp.get_context("spawn")


def _spawn_pool(workers):
    import concurrent.futures as cf

    return cf.ProcessPoolExecutor(max_workers=max(1, workers), mp_context=_spawn_ctx())


def _oracle_slab_worker(quad, n_eq, rows, warm, steps, kn, scheme, streaming, barrier, out):
    """One timing process: the oracle on a periodic 4096 x rows slab of the workload (u_y =
    1e-3 sin x + 1e-3 sin y sin x); `warm` levels untimed, then `steps` levels timed as one
    run with a record at every level (one observation pass per level)."""
    import oracle

    oracle.build()
    P = oracle.Problem(quad, n_eq, 4096, rows, kn, scheme=scheme,
                       streaming=streaming if quad.endswith("-GH") else "lax_wendroff")
    f = P.init_shear(1e-3, 1e-3)
    if warm:
        P.run(f, warm, record=True)
    barrier.wait()
    t0 = time.monotonic()
    P.run(f, steps, record=True, n0=warm)
    out.put((t0, time.monotonic()))


def oracle_throughput(quad, n_eq, rows, warm, steps, kn, scheme="second_order", streaming="lax_wendroff",
                      procs=1):
    """MLUPS of `procs` oracle processes, each on its own slab, started together (a
    barrier) and timed from the first start to the last finish (CLOCK_MONOTONIC is
    shared by the processes)."""
    ctx = _spawn_ctx()
    barrier = ctx.Barrier(procs)
    out = ctx.Queue()
    ps = [ctx.Process(target=_oracle_slab_worker, args=(quad, n_eq, rows, warm, steps, kn, scheme, streaming,
                                                        barrier, out)) for _ in range(procs)]
    for p in ps:
        p.start()
    spans = [out.get() for _ in ps]
    for p in ps:
        p.join()
    wall = max(t1 for _, t1 in spans) - min(t0 for t0, _ in spans)
    return procs * 4096 * rows * steps / wall / 1e6, wall


def _oracle_grid_job(quad, n_eq, nx, ny, kn, u0, u1, steps):
    """Wall time of one oracle run of the whole nx x ny grid (a record per level)."""
    import oracle

    oracle.build()
    P = oracle.Problem(quad, n_eq, nx, ny, kn)
    f = P.init_shear(u0, u1)
    t0 = time.monotonic()
    P.run(f, steps, record=True)
    return time.monotonic() - t0


def oracle_grid_mlups(quad, n_eq, nx, ny, kn, u0, u1, steps):
    """Single-thread MLUPS of the oracle on a whole grid, in a spawned process."""
    with _spawn_pool(1) as ex:
        wall = ex.submit(_oracle_grid_job, quad, n_eq, nx, ny, kn, u0, u1, steps).result()
    return nx * ny * steps / wall / 1e6, wall


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(args):
    """The FP64 oracle as it stands on the host cores: one process, and one process per
    core (independent slabs, the oracle itself is single-threaded)."""
    cores = host_cores()
    one, el1 = oracle_throughput(args.quad, args.n_eq, args.cpu_rows, 1, args.cpu_steps, args.kn, args.scheme,
                                 args.streaming, procs=1)
    allc, elc = oracle_throughput(args.quad, args.n_eq, args.cpu_rows, 1, args.cpu_steps, args.kn, args.scheme,
                                  args.streaming, procs=cores)
    # whole grids, one process: the 64 x 1 FP64 correctness case in full (D2Q16-GH, N = 2,
    # Kn 0.1, 5000 levels) and the benchmark's problem on a 256^2 grid for a bounded run
    whole = {}
    v, w = oracle_grid_mlups("D2Q16-GH", 2, 64, 1, 0.1, 1e-3, 0.0, 5000)
    whole["64x1 D2Q16-GH N=2, 5000 levels (in full)"] = {"mlups": round(v, 5), "s": round(w, 2)}
    v, w = oracle_grid_mlups(args.quad, args.n_eq, 256, 256, args.kn, 1e-3, 1e-3, args.cpu_grid_steps)
    whole[f"256x256 {args.quad} N={args.n_eq}, {args.cpu_grid_steps} levels"] = {"mlups": round(v, 5),
                                                                                  "s": round(w, 2)}
    return {"value": round(allc, 5), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, {args.quad} N={args.n_eq}: {cores} processes (one per host core), each on "
                      f"its own periodic 4096x{args.cpu_rows} slab of the workload, {args.cpu_steps} levels "
                      f"with a record per level ({elc:.1f} s)",
            "single_thread": {"value": round(one, 5), "cores": 1,
                              "sample": f"one process, 4096x{args.cpu_rows} slab, {args.cpu_steps} levels "
                                        f"({el1:.1f} s)"},
            "whole_grids": whole}


def _oracle_rows_job(quad, n_eq, nx, kn, u0, steps, scheme="second_order", streaming="lax_wendroff"):
    """The oracle's nx x 1 run of the y-independent wave u_y = u0 sin x (every row of an
    nx x ny lattice started the same way equals it): every level's record, the final u_y and
    sigma_xy, and the decay rate by the oracle's fit rule."""
    import oracle

    oracle.build()
    P = oracle.Problem(quad, n_eq, nx, 1, kn, scheme=scheme,
                       streaming=streaming if quad.endswith("-GH") else "lax_wendroff")
    f = P.init_shear(u0)
    d = P.run(f, steps)
    m = P.moments(f)
    t_fit = min(5.0 * P.tau, d[-1, 0] / 4.0)
    try:
        rate = oracle.decay_fit(d[:, 0], d[:, 4], t_fit)
    except ValueError:
        rate = float("nan")
    return {"t": d[:, 0], "amp": d[:, 4], "uy": m["uy"][0], "sxy": m["sxy"][0], "rate": rate, "t_fit": t_fit}


def run_reference(args):
    """Reference arm: the FP64 oracle (no code of the paper exists to run) on the host cores,
    one process per core, each on a 4096 x ref_rows slab of the workload."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    cores = host_cores()
    value, wall = oracle_throughput(args.quad, args.n_eq, args.ref_rows, args.warmup, args.steps, args.kn,
                                    args.scheme, args.streaming, procs=cores)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "MLUPS", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * wall / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (analytic shear-wave initial condition)",
        "config": {"workload": workload_name(args), "quadrature": args.quad, "n_eq": args.n_eq, "nx": 4096,
                   "ny": args.ref_rows, "kn": args.kn,
                   "note": f"each step: one time level of the oracle in each of {cores} processes (one per host "
                           f"core), each on its own periodic 4096 x {args.ref_rows} slab (a bounded sample of the "
                           "4096^2 workload); the timed levels run as one call with a record per level"},
        "cpu_baseline": {"value": round(value, 5), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} x 4096x{args.ref_rows} slabs, {args.steps} levels after {args.warmup} "
                                   f"untimed ({wall:.1f} s)"},
        "e2e": {"value": round(value, 5), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- other workloads

def _common(args, metric, value, unit, extra):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic"}
    line.update(extra)
    print(json.dumps(line), flush=True)


def run_batch(args):
    """Batching workload: 512 uneven instances, one persistent launch, against the plain
    per-instance method (each instance alone on its own lattice) on a seeded sample."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_0908_4520_gb300 import Batch, Lattice, autotune, inputs

    inst = inputs.batch_instances(args.instances)
    tuned = autotune.tune(inst, "f32")
    stream = torch.cuda.Stream()
    qmap = {"D2Q16-GH": 16, "D2Q36-GH": 36, "D2Q64-GH": 64}
    need = sum(2 * qmap[d["quadrature"]] * d["nx"] * d["ny"] * 4 + 8 * (d["max_steps"] + 2) + 8 * d["nx"] + 1024
               for d in inst)
    b = Batch("f32", budget_bytes=int(need * 1.2) + (64 << 20), threads=tuned["threads"],
              smem_bytes=tuned["smem_bytes"], warp_cells=tuned.get("warp_cells", -1), stream=stream.cuda_stream)
    slots = [b.add(d["quadrature"], d["n_eq"], d["nx"], d["ny"], d["kn"], d["u0"], d["max_steps"], 1e-3)
             for d in inst]
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        b.run(0)
        ev1.record(stream)
    b.sync()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    prof = b.run_profile()
    levels = [b.state(sl)["level"] for sl in slots]
    cells = np.array([d["nx"] * d["ny"] for d in inst], dtype=np.float64)
    q = np.array([qmap[d["quadrature"]] for d in inst], dtype=np.float64)
    updates = float(np.sum(cells * np.array(levels)))
    bytes_alg = float(np.sum(cells * np.array(levels) * 2 * q * 4))
    # the work of the largest 5 % of instances (bytes moved: cells x levels x 2 q x 4)
    work = cells * np.array(levels) * 2 * q * 4
    top = np.sort(work)[::-1][: max(1, len(work) // 20)]
    # plain per-instance method on a seeded sample, scaled by cost
    rng = np.random.default_rng(9084523)
    sample = rng.choice(len(inst), size=min(args.plain_sample, len(inst)), replace=False)
    t_plain, cost_s = 0.0, 0.0
    for i in sample:
        d = inst[i]
        L = Lattice(d["quadrature"], d["n_eq"], d["nx"], d["ny"], d["kn"], stream=stream.cuda_stream)
        L.init_shear_wave(d["u0"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L.step(levels[i] - 1)
        L.synchronize()
        t_plain += time.perf_counter() - t0
        cost_s += cells[i] * levels[i]
        L.close()
    t_plain_total = t_plain * updates / cost_s
    done = sum(b.state(sl)["done"] for sl in slots)
    _common(args, "aggregate MLUPS of 512 uneven shear-wave instances (persistent batched launch)",
            round(updates / (ms / 1e3) / 1e6, 2), "MLUPS", {
                "dtype": "f32", "ms_total": round(ms, 3), "instances": len(inst), "finished": int(done),
                "cell_updates": updates, "algorithmic_bytes": bytes_alg,
                "achieved_gbs": round(bytes_alg / (ms / 1e3) / 1e9, 1),
                "launch_shape": {"threads": tuned["threads"], "smem_bytes": tuned["smem_bytes"],
                                 "warp_cells": tuned.get("warp_cells"), "autotuned": True,
                                 "searched": tuned.get("searched")},
                "tail": {"launch_span_s": round(prof["span_s"], 4), "last_cta_alone_s": round(prof["tail_s"], 4),
                         "tail_share_of_launch": round(prof["tail_s"] / prof["span_s"], 4), "ctas": prof["ctas"],
                         "largest_5pct_instances_share_of_bytes": round(float(top.sum() / work.sum()), 4)},
                "gpu_launches": b.launches,
                "plain_per_instance": {"mlups": round(updates / t_plain_total / 1e6, 2),
                                       "sample": f"{len(sample)} seeded instances alone, same levels, time scaled "
                                                 "by cell updates to all instances",
                                       "est_total_s": round(t_plain_total, 3)},
                "speedup_vs_plain": round(t_plain_total / (ms / 1e3), 2),
                "config": {"workload": "512 instances, nx in 32..1024, ny in {1,4}, D2Q16/36/64-GH, N 2..4, "
                                       "Kn log-uniform 0.01..10, U0 1e-3, stop sqrt(H/H0) <= 1e-3 or 20000 levels",
                           "seed": 9084521}})
    b.close()


def issue_roof(key, mlups):
    """The instruction-issue roofline of a kernel whose warp instructions per cell were counted
    by ncu (profiles/ncu_instructions.json, valid while the kernel sources' code is unchanged):
    every SM issuing 4 warp instructions per cycle at the maximum SM clock."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_instructions.json")) as fh:
            ent = json.load(fh).get(key)
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mhz = float(json.load(fh).get("sm_max_mhz", 2070.0))
    except (OSError, ValueError):
        return None
    if not ent or ent.get("kernel_digest") != kernel_digest():
        return None
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 4 * mhz * 1e6 / ent["warp_instructions_per_cell"] / 1e6
    return {"bound": "alu", "achieved": mlups, "peak": round(peak, 1), "unit": "MLUPS",
            "frac": round(mlups / peak, 4), "warp_instructions_per_cell": round(ent["warp_instructions_per_cell"], 2),
            "peak_source": f"{sms} SMs x 4 warp instructions per cycle x {mhz:.0f} MHz / instructions per cell "
                           f"({ent['profile']})"}


def run_precision(args):
    """Precision workload: D2Q64-GH, N = 4, 2048^2, U0 = 1e-4, 16-bit deviation storage
    (stochastic rounding) and FP32: MLUPS, and every run's error against the FP64 oracle
    (the same y-independent wave on 2048 x 1, every row of the GPU grid equals it): decay
    rate, amplitude history, u_y field; the 16-bit errors against the FP32 run beside them."""
    import numpy as np
    import torch

    from paper_0908_4520_gb300 import inputs

    kns = inputs.precision_kn()[: args.kn_count]
    n = args.n_precision
    steps = args.precision_steps
    # the oracle runs (one per Kn) start first, in spawned processes
    pool = _spawn_pool(min(len(kns), host_cores()))
    futs = [pool.submit(_oracle_rows_job, "D2Q64-GH", 4, n, kn, 1e-4, steps) for kn in kns]

    import __graft_entry__

    __graft_entry__.build()
    from paper_0908_4520_gb300 import Lattice

    out = {}
    stream = torch.cuda.Stream()
    for prec in ("f32", "f16", "bf16"):
        rows = {"ms": [], "rate": [], "amp": [], "uy": []}
        for kn in kns:
            c = inputs.precision_config(kn, prec, nx=n, steps=steps)
            L = Lattice(c["quadrature"], c["n_eq"], n, n, kn, precision=prec, stream=stream.cuda_stream,
                        diag_capacity=steps + 8)
            L.init_shear_wave(c["u0"])
            L.step(args.warmup)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                ev0.record(stream)
                L.step(steps - args.warmup)
                ev1.record(stream)
            torch.cuda.synchronize()
            rows["ms"].append(ev0.elapsed_time(ev1) / (steps - args.warmup))
            rec = L.diagnostics()
            rows["amp"].append(rec["amp"])
            t_fit = min(5.0 * L.info["tau"], rec["t"][-1] / 4.0)
            try:
                rows["rate"].append(L.fit_decay(t_fit)[0])
            except Exception:
                rows["rate"].append(float("nan"))
            rows["uy"].append(L.moments()["uy"][:: max(1, n // 64)])
            bpc = L.info["bytes_per_cell_update"]
            L.close()
        out[prec] = rows | {"bpc": bpc}
    ora = [f.result() for f in futs]
    pool.shutdown()
    peak, _ = peaks()
    u0 = 1e-4
    res = {}
    for prec in ("f32", "f16", "bf16"):
        r = out[prec]
        ms = float(np.median(r["ms"]))
        rate_err = [abs(a / o["rate"] - 1) for a, o in zip(r["rate"], ora)]
        amp_err = [float(np.max(np.abs(a - o["amp"])) / u0) for a, o in zip(r["amp"], ora)]
        uy_err = [float(np.sqrt(np.mean((u - o["uy"][None, :]) ** 2)) / (u0 / np.sqrt(2))) for u, o in zip(r["uy"], ora)]
        res[prec] = {"mlups": round(n * n / (ms / 1e3) / 1e6, 1), "ms_per_step": round(ms, 4),
                     "algorithmic_bytes_per_cell": r["bpc"],
                     "roofline_frac": round(r["bpc"] * n * n / (ms / 1e3) / 1e9 / peak, 4),
                     "decay_rate_rel_err_vs_oracle": [float("%.3g" % e) for e in rate_err],
                     "max_decay_rate_rel_err_vs_oracle": float("%.3g" % max(rate_err)),
                     "max_amp_err_over_u0_vs_oracle": float("%.3g" % max(amp_err)),
                     "max_uy_rms_err_over_initial_rms_vs_oracle": float("%.3g" % max(uy_err))}
        if prec != "f32":
            rel = [abs(a / b - 1) for a, b in zip(r["rate"], out["f32"]["rate"])]
            res[prec]["max_decay_rate_rel_err_vs_f32"] = float("%.3g" % max(rel))
        roof = issue_roof(f"D2Q64-GH/4/{prec}", res[prec]["mlups"])
        if roof:
            res[prec]["roofline_issue"] = roof
    _common(args, "MLUPS of 16-bit deviation storage (D2Q64-GH, N=4) and its errors vs the FP64 oracle",
            res["f16"]["mlups"], "MLUPS", {
                "steps": steps, "warmup": args.warmup,
                "dtype": "f16 storage, f32 arithmetic", "per_precision": res,
                "kn": [round(k, 5) for k in kns],
                "oracle": f"FP64 oracle, D2Q64-GH N=4 on {n}x1 (u_y = 1e-4 sin x does not depend on y), "
                          f"{steps} levels, one spawned process per Kn",
                "config": {"workload": f"shear wave {n}x{n}, D2Q64-GH, N=4, U0=1e-4, {steps} levels (the first "
                                       f"{args.warmup} untimed), Kn log-uniform 0.01..10 (seed 9084520)"}})


def run_driven(args):
    """Driven standing shear wave (Sec. 4): body force g_y = A_f sin(x) cos(phi t), fluid at
    rest at t = 0; amplitude |U|/A_f and phase lag of the periodic response of u_y, and the
    amplitude of the shear stress sigma_xy, for each set and Kn, next to the Navier-Stokes
    and R13 closed forms (Kn = tau, the paper's Eq. KN) and to the driven DVM (Sec. 3.3) on
    the GPU with the 8-point (D2Q64-GH's) and 20-point (D2Q400's) Gauss-Hermite rules."""
    import numpy as np

    import __graft_entry__

    __graft_entry__.build()
    from paper_0908_4520_gb300 import Lattice, capi

    # 128 cells: the Table 1 sets have small lattice speeds (c = 0.36 for D2Q25), so their
    # dt = dx / c is large; at 64 cells their response is still 1.5-2.6 % off at Kn -> 0
    amp, phi, nx = 1e-4, 1.0, 128
    kns = [0.01, 0.05, 0.1, 0.2, 0.5, 1.0, 1.5]
    # the paper's figures (Sec. 4): exm (D2Q9, D2Q16, D2Q400 with N = 1, here the 20-point DVM),
    # normal/lag (D2Q9, D2Q16, D2Q25 of Table 1 with N = 2, 3, 4), diff (expansion orders),
    # three (same quadrature order, different abscissae); plus the benchmark's sets
    figures = {
        ("D2Q9", 2): ["exm", "normal", "lag"], ("D2Q16-int", 2): ["diff"],
        ("D2Q16-int", 3): ["normal", "lag", "diff", "three"], ("D2Q17", 3): ["three"], ("D2Q21", 3): ["three"],
        ("D2Q25", 2): ["diff"], ("D2Q25", 3): ["diff"], ("D2Q25", 4): ["normal", "lag", "diff"],
        ("D2Q16-GH", 1): ["exm"], ("D2Q16-GH", 2): ["exm"], ("D2Q16-GH", 3): ["exm"],
        ("D2Q36-GH", 3): [], ("D2Q64-GH", 4): [], ("D2Q37", 3): [],
    }
    sets = list(figures)
    rows = []
    t_wall = time.perf_counter()
    cell_updates = 0

    def fit(t, y):
        sel = t >= t[-1] - 4 * np.pi / phi
        X = np.stack([np.cos(phi * t[sel]), np.sin(phi * t[sel])], axis=1)
        (a, b), *_ = np.linalg.lstsq(X, y[sel], rcond=None)
        return (a - 1j * b) / amp

    def t_end(kn):
        # the start-up transient decays at least as fast as the shear mode, exp(-kn t)
        return max(10.0 / kn, 30.0)

    dvm = {}
    for nodes in (8, 20):
        dvm_dt = 0.5 * (2 * np.pi / nx) / float(np.max(np.abs(np.polynomial.hermite_e.hermegauss(nodes)[0])))
        for kn in kns:
            nd = int(t_end(kn) / dvm_dt)
            A, S = capi.lb_dvm_run_forced([kn], nodes, nx, 0.0, amp, phi, nd)
            td = dvm_dt * np.arange(nd + 1)
            U, Sg = fit(td, A[0]), fit(td, S[0])
            dvm[(nodes, kn)] = {"amplitude": round(abs(U), 6), "phase_lag": round(float(-np.angle(U)), 6),
                                "shear_amplitude": round(abs(Sg), 6)}
    for quad, N in sets:
        for kn in kns:
            L = Lattice(quad, N, nx, 1, kn, precision="f64", kn_convention="paper", isothermal=True,
                        force_amp=amp, force_freq=phi, diag_capacity=1 << 16)
            L.init_shear_wave(0.0)
            dt = L.info["dt"]
            n = int(t_end(kn) / dt)
            L.step(n)
            rec = L.diagnostics()
            L.close()
            cell_updates += nx * n
            U, Sg = fit(rec["t"], rec["amp"]), fit(rec["t"], rec["shear"])
            ns = 1.0 / (1j * phi + kn)
            i = 1j
            num = 288 * kn**4 * i - 510 * phi * kn**3 + (520 * i - 225 * phi**2 * i) * kn**2 - 375 * phi * kn + 150 * i
            den = (288 * phi * kn**4 + (510 * phi**2 * i - 270 * i) * kn**3 + (745 * phi - 225 * phi**3) * kn**2
                   + (375 * phi**2 * i - 150 * i) * kn + 150 * phi)
            r13 = -num / den
            rows.append({"set": quad, "N": N, "figures": figures[(quad, N)], "kn": kn,
                         "amplitude": round(abs(U), 6),
                         "phase_lag": round(float(-np.angle(U)), 6), "shear_amplitude": round(abs(Sg), 6),
                         "ns": {"amplitude": round(abs(ns), 6), "phase_lag": round(float(-np.angle(ns)), 6)},
                         "r13": {"amplitude": round(abs(r13), 6), "phase_lag": round(float(-np.angle(r13)), 6)},
                         "dvm8": dvm[(8, kn)], "dvm20": dvm[(20, kn)], "levels": n})
    wall = time.perf_counter() - t_wall
    _common(args, "driven standing shear wave: amplitude and phase lag of u_y vs Kn (Sec. 4), LB on the GPU",
            round(cell_updates / wall / 1e6, 3), "MLUPS", {
                "dtype": "f64", "higher_is_better": True, "results": rows,
                "config": {"workload": f"body force A_f sin x cos(phi t), A_f {amp}, phi {phi}, {nx}x1 periodic, "
                                       "fluid at rest at t = 0, isothermal, Kn = tau; response fitted over the "
                                       "last two periods; DVM: cfl 0.5, same grid", "wall_s": round(wall, 2)}})


def run_serve(args):
    """Serving workload: seeded Poisson streams of shear-wave solves (10 % large 1024^2
    D2Q36-GH, FP16 deviation storage) replayed in real time through the request loop,
    against the same streams solved sequentially with the plain per-instance method.

    The specified rate (2000/s) offers far more work than one GPU completes, so it is run
    on a finite prefix of the stream (queue growth shows in the latency); a second stream
    is offered at the rate that would load the sequential plain method to about 80 %."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_0908_4520_gb300 import Lattice, inputs
    from paper_0908_4520_gb300.serve import Server, replay

    def is_large(r):
        return r["nx"] * r["ny"] >= 65536

    def plain_solve(r, levels):
        L = Lattice(r["quadrature"], r["n_eq"], r["nx"], r["ny"], r["kn"], precision="f16",
                    diag_capacity=levels + 2)
        L.init_shear_wave(r["u0"])
        torch.cuda.synchronize()
        t = time.perf_counter()
        L.step(levels - 1)
        L.synchronize()
        el = time.perf_counter() - t
        L.close()
        return el

    # sequential plain method: service time per level (small lattices are launch-bound) and per
    # cell update (large ones are bandwidth-bound), from a seeded sample solved alone at its cap
    prefix = inputs.serving_stream(n=args.requests, rate=args.rate)
    rng = np.random.default_rng(9084524)
    smp = [prefix[i] for i in rng.choice(len(prefix), size=min(args.plain_sample, len(prefix)), replace=False)]
    big = [r for r in smp if is_large(r)][:3]
    small = [r for r in smp if not is_large(r)]
    lv_big, lv_small = 2000, 2000
    t_cell = sum(plain_solve(r, lv_big) for r in big) / max(1, sum(r["nx"] * r["ny"] * lv_big for r in big))
    t_lvl = sum(plain_solve(r, lv_small) for r in small) / max(1, len(small) * lv_small)

    def service(r, levels):
        return t_cell * r["nx"] * r["ny"] * levels if is_large(r) else t_lvl * levels

    def sequential_plain(reqs, levels):
        """The plain per-instance method run for real on the same stream: requests are taken
        one after another in arrival order (waiting for an arrival when idle), each solved on
        its own lattice (create, init, the served number of levels, decay fit, destroy)."""
        lat = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r in reqs:
            now = time.perf_counter() - t0
            if now < r["arrival"]:
                time.sleep(r["arrival"] - now)
            n = levels[r["id"]]
            L = Lattice(r["quadrature"], r["n_eq"], r["nx"], r["ny"], r["kn"], precision="f16",
                        diag_capacity=n + 2)
            L.init_shear_wave(r["u0"])
            L.step(n - 1)
            try:
                L.fit_decay(5.0 * L.info["tau"])
            except Exception:
                pass
            L.close()
            lat.append(time.perf_counter() - t0 - r["arrival"])
        return np.array(lat), time.perf_counter() - t0

    def serve(reqs, measure_plain):
        srv = Server(precision="f16", chunk=args.chunk, budget_bytes=32 << 30, large_budget_bytes=128 << 30,
                     max_large=args.max_large)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        resp = replay(srv, reqs)
        wall = time.perf_counter() - t0
        srv.close()
        lat = np.array([r["finished"] - r["arrival"] for r in resp])
        levels = {r["id"]: r["levels"] for r in resp}
        if measure_plain:
            lat_plain, t_plain = sequential_plain(reqs, levels)
            how = "measured: the same requests solved one after another in real time (plain per-instance method)"
        else:
            # modelled: FIFO over the sampled per-level / per-cell service times
            t_free, lat_plain = 0.0, []
            for r in reqs:
                start = max(t_free, r["arrival"])
                t_free = start + service(r, levels[r["id"]])
                lat_plain.append(t_free - r["arrival"])
            lat_plain, t_plain = np.array(lat_plain), t_free
            how = ("modelled: FIFO of the sampled service times (the offered load is ~10^2 x what one GPU "
                   "completes; running it would take hours)")
        return levels, {"requests": len(reqs), "completed": len(resp), "wall_s": round(wall, 3),
                        "arrival_span_s": round(max(r["arrival"] for r in reqs), 3),
                        "solves_per_s": round(len(resp) / wall, 2),
                        "latency_s": {"p50": round(float(np.percentile(lat, 50)), 4),
                                      "p99": round(float(np.percentile(lat, 99)), 4)},
                        "failed": int(sum(1 for r in resp if r["status"] != 0)),
                        "sequential_plain": {"solves_per_s": round(len(reqs) / t_plain, 2),
                                             "latency_s": {"p50": round(float(np.percentile(lat_plain, 50)), 4),
                                                           "p99": round(float(np.percentile(lat_plain, 99)), 4)},
                                             "how": how}}

    lv, spec = serve(prefix, False)
    # mean plain service demand of the stream (levels as served) -> rate for ~80 % utilisation
    demand = float(np.mean([service(r, lv[r["id"]]) for r in prefix]))
    rate80 = 0.8 / demand
    _, util = serve(inputs.serving_stream(n=args.requests_util, rate=rate80, seed=9084523), True)
    util["rate_per_s"] = round(rate80, 3)
    _common(args, "served shear-wave solves per second with p50/p99 latency (continuous batching)",
            spec["solves_per_s"], "solves/s", {
                "dtype": "f16 storage, f32 arithmetic", "higher_is_better": True,
                "as_specified_prefix": spec, "at_80pct_plain_utilisation": util,
                "plain_service_model": {"s_per_level_small": t_lvl, "s_per_cell_update_large": t_cell,
                                        "sample": f"{len(small)} small and {len(big)} large requests of the "
                                                  f"stream solved alone for 2000 levels each (FP16 storage)",
                                        "mean_demand_s": round(demand, 4)},
                "config": {"workload": f"Poisson stream, first {args.requests} requests at {args.rate}/s (seed "
                                       "9084522), 10% 1024^2 D2Q36-GH N=3, else nx 32..1024 x ny 1/4 "
                                       "D2Q16/36/64-GH, N 2..4; Kn log-uniform 0.01..10, U0 1e-4, stop "
                                       "sqrt(H/H0) <= 1e-3 or 20000 levels; FP16 deviation storage",
                           "chunk": args.chunk, "max_large": args.max_large,
                           "budget_gb": 160, "timing": "wall clock of the real-time replay"}})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quad", default="D2Q36-GH")
    ap.add_argument("--also", default="D2Q37", help="second quadrature measured on the same grid ('' = none)")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--n-eq", type=int, default=3)
    ap.add_argument("--precision", default="f32", choices=["f32", "f64", "f16", "bf16"])
    ap.add_argument("--scheme", default="second_order", choices=["second_order", "first_order"])
    ap.add_argument("--streaming", default="lax_wendroff", choices=["lax_wendroff", "upwind2"])
    ap.add_argument("--kn", type=float, default=0.1)
    ap.add_argument("--e2e-steps", type=int, default=0, help="levels of the end-to-end leg (0: --steps)")
    ap.add_argument("--cpu-rows", type=int, default=48)
    ap.add_argument("--cpu-steps", type=int, default=10)
    ap.add_argument("--cpu-grid-steps", type=int, default=40, help="levels of the oracle's whole 256^2 run")
    ap.add_argument("--ref-rows", type=int, default=16)
    ap.add_argument("--step-kernel", default="auto", choices=["auto", "plain", "tma", "tma_store"],
                    help="step kernel of the timed lattice (auto: the library's choice)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--check-steps", type=int, default=2000,
                    help="levels of the error check against the oracle (0 = no check)")
    ap.add_argument("--workload", default="plain", choices=["plain", "batch", "precision", "serve", "driven"])
    ap.add_argument("--requests", type=int, default=400)
    ap.add_argument("--requests-util", type=int, default=150)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--chunk", type=int, default=200)
    ap.add_argument("--max-large", type=int, default=8)
    ap.add_argument("--instances", type=int, default=512)
    ap.add_argument("--plain-sample", type=int, default=24)
    ap.add_argument("--n-precision", type=int, default=2048)
    ap.add_argument("--precision-steps", type=int, default=2000)
    ap.add_argument("--kn-count", type=int, default=8)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "driven":
        run_driven(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
