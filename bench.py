#!/usr/bin/env python
"""Benchmark of the M1 radiation step on B300: cell updates per second.

Default workload: the 3D Cartesian hot-sphere box, 256^3 cells, FP32
transport with the FP64 emission term, Kramers-like opacity, chat = 30
(seeded synthetic inputs, see workloads.hot_sphere_3d).  One benchmark step is
one full radiation step (transport + implicit coupling) over all cells.  The
plain FP64 form is timed on the same grid for comparison.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With --gpus N > 1 (launched by
torch.distributed.run) every rank advances its own replica of the grid
(weak scaling, no collective on the data path) and `value` counts the cell
updates of all ranks over the slowest rank's time.  `--impl reference` times
the CPU oracle on the host cores on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "radiation cell updates/s on 1 B300 + % HBM roofline; FP32+MLP vs FP64 plain"
UNIT = "cell updates/s"
# algorithmic bytes per cell update of the fused step (each field read once and
# written once; halos, tables and ghost layers excluded)
BYTES_PER_CELL = {("split", 3): 68, ("fp64", 3): 136, ("split", 2): 52, ("fp64", 2): 104}
PRECISION_DETAIL = {
    "split": "FP32 storage and transport; in the coupling the residual E* - a T^4 of the single "
             "solve within one FP32 rounding of exact (compensated FP32 products), a T^4, the "
             "residual and the numerator of the Newton iterations in FP64, the determinant, its "
             "reciprocal and the increments of T and E in FP32; learned guess: hidden layers "
             "bf16 x bf16 -> FP32 on the tensor cores",
    "fp64": "FP64 throughout"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# sources each profiled kernel is compiled from (a change to any of them
# invalidates its committed ncu figures)
STEP_SOURCES = ("m1_math.cuh", "m1_internal.h", "m1_cell.cuh", "m1_step.cuh", "m1_step_tma.cuh",
                "m1_step_tma2.cuh", "tma.cuh", "step_launch.cuh", "step_tables.cuh", "step_split.cu",
                "step_fp64.cu")
GAS_SOURCES = ("m1_math.cuh", "m1_internal.h", "hydro.cuh", "hydro.cu")


def kernel_hash(sources=STEP_SOURCES):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2606_26268_b300", "csrc")
    for name in sources:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def _sources_of(key):
    return GAS_SOURCES if key.endswith("gas_step") else STEP_SOURCES


def profiled_entry(workload, precision):
    """The committed ncu record of the same kernel source, or None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        key = "%s/%s" % (workload, precision)
        e = d.get(key)
        if e and e.get("kernel_hash") == kernel_hash(_sources_of(key)):
            return e
    except Exception:
        pass
    return None


# thread instructions issued per second at 2032 MHz: 148 SMs x 4 schedulers x
# 32 lanes (one warp instruction per scheduler per clock)
ISSUE_PEAK = 148 * 4 * 32 * 2.032e9


def issue_view(workload, precision, cells, kernel_ms):
    e = profiled_entry(workload, precision)
    if not e or "thread_inst_per_cell" not in e:
        return None
    ipc = float(e["thread_inst_per_cell"])
    achieved = ipc * cells / (kernel_ms * 1e-3)
    return {"inst_per_cell": ipc, "achieved": achieved, "peak": ISSUE_PEAK,
            "unit": "thread-inst/s", "frac": achieved / ISSUE_PEAK,
            "peak_kind": "148 SM x 4 schedulers x 32 lanes x 2032 MHz"}


def profiled_traffic(workload, precision):
    """DRAM bytes per launch from a committed ncu summary of the same kernel
    source (null if the kernel changed since the capture)."""
    e = profiled_entry(workload, precision)
    return float(e["dram_bytes_per_launch"]) if e else None


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 7:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = [n for i, n in enumerate(names) if any(r[3 + i] == "Active" for r in rows)]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][1]) if rows[0][1].replace(".", "").isdigit() else None,
                "samples": len(rows), "reasons": reasons}


def make_workload(name):
    import workloads as W
    if name.startswith("hotsphere3d"):
        n = int(name.split("_")[1]) if "_" in name else 256
        return W.hot_sphere_3d(n)
    if name.startswith("turb2d"):
        n = int(name.split("_")[1]) if "_" in name else 1024
        return W.turbulent_2d((n, n))
    raise SystemExit("unknown workload %s" % name)


def train_guess(R, torch, dev, args):
    """Logs converged Newton solves of the 2D non-equilibrium turbulent box and
    trains the network on them with the library's training kernels."""
    import workloads as W
    t0 = time.perf_counter()
    p = W.turbulent_2d((args.train_n, args.train_n), nonequilibrium=True)
    p.implicit_mode = "newton"
    p.newton_rtol = 1e-12
    r = R.from_problem(p, args.precision, device=dev)
    cap = p.N * args.train_steps
    buf = torch.zeros((cap, 4), dtype=torch.float32, device=dev)
    r.log_bind(buf, stride=1)
    r.step(args.train_steps)
    n = r.log_count()
    loss = r.mlp_train(buf[:n].contiguous(), epochs=args.train_epochs, batch=4096, lr=2e-3, seed=1)
    theta = r.mlp_get()
    r.close()
    return theta, {"records": int(n), "epochs": args.train_epochs, "final_mse": loss,
                   "source": p.name, "seconds": time.perf_counter() - t0}


def time_steps(r, torch, steps, warmup, dt):
    """Device time of `steps` steps (events on the library's stream), after
    `warmup` steps, with synchronisation on both sides; also the per-launch
    kernel times."""
    s = r.stream
    r.step(warmup, dt)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    r.profile_begin(steps)
    with torch.cuda.stream(s):
        ev[0].record(s)
        for k in range(steps):
            r.step(1, dt)
            ev[k + 1].record(s)
    torch.cuda.synchronize()
    kern_ms, queue_ms, n = r.profile_end()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
    return sum(per), per, {"step_kernel_ms": kern_ms / max(n, 1), "queue_pass_ms": queue_ms / max(n, 1)}


def guess_gain_2d(R, torch, dev, args, theta, n=1024, steps=10):
    """The 2D non-equilibrium box (E = (1 + 0.5 g)^4 against T = 1), split,
    Newton rtol 1e-7: its first `steps` steps from the initial state with and
    without the learned guess; device time per step and Newton iterations
    per cell and step."""
    import workloads as W
    p = W.turbulent_2d((n, n), nonequilibrium=True)
    p.newton_rtol = 1e-7
    out = {"workload": p.name, "cells": p.N, "steps": steps,
           "form": "split, Newton rtol 1e-7, the first steps from the initial state"}
    for name, extra in (("with_guess", dict(use_mlp=1, mlp_gate=args.mlp_gate)),
                        ("without_guess", {})):
        r = R.from_problem(p, "split", device=dev, implicit_mode="newton", **extra)
        if extra:
            r.mlp_set(theta)
        r.set_launch(2, 8)
        dt = r.dt()
        ms, per, kt = time_steps(r, torch, steps, 0, dt)
        st = r.stats()
        r.close()
        out[name] = {"ms_per_step": ms / steps, "step_kernel_ms": kt["step_kernel_ms"],
                     "queue_pass_ms": kt["queue_pass_ms"],
                     "iters_per_cell_step": st["iters"] / max(1, st["steps"]) / p.N}
    return out


def split_error_record():
    """The split form's error per configuration, measured at full size by
    tests/split_error_report.py (too long for every bench run) and committed
    with the hash of the step-kernel sources it ran on."""
    path = os.path.join(ROOT, "profiles", "split_error.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    rows = {}
    for k, v in d.get("configs", {}).items():
        a = v["after_steps"]
        row = {"steps": v["steps"], "cell_E": a["cell_E"], "cell_F": a["cell_F"],
               "cell_e": a["cell_e"], "norm_E": a["norm_E"], "norm_F": a["norm_F"],
               "norm_e": a["norm_e"]}
        if "oracle_spread_1e-7" in v:
            row["oracle_spread_1e-7_norm_E"] = v["oracle_spread_1e-7"]["norm_E"]
        rows[k] = row
    return {"source": "profiles/split_error.json (python tests/split_error_report.py)",
            "date": d.get("date"), "current_kernel": d.get("kernel_sources_hash") == kernel_hash(),
            "against": "FP64 oracle on the same float-rounded inputs", "configs": rows}


def link_bandwidth(torch, mb=256, reps=5):
    """Host<->device copy rates of this machine (GB/s): pinned 256 MB copies host
    to device, device to host, and both at once on two streams."""
    n = mb * 1024 * 1024 // 4
    h = torch.empty(n, dtype=torch.float32, pin_memory=True)
    h2 = torch.empty(n, dtype=torch.float32, pin_memory=True)
    d = torch.empty(n, dtype=torch.float32, device="cuda")
    d2 = torch.empty(n, dtype=torch.float32, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def rate(fn, bytes_per_rep):
        fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return reps * bytes_per_rep / (time.perf_counter() - t) / 1e9

    def both():
        with torch.cuda.stream(s1):
            d.copy_(h, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)

    return {"h2d": rate(lambda: d.copy_(h, non_blocking=True), 4 * n),
            "d2h": rate(lambda: h.copy_(d, non_blocking=True), 4 * n),
            "both": rate(both, 8 * n)}


def max_over_ranks(x, world, device):
    """Largest value of x over the ranks (x itself at world size 1)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank, steps, ms_max, world):
    """Cell updates per second of all ranks over the slowest rank's time
    (every rank advances its own replica: weak scaling)."""
    return world * cells_per_rank * steps / (ms_max * 1e-3)


def time_batch(b, torch, steps, warmup):
    """Device time of `steps` batch steps replayed as one captured graph,
    after `warmup` steps (events on the batch's stream)."""
    s = b.stream
    b.step(warmup)
    b.step(steps)          # captures the graph of `steps` steps once
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        e0.record(s)
        b.step(steps)
        e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_batched(args, R, torch, dev, theta, hbm, world=1):
    """64 independent 2D turbulent boxes of uneven sizes (64^2 to 512^2,
    kappa0 scale log-uniform in [1e-2, 1e2]) advanced together: FP32
    transport, Newton coupling from the learned guess, one persistent launch
    per step (plus the queue pass) replayed from a CUDA graph with the tuned
    launch shape; against the plain FP64 loop of one rad_step per grid."""
    import workloads as W
    probs = W.batched_2d(64)
    cells = int(sum(p.N for p in probs))
    rtol = 1e-7
    for p in probs:
        p.newton_rtol = rtol
    extra = dict(use_mlp=1, mlp_gate=args.mlp_gate) if theta is not None else {}
    mem = [R.from_problem(p, "split", device=dev, implicit_mode="newton", **extra) for p in probs]
    b = R.RadBatch(mem)
    if theta is not None:
        b.mlp_set(theta)
    if args.batch_launch:
        v_, c_ = (int(x) for x in args.batch_launch.split(","))
        b.set_launch(v_, c_)
        tuned = (v_, c_, None)
    else:
        tuned = b.tune(3)
    steps = max(args.steps, 10)
    ms_local = time_batch(b, torch, steps, args.warmup)
    ms = max_over_ranks(ms_local, world, dev)
    status = b.sync()
    st = b.stats()
    launch = b.get_launch()
    lps = b.launches_per_step()
    b.close()
    for m in mem:
        m.close()
    # plain FP64 per-grid loop on the same grids
    mem64 = [R.from_problem(p, "fp64", device=dev, implicit_mode="once") for p in probs]
    for m in mem64:
        m.step(1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k64 = 2
    e0.record()
    for _ in range(k64):
        for m in mem64:
            m.step(1)
    e1.record()
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    for m in mem64:
        m.close()
    value = whole_job_rate(cells, steps, ms, world)
    bpc = BYTES_PER_CELL[("split", 2)]
    achieved = bpc * cells / (ms_local / steps * 1e-3) / 1e9
    state_gb = cells * (2 * 6 + 1) * 4 / 1e9
    return {"workload": "batched_2d_64", "grids": len(probs), "cells": cells,
            "sizes": [int(p.n[0]) for p in probs], "value": value, "unit": UNIT,
            "steps": steps, "ms_per_step": ms / steps, "graph": True,
            "launch": {"variant": launch[0], "chunk": launch[1], "ctas": launch[3],
                       "tuned_ms": tuned[2]},
            "form": "split transport, Newton coupling (rtol %g)%s" % (
                rtol, " from the learned guess" if theta is not None else ""),
            "gpu_launches": steps * lps, "status": int(status), "iters": st["iters"],
            "hbm": {"achieved": achieved, "peak": hbm, "frac": achieved / hbm,
                    "bytes_per_cell": bpc},
            "l2": "state %.2f GB (both buffers), above the 126 MB L2" % state_gb,
            "fp64_loop": {"value": cells * k64 / (ms64 * 1e-3), "unit": UNIT,
                          "ms_per_step": ms64 / k64, "launches_per_step": len(probs),
                          "form": "FP64, single linearised solve, one rad_step per grid"}}


def run_ours(args):
    import torch
    import torch.distributed as dist
    import paper_2606_26268_b300 as R
    from paper_2606_26268_b300 import build as B
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if world > 1:
        dist.barrier()

    prob = make_workload(args.workload)
    N = prob.N
    ndim = prob.ndim
    hbm, peak_kind = peaks()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # --- learned guess: trained on solves logged from the 2D non-equilibrium
    # turbulent box (FP32 transport, Newton coupling), before any timing
    theta, train_info = None, None
    if args.form == "mlp":
        theta, train_info = train_guess(R, torch, dev, args)

    # --- headline form -----------------------------------------------------
    implicit = "newton" if args.form in ("mlp", "newton") else args.implicit
    extra = dict(use_mlp=1, mlp_gate=args.mlp_gate) if args.form == "mlp" else {}
    # Newton tolerance: FP64 1e-12; the split form stores T in float, so its
    # iteration stops at the storage precision (same test with and without
    # the learned guess)
    rtol = args.rtol if args.rtol > 0 else (1e-7 if args.precision == "split" else 1e-12)
    prob.newton_rtol = rtol
    r = R.from_problem(prob, args.precision, device=dev, implicit_mode=implicit, **extra)
    if theta is not None:
        r.mlp_set(theta)
    dt = r.dt()
    if args.launch:
        v_, c_ = (int(x) for x in args.launch.split(","))
        r.set_launch(v_, c_)
        tuned = (v_, c_, None)
    else:
        tuned = r.tune(3) if not args.no_tune else r.get_launch()[:2] + (None,)
    barrier()
    with Clocks(local) as clk:
        barrier()
        t0 = time.perf_counter()
        total_ms, per, kt = time_steps(r, torch, args.steps, args.warmup, dt)
        barrier()
        wall = time.perf_counter() - t0
    clocks = clk.summary()
    status = r.sync()
    st = r.stats()
    launches = args.steps * r.launches_per_step()
    ms_max = max_over_ranks(total_ms, world, dev)
    value = whole_job_rate(N, args.steps, ms_max, world)
    # the dominant kernel: the fused step kernel, timed by events around its
    # own launches (the queue pass of the Newton form is reported beside it)
    kernel_ms = kt["step_kernel_ms"]
    bpc = BYTES_PER_CELL[(args.precision, ndim)]
    achieved = bpc * N / (kernel_ms * 1e-3) / 1e9
    r.close()
    del r

    # --- end to end through the C ABI with host buffers --------------------
    e2e = None
    if rank == 0 or True:
        nc = prob.ncomp
        dtype = np.float64 if args.precision == "fp64" else np.float32
        tdt = torch.float64 if dtype == np.float64 else torch.float32

        def pinned(a):
            t_ = torch.empty(a.size, dtype=tdt, pin_memory=True)
            t_.numpy()[:] = a.ravel()
            return t_.numpy()

        h_rho, h_T, h_E = pinned(prob.rho), pinned(prob.T), pinned(prob.E)
        h_v, h_F = pinned(np.asarray(prob.v)[:nc]), pinned(np.asarray(prob.F)[:nc])
        outs = {k: pinned(np.zeros(N * (nc if k in ("F", "m") else 1))) for k in ("E", "F", "e", "m")}
        r2 = R.from_problem(prob, args.precision, device=dev, implicit_mode=implicit, **extra)
        if theta is not None:
            r2.mlp_set(theta)
        r2.set_launch(tuned[0], tuned[1])
        ksteps = max(1, min(args.steps, 8))
        # asynchronous host transfers: the upload of step k + 1 overlaps the
        # read-back of step k (the link carries both directions at once)
        def one_step():
            r2.set_gas_async(h_rho, h_v, h_T)
            r2.set_rad_async(h_E, h_F)
            r2.step(1, dt)
            for k in outs:
                r2.read_async(k, outs[k])

        one_step()
        assert r2.sync() == 0
        barrier()
        t0 = time.perf_counter()
        for _ in range(ksteps):
            one_step()
        st_e2e = r2.sync()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
        assert st_e2e == 0, st_e2e
        isz = np.dtype(dtype).itemsize
        e2e = {"value": whole_job_rate(N, ksteps, e2e_s * 1e3, world), "unit": UNIT,
               "h2d_bytes_per_step": int((3 + 2 * nc) * N * isz),
               "d2h_bytes_per_step": int((2 + 2 * nc) * N * isz), "steps": ksteps,
               "transfers": "rad_set_gas/rad_set_rad/rad_read host_async from pinned memory, "
                            "one rad_sync at the end",
               "link_gbs": link_bandwidth(torch)}
        r2.close()

    # --- comparison forms on the same grid ------------------------------------
    forms = {}
    if not args.skip_forms:
        for name, prec, impl, ex in (("split_newton_no_guess", args.precision, "newton", {}),
                                     ("split_once", args.precision, "once", {})):
            if name == "split_newton_no_guess" and args.form != "mlp":
                continue
            rr = R.from_problem(prob, prec, device=dev, implicit_mode=impl, **ex)
            rr.set_launch(tuned[0], tuned[1])
            ms_, per_, kt_ = time_steps(rr, torch, args.steps, 3, dt)
            st_ = rr.stats()
            rr.close()
            forms[name] = {"value": N * args.steps / (ms_ * 1e-3), "unit": UNIT,
                           "ms_per_step": ms_ / args.steps, "iters": st_["iters"],
                           "iters_per_cell_step": st_["iters"] / max(1, st_["steps"]) / N,
                           "step_kernel_ms": kt_["step_kernel_ms"],
                           "queue_pass_ms": kt_["queue_pass_ms"],
                           "launches_per_step": 2 if impl == "newton" else 1}

    # --- what the learned guess changes: Newton iterations and time per step
    # with and without it, on the headline grid (from the timed runs above)
    # and on the 2D non-equilibrium box (1024^2, its first steps, where the
    # coupling moves T most)
    if not args.skip_forms and args.form == "mlp":
        lg = {"hotsphere": {
            "with_guess": {"ms_per_step": ms_max / args.steps,
                           "step_kernel_ms": kt["step_kernel_ms"],
                           "queue_pass_ms": kt["queue_pass_ms"],
                           "iters_per_cell_step": st["iters"] / max(1, st["steps"]) / N},
            "without_guess": None}}
        if "split_newton_no_guess" in forms:
            f_ = forms["split_newton_no_guess"]
            lg["hotsphere"]["without_guess"] = {
                "ms_per_step": f_["ms_per_step"], "step_kernel_ms": f_["step_kernel_ms"],
                "queue_pass_ms": f_["queue_pass_ms"],
                "iters_per_cell_step": f_["iters_per_cell_step"]}
        lg["turb2d_neq_1024"] = guess_gain_2d(R, torch, dev, args, theta)
        forms["learned_guess"] = lg

    # --- the two-stage (RK2 / IMEX1) step of the paper's runs, headline form
    if not args.skip_forms:
        r2k = R.from_problem(prob, args.precision, device=dev, implicit_mode=implicit,
                             integrator="rk2", **extra)
        if theta is not None:
            r2k.mlp_set(theta)
        r2k.set_launch(tuned[0], tuned[1])
        ms_, per_, kt_ = time_steps(r2k, torch, max(4, args.steps // 2), 3, dt)
        n_ = max(4, args.steps // 2)
        st_ = r2k.stats()
        sr_ = r2k.sync()
        r2k.close()
        forms["rk2"] = {"value": N * n_ / (ms_ * 1e-3), "unit": UNIT, "ms_per_step": ms_ / n_,
                        "steps": n_, "form": args.form + ", two-stage RK2 (each cell updated "
                        "once per step, two transport + coupling passes)",
                        "step_kernel_ms_per_pass": kt_["step_kernel_ms"],
                        "launches_per_step": 2 * (2 if implicit == "newton" else 1) + 1,
                        "iters": st_["iters"], "status": int(sr_)}

    # --- the spherical disk (table opacity) in the headline form ------------
    if not args.skip_forms and not args.skip_disk:
        import workloads as W
        pd = W.disk_spherical()
        pd.newton_rtol = rtol
        rd = R.from_problem(pd, args.precision, device=dev, implicit_mode=implicit, **extra)
        if theta is not None:
            rd.mlp_set(theta)
        if args.disk_launch:
            tv = tuple(int(x) for x in args.disk_launch.split(","))
            rd.set_launch(*tv)
        else:
            tv = rd.tune(2)
        dtd = rd.dt()
        msd, perd, ktd = time_steps(rd, torch, 10, 3, dtd)
        std_ = rd.stats()
        sd = rd.sync()
        rd.close()
        forms["disk_spherical"] = {
            "workload": pd.name, "cells": pd.N, "value": pd.N * 10 / (msd * 1e-3), "unit": UNIT,
            "ms_per_step": msd / 10, "steps": 10, "form": args.form, "iters": std_["iters"],
            "status": int(sd), "launch": {"variant": tv[0], "chunk": tv[1]},
            "hbm_frac": BYTES_PER_CELL[(args.precision, 3)] * pd.N / (ktd["step_kernel_ms"] * 1e-3)
            / 1e9 / hbm}

    # --- the 2D turbulent box (1024^2, periodic), split and plain FP64 ------
    if not args.skip_forms and not args.skip_2d:
        import workloads as W
        p2 = W.turbulent_2d((1024, 1024))
        out2 = {"workload": p2.name, "cells": p2.N, "unit": UNIT,
                "form": "single linearised solve, 1024^2 periodic, E = a T^4 and F = 0 at start",
                "l2": "state 55 MB (split) / 109 MB (FP64) per buffer, inside the 126 MB L2"}
        for prec, n2 in (("split", 50), ("fp64", 10)):
            r2d = R.from_problem(p2, prec, device=dev, implicit_mode="once")
            if prec == "split" and args.launch_2d:
                tv2 = tuple(int(x) for x in args.launch_2d.split(","))
                r2d.set_launch(*tv2)
            else:
                tv2 = r2d.tune(2)
            dt2 = r2d.dt()
            ms2, _, kt2 = time_steps(r2d, torch, n2, 3, dt2)
            st2 = r2d.sync()
            r2d.close()
            out2[prec] = {"value": p2.N * n2 / (ms2 * 1e-3), "ms_per_step": ms2 / n2, "steps": n2,
                          "status": int(st2), "launch": {"variant": tv2[0], "chunk": tv2[1]},
                          "hbm_frac": BYTES_PER_CELL[(prec, 2)] * p2.N
                          / (kt2["step_kernel_ms"] * 1e-3) / 1e9 / hbm}
        forms["turb2d_1024"] = out2

    # --- the paper's performance workload: the 3D pulse with the gas evolved,
    # RK2 (gas step, radiation transport, sources in each stage) ------------
    if not args.skip_forms and not args.skip_rhd:
        import workloads as W
        pr = W.pulse_3d_rhd(args.rhd_n)
        rr = R.from_problem(pr, args.precision, device=dev)
        tvr = rr.tune(2)
        dtr = rr.dt()
        tc = time.perf_counter()
        for _ in range(5):
            rr.dt()  # the gas CFL reduction and its 8-byte read-back
        cfl_ms = (time.perf_counter() - tc) / 5 * 1e3
        nr = 6
        msr, perr, ktr = time_steps(rr, torch, nr, 3, dtr)
        srr = rr.sync()
        rr.close()
        pass_ms = msr / nr / 2
        gas_ms = pass_ms - ktr["step_kernel_ms"] - ktr["queue_pass_ms"]
        gas_bytes = (40 if args.precision != "fp64" else 80) * pr.N
        forms["rhd_pulse3d"] = {
            "workload": pr.name, "cells": pr.N, "value": pr.N * nr / (msr * 1e-3), "unit": UNIT,
            "ms_per_step": msr / nr, "steps": nr,
            "form": "gas step + radiation transport + coupling per stage, two-stage RK2, "
                    "single solve (no absorption), scattering only",
            "radiation_kernel_ms_per_pass": ktr["step_kernel_ms"],
            "gas_step_ms_per_pass": gas_ms,
            "gas_step_roofline": {
                "bound": "hbm", "achieved": gas_bytes / (gas_ms * 1e-3) / 1e9, "peak": hbm,
                "unit": "GB/s", "frac": gas_bytes / (gas_ms * 1e-3) / 1e9 / hbm,
                "bytes_per_cell": gas_bytes // pr.N,
                "traffic": profiled_traffic(pr.name, args.precision + "/gas_step")},
            "launches_per_step": 4, "status": int(srr),
            "cfl_ms": cfl_ms,
            "launch": {"variant": tvr[0], "chunk": tvr[1]},
            "paper": "7.6e8 (MI250X node) and 1.2e9 (MI300 node) cell updates/s for this "
                     "cycle with 256^3 per node; not the same hardware"}

    # --- plain FP64 form on the same grid -----------------------------------
    fp64 = None
    if args.precision != "fp64" and not args.skip_fp64:
        r3 = R.from_problem(prob, "fp64", device=dev, implicit_mode=args.implicit)
        if not args.no_tune:
            r3.tune(1)
        k64 = max(2, args.steps // 4)
        ms64, per64, kt64 = time_steps(r3, torch, k64, 2, dt)
        r3.close()
        ms64 = max_over_ranks(ms64, world, dev)
        b64 = BYTES_PER_CELL[("fp64", ndim)]
        km64 = kt64["step_kernel_ms"]
        fp64 = {"value": whole_job_rate(N, k64, ms64, world), "unit": UNIT,
                "steps": k64, "ms_per_step": ms64 / k64,
                "hbm_frac": b64 * N / (km64 * 1e-3) / 1e9 / hbm}

    # --- batched grids --------------------------------------------------------
    batched = None
    if not args.skip_batch:
        batched = run_batched(args, R, torch, dev, theta, hbm, world)

    # --- CPU baseline: the oracle on the host cores, bounded sample (one
    # process on one GPU only: a multi-rank line carries none) --------------
    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        cpu = cpu_baseline(prob, dt, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.precision == "split" else "f64",
            "data": "synthetic (seeded hot-sphere box: log-normal density, Kramers opacity)",
            "config": {"workload": prob.name, "cells": N, "precision": args.precision,
                       "precision_detail": PRECISION_DETAIL[args.precision],
                       "form": args.form, "implicit": implicit, "chat": prob.chat, "dt": dt,
                       "mlp_gate": args.mlp_gate if args.form == "mlp" else None,
                       "newton_rtol": rtol if implicit == "newton" else None,
                       "guess_training": train_info,
                       "launch": {"variant": tuned[0], "chunk": tuned[1], "tuned_ms": tuned[2]},
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "state larger than L2 (%.2f GB per buffer)" % (
                           (3 + 2 * prob.ncomp) * N * (4 if args.precision == "split" else 8) / 1e9)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "peak_kind": peak_kind,
                         "bytes_per_cell": bpc, "kernel_ms": kernel_ms,
                         "kernel": "fused step kernel (events around its launches)",
                         "queue_pass_ms": kt["queue_pass_ms"], "step_ms": statistics.mean(per),
                         "traffic": profiled_traffic(prob.name, args.precision),
                         # the bound this kernel actually meets: instruction
                         # issue, from the ncu instruction count of the same
                         # source (null if the kernel changed since)
                         "issue": issue_view(prob.name, args.precision, N, kernel_ms)},
            "e2e": e2e,
            "split_error": split_error_record(),
            "cpu_baseline": cpu,
            "fp64_plain": fp64,
            "forms": forms,
            "batched": batched,
            "gpu_launches": launches,
            "clocks": clocks,
            "status": int(status),
            "stats": st,
            "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def cpu_baseline(prob, dt, seconds):
    """The oracle, as it stands, timed on the host cores on a random sample of
    the workload's cells (one step of each sampled cell from the same initial
    state); rate = sampled cell updates per second."""
    import oracle
    o = oracle.Oracle(prob, nthreads=0)
    threads = oracle.max_threads()
    rng = np.random.default_rng(0)
    n = 20000
    cells = rng.choice(prob.N, size=n, replace=False)
    t0 = time.perf_counter()
    o.step_cells(cells, dt)
    t1 = time.perf_counter() - t0
    n2 = int(min(prob.N, max(n, n * seconds / max(t1, 1e-6))))
    cells = rng.choice(prob.N, size=n2, replace=False)
    t0 = time.perf_counter()
    o.step_cells(cells, dt)
    t2 = time.perf_counter() - t0
    # the same oracle on one host thread, on a tenth of the sample
    o1 = oracle.Oracle(prob, nthreads=1)
    n1 = max(1000, n2 // 10)
    c1 = rng.choice(prob.N, size=n1, replace=False)
    t0 = time.perf_counter()
    o1.step_cells(c1, dt)
    t3 = time.perf_counter() - t0
    return {"value": n2 / t2, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d random cells of %s, one step each from the initial state "
                      "(%.1f s)" % (n2, prob.name, t2),
            "one_thread": {"value": n1 / t3, "cores": 1, "cells": n1}}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    prob = make_workload(args.workload)
    o = oracle.Oracle(prob, nthreads=0)
    dt = o.dt()
    rng = np.random.default_rng(1)
    sample = int(min(prob.N, args.ref_cells))
    cells = rng.choice(prob.N, size=sample, replace=False)
    for _ in range(args.warmup):
        o.step_cells(cells[: max(1, sample // 10)], dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step_cells(cells, dt)
    el = time.perf_counter() - t0
    value = sample * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": prob.name, "cells": prob.N, "precision": "fp64 (oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(),
                             "kind": "oracle",
                             "sample": "%d random cells per step of %s" % (sample, prob.name)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hotsphere3d_256")
    ap.add_argument("--precision", default="split", choices=["split", "fp64"])
    ap.add_argument("--implicit", default="once", choices=["once", "newton"])
    ap.add_argument("--form", default="mlp", choices=["mlp", "newton", "once"],
                    help="mlp: FP32 transport + Newton coupling from the learned guess")
    ap.add_argument("--mlp-gate", type=float, default=1e-2)
    ap.add_argument("--rtol", type=float, default=0.0, help="Newton tolerance (0: by precision)")
    ap.add_argument("--train-n", type=int, default=512)
    ap.add_argument("--train-steps", type=int, default=4)
    ap.add_argument("--train-epochs", type=int, default=4)
    ap.add_argument("--skip-forms", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-cells", type=int, default=200000)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--skip-batch", action="store_true")
    ap.add_argument("--skip-disk", action="store_true")
    ap.add_argument("--skip-rhd", action="store_true")
    ap.add_argument("--skip-2d", action="store_true")
    ap.add_argument("--rhd-n", type=int, default=256, help="RHD pulse grid (n^3)")
    ap.add_argument("--launch", default="", help="variant,chunk (skips the autotuner)")
    ap.add_argument("--batch-launch", default="",
                    help="variant,chunk of the batched form (skips its autotuner)")
    ap.add_argument("--disk-launch", default="",
                    help="variant,chunk of the spherical disk form (skips its autotuner)")
    ap.add_argument("--2d-launch", dest="launch_2d", default="",
                    help="variant,chunk of the split 2D box form (skips its autotuner)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
