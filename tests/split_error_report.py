"""Split-form error per configuration at full size, as numbers.

For each workload the split form (FP32 transport, coupling of Sect. 2.8 with
the FP64 emission residual) runs on the GPU and the FP64 oracle on the same
float-rounded inputs with the same step; the report gives, per field, the
largest per-cell relative error (E and e against themselves, F against E)
and the normwise relative error, after the full step count and after one
step.  Where a workload amplifies perturbations (the hot sphere, the disk),
the oracle's own response to 1e-7 relative perturbations of its inputs
(E, rho, T) is given beside it.

    python tests/split_error_report.py OUT.json [--only NAME ...] [--threads N]

Needs a GPU and takes tens of minutes on the host cores for the 256^3 box.
Writes OUT.json and prints one line per workload.  Not collected by pytest.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from helpers import rounded  # noqa: E402


def field_errors(g, o, ncomp):
    E = o["E"]
    out = {"cell_E": float(np.max(np.abs(g["E"] - E) / np.abs(E))),
           "cell_F": float(max(np.max(np.abs(g["F"][q] - o["F"][q]) / E) for q in range(ncomp))),
           "cell_e": float(np.max(np.abs(g["e"] - o["e"]) / np.abs(o["e"]))),
           "norm_E": float(np.linalg.norm(g["E"] - E) / np.linalg.norm(E)),
           "norm_F": float(np.linalg.norm(g["F"][:ncomp] - o["F"][:ncomp]) / np.linalg.norm(E)),
           "norm_e": float(np.linalg.norm(g["e"] - o["e"]) / np.linalg.norm(o["e"]))}
    return out


def oracle_run(q, nsteps, dt, threads, rtol=None):
    r = q.copy()
    if rtol is not None:
        r.newton_rtol = rtol
    o = oracle.Oracle(r, nthreads=threads)
    o.step(nsteps, dt)
    return {"E": o.E, "F": o.F, "e": o.e}


def spread(q, nsteps, dt, threads, ref, rtol=None):
    """Normwise and per-cell change of the oracle's E after nsteps when E,
    rho and T are perturbed by 1e-7 relative (seeded)."""
    q2 = q.copy()
    rng = np.random.default_rng(0)
    for k in ("E", "rho", "T"):
        a = getattr(q2, k)
        setattr(q2, k, a * (1 + 1e-7 * rng.standard_normal(a.shape)))
    o2 = oracle_run(q2, nsteps, dt, threads, rtol)
    return {"norm_E": float(np.linalg.norm(o2["E"] - ref["E"]) / np.linalg.norm(ref["E"])),
            "cell_E": float(np.max(np.abs(o2["E"] - ref["E"]) / ref["E"]))}


def gpu_run(R, q, nsteps, dt, theta=None, launch=None, **kw):
    r = R.from_problem(q, "split", **kw)
    if theta is not None:
        r.mlp_set(theta)
    if launch == "tune":
        launch = r.tune(2)[:2]
    elif launch is not None:
        r.set_launch(*launch)
    r.step(nsteps, dt)
    st = r.sync()
    out = {k: np.asarray(r.read(k), dtype=np.float64) for k in ("E", "F", "e")}
    out["stats"] = r.stats()
    out["launch"] = r.get_launch()[:2]
    r.close()
    assert st == R.RAD_OK, st
    return out


def report_single(R, name, p, nsteps, threads, theta=None, newton=False, with_spread=False,
                  launch=None):
    t0 = time.time()
    q = rounded(p, np.float32)
    kw = {}
    rtol_gpu, rtol_ref = None, None
    if newton:
        q.implicit_mode = "newton"
        q.newton_rtol = 1e-7
        rtol_ref = 1e-12
        kw = dict(implicit_mode="newton")
        if theta is not None:
            kw.update(use_mlp=1, mlp_gate=1e-2)
    dt = oracle.Oracle(q).dt()
    res = {"workload": p.name, "cells": p.N, "steps": nsteps, "dt": dt,
           "form": ("Newton rtol 1e-7%s" % (" from the learned guess" if theta is not None else ""))
           if newton else "single linearised solve",
           "oracle": "FP64%s" % (", Newton rtol 1e-12" if newton else "")}
    g1 = gpu_run(R, q, 1, dt, theta, launch, **kw)
    res["launch"] = {"variant": int(g1["launch"][0]), "chunk": int(g1["launch"][1])}
    launch = tuple(g1["launch"])
    o1 = oracle_run(q, 1, dt, threads, rtol_ref)
    res["one_step"] = field_errors(g1, o1, p.ncomp)
    g = gpu_run(R, q, nsteps, dt, theta, launch, **kw)
    o = oracle_run(q, nsteps, dt, threads, rtol_ref)
    res["after_steps"] = field_errors(g, o, p.ncomp)
    if with_spread:
        res["oracle_spread_1e-7"] = spread(q, nsteps, dt, threads, o, rtol_ref)
    res["seconds"] = time.time() - t0
    return res


def report_batch(R, threads, theta, nsteps=100):
    t0 = time.time()
    probs = W.batched_2d(64, nsteps=nsteps)
    qs = []
    for p in probs:
        q = rounded(p, np.float32)
        q.implicit_mode = "newton"
        q.newton_rtol = 1e-7
        qs.append(q)
    mem = [R.from_problem(q, "split", implicit_mode="newton", use_mlp=1, mlp_gate=1e-2)
           for q in qs]
    dts = [m.dt() for m in mem]
    b = R.RadBatch(mem)
    b.mlp_set(theta)
    b.step(nsteps)
    assert b.sync() == R.RAD_OK
    worst = {}
    num = {"E": 0.0, "F": 0.0, "e": 0.0}
    den = {"E": 0.0, "e": 0.0}
    for q, m, dt in zip(qs, mem, dts):
        g = {k: np.asarray(m.read(k), dtype=np.float64) for k in ("E", "F", "e")}
        o = oracle_run(q, nsteps, dt, threads, 1e-12)
        e = field_errors(g, o, q.ncomp)
        for k in ("cell_E", "cell_F", "cell_e"):
            worst[k] = max(worst.get(k, 0.0), e[k])
        num["E"] += float(np.sum((g["E"] - o["E"]) ** 2))
        num["F"] += float(np.sum((g["F"][:q.ncomp] - o["F"][:q.ncomp]) ** 2))
        num["e"] += float(np.sum((g["e"] - o["e"]) ** 2))
        den["E"] += float(np.sum(o["E"] ** 2))
        den["e"] += float(np.sum(o["e"] ** 2))
    b.close()
    for m in mem:
        m.close()
    worst.update({"norm_E": (num["E"] / den["E"]) ** 0.5, "norm_F": (num["F"] / den["E"]) ** 0.5,
                  "norm_e": (num["e"] / den["e"]) ** 0.5})
    return {"workload": "batched_2d_64", "grids": len(qs), "cells": int(sum(q.N for q in qs)),
            "steps": nsteps, "form": "batch, Newton rtol 1e-7 from the learned guess, each grid "
            "its own CFL step", "oracle": "FP64, Newton rtol 1e-12, grid by grid",
            "after_steps": worst, "seconds": time.time() - t0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("out")
    ap.add_argument("--only", nargs="*", default=None)
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    import torch
    assert torch.cuda.is_available(), "needs a GPU"
    from paper_2606_26268_b300 import build
    build.build()
    import paper_2606_26268_b300 as R
    import bench
    targs = argparse.Namespace(train_n=512, train_steps=4, train_epochs=4, precision="split")
    theta, _ = bench.train_guess(R, torch, torch.device("cuda", 0), targs)

    jobs = {
        "config1_pulse1d": lambda: report_single(R, "config1", W.pulse_1d(512, 200), 200,
                                                 args.threads),
        "config2_turb2d": lambda: report_single(R, "config2", W.turbulent_2d((1024, 1024)), 100,
                                                args.threads),
        "config2b_turb2d_neq": lambda: report_single(
            R, "config2b", W.turbulent_2d((1024, 1024), nonequilibrium=True), 100, args.threads,
            with_spread=True),
        "config3_hotsphere_headline": lambda: report_single(
            R, "config3", W.hot_sphere_3d(256), 100, args.threads, theta=theta, newton=True,
            with_spread=True, launch="tune"),
        "config4_disk": lambda: report_single(R, "config4", W.disk_spherical(), 50, args.threads,
                                              theta=theta, newton=True, with_spread=True,
                                              launch="tune"),
        "config5_batch": lambda: report_batch(R, args.threads, theta),
    }
    out = {"what": "split form against the FP64 oracle on the same float-rounded inputs",
           "host_threads": oracle.max_threads() if args.threads == 0 else args.threads,
           "date": time.strftime("%Y-%m-%d %H:%M:%S"),
           "kernel_sources_hash": bench.kernel_hash(), "configs": {}}
    if os.path.exists(args.out):
        with open(args.out) as f:
            prev = json.load(f)
        out["configs"].update(prev.get("configs", {}))
    for name, job in jobs.items():
        if args.only and name not in args.only:
            continue
        res = job()
        out["configs"][name] = res
        a = res["after_steps"]
        print("%-28s E %.2e/%.2e  F %.2e/%.2e  e %.2e/%.2e (cell/norm)  %.0fs" % (
            name, a["cell_E"], a["norm_E"], a["cell_F"], a["norm_F"], a["cell_e"], a["norm_e"],
            res["seconds"]), flush=True)
        with open(args.out, "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
