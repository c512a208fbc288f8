#!/usr/bin/env python
"""Benchmark: exponential-DG EPI2 steps on the GPU through libexpdg.

Workload (N = 1): 2D compressible Euler (gamma = 1.4) isentropic vortex
(strength 5, decay 1, free stream (1, 1), centre (5, 5)) on the periodic
[0,10]^2, 64 x 64 quadrilaterals, p = 4 LGL (409,600 unknowns), Lax-Friedrichs
flux, EPI2 steps of dt = 0.05 with Krylov tolerance 1e-10.  One step = one
residual, one adaptive augmented-Krylov phi_1 solve (Jv applies, Gram-Schmidt,
phi(H) checks) and the state update.

`value` times the mixed form (FP32 R/Jv, float-float Krylov basis and
orthogonalisation, FP64 phi(H) and FP64 state update), the production form;
its relative L2 error against the FP64 form after one step from the same state
is reported as `err_vs_fp64`.  The FP64 form is timed too (`fp64_form`).
L2 is flushed (a 512 MiB write) between timed steps, outside the timed region.

`python bench.py --gpus N --steps K --warmup W [--impl reference]`; for N > 1
launch under torchrun: every rank runs an independent replica of the
workload (the solve has no data-parallel exchange), value = all ranks' units
over the max time.  `--impl reference` times the FP64 CPU oracle on this
host's cores instead (the paper publishes no code).
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-steps/s"
UNIT = "DOF-steps/s"
WORKLOAD = ("2D Euler isentropic vortex, periodic [0,10]^2, 64x64 quads, p=4 LGL, 409,600 unknowns, "
            "LF flux, EPI2, dt=0.05, Krylov tol 1e-10")
CFG = dict(dim=2, p=4, ne=[64, 64, 1], lo=[0.0, 0.0, 0.0], hi=[10.0, 10.0, 1.0], eq=2, gamma=1.4,
           scheme=2, krylov_tol=1e-10, m_max=64, m_step=5, max_substeps=32)
DT = 0.05
CLASSES = ["residual", "jv", "dots", "update", "phi", "combine", "vector"]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_step_rate(steps=1):
    """FP64 CPU oracle: DOF-steps/s over `steps` EPI2 steps of the workload."""
    from oracle import dg, integrators
    from paper_2011_01316_gb300 import inputs
    mesh = dg.Mesh(dim=2, p=4, ne=(64, 64), lo=(0.0, 0.0), hi=(10.0, 10.0), eq="euler")
    q = inputs.isentropic_vortex(dg.node_coords(mesh), 0.0).reshape(-1)
    t0 = time.perf_counter()
    for _ in range(steps):
        q, _ = integrators.step(mesh, q, DT, tol=CFG["krylov_tol"], m_max=CFG["m_max"], m_step=CFG["m_step"])
    dt = time.perf_counter() - t0
    return mesh.n_unknowns * steps / dt, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_step_rate(1)
    rates, times = [], []
    for _ in range(args.steps):
        r, t = oracle_step_rate(1)
        rates.append(r)
        times.append(t)
    value = len(times) * 409600 / sum(times)
    sample = f"{args.steps} full EPI2 steps of the workload (409,600 unknowns each), single thread"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "impl": "FP64 CPU oracle (numpy)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="expdg", choices=["expdg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=3)
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2011_01316_gb300 import expdg, inputs

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    ctx = expdg.Context(**CFG, prec=expdg.EXPDG_MIXED)
    ctx.set_stream(stream)
    ctx64 = expdg.Context(**CFG, prec=expdg.EXPDG_FP64)
    ctx64.set_stream(stream)
    q0 = torch.from_numpy(np.ascontiguousarray(inputs.isentropic_vortex(ctx.node_coords(), 0.0))).cuda()
    N = ctx.n
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # accuracy of the mixed form against the FP64 form, one step from the same state
    qa = q0.clone()
    qb = q0.clone()
    ctx.step(qa, DT)
    ctx64.step(qb, DT)
    err_vs_fp64 = float(torch.linalg.vector_norm(qa - qb) / torch.linalg.vector_norm(qb))

    def timed(c, q, k):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        per, iters = [], []
        for _ in range(k):
            flush.zero_()
            ev0.record(stream)
            st, _ = c.step(q, DT)
            ev1.record(stream)
            ev1.synchronize()
            per.append(ev0.elapsed_time(ev1))
            iters.append(st["krylov_iters"])
        return per, iters

    q = q0.clone()
    for _ in range(args.warmup):
        ctx.step(q, DT)
    # timed region: K steps from the initial state, launch counting only
    q = q0.clone()
    ctx.profile_enable(False)
    barrier()
    with ClockSampler(local) as clk:
        per, iters = timed(ctx, q, args.steps)
        barrier()
    launches = sum(v["launches"] for v in ctx.profile_get(reset=True).values())
    t_local = sum(per) / 1e3
    t = torch.tensor([t_local], device="cuda", dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    value = world * N * args.steps / t_max
    # the same K steps again with a CUDA event pair around every launch
    q = q0.clone()
    ctx.profile_enable(True)
    per_prof, _ = timed(ctx, q, args.steps)
    kern = ctx.profile_get(reset=True)
    ctx.profile_enable(False)

    # per-kernel-class profile over the timed region
    hbm, peak_kind = peaks()
    bw = {k: v for k, v in kern.items() if k in ("jv", "dots", "update", "residual", "combine")}
    dom = max(bw, key=lambda k: bw[k]["ms"])
    d = kern[dom]
    achieved = (d["bytes"] / d["launches"]) / (d["ms"] / d["launches"] * 1e-3) / 1e9 if d["ms"] > 0 else 0.0
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": None, "peak_kind": peak_kind,
                "kernel_share": d["ms"] / max(1e-9, sum(v["ms"] for v in kern.values()))}

    # FP64 form, same workload
    q = q0.clone()
    ctx64.step(q, DT)
    per64, it64 = timed(ctx64, q, args.fp64_steps)
    fp64 = {"value": N * len(per64) / (sum(per64) / 1e3), "ms_per_step": sum(per64) / len(per64),
            "steps": len(per64), "krylov_iters_per_step": statistics.mean(it64)}

    # end to end through the C-ABI with pinned host buffers (copies inside the call)
    qh = torch.empty(q0.shape, dtype=torch.float64, pin_memory=True)
    qh.copy_(q0.cpu())
    ctx.step(qh, DT)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.step(qh, DT)
    barrier()
    te = time.perf_counter() - t0
    e2e = {"value": world * N * args.steps / te, "unit": UNIT, "h2d_bytes_per_step": 8 * N,
           "d2h_bytes_per_step": 8 * N}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, tt = oracle_step_rate(1)
        cpu = {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one full EPI2 step of the workload ({tt:.1f} s, single thread, numpy FP64)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+ff(48-bit)+f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "precision": "mixed: FP32 R/Jv, float-float Krylov, FP64 phi(H)",
                           "l2": "flushed between timed steps (512 MiB write)",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "err_vs_fp64": err_vs_fp64, "fp64_form": fp64, "e2e": e2e, "gpu_launches": launches,
                "roofline": roofline, "kernels": kern, "cpu_baseline": cpu, "clocks": clk.summary(),
                "ms_per_step_min": min(per), "ms_per_step_median": statistics.median(per),
                "krylov_iters_per_step": statistics.mean(iters),
                "ms_per_step_profiled": sum(per_prof) / len(per_prof)}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
