#!/usr/bin/env python
"""Benchmark: exponential-DG EPI2 steps on the GPU through libexpdg.

Workload (N = 1): 3D compressible Euler (gamma = 1.4) density wave
rho = 1 + 0.2 sin(x + y + z), velocity (1, 1, 1), pressure 1, on the periodic
[0, 2 pi]^3, 32^3 hexahedra, p = 3 LGL (10,485,760 unknowns), Lax-Friedrichs
flux, EPI2 steps of dt = 0.1 with Krylov tolerance 1e-8.  One step = the
linearisation state, one residual, one adaptive augmented-Krylov phi_1 solve
(operator applies, orthogonalisation, phi(H) checks) and the state update.

`value` times the mixed form: FP32 arithmetic for the residual R and the
operator applies L v (FP32 accumulation); FP64 Krylov basis, Arnoldi inner
products and orthogonalisation, phi(H) and state update; incomplete
orthogonalisation over the last 4 basis vectors (the procedure of KIOPS, the
paper's Krylov solver, Sec. 1 and 2.3).  Its error after one step from the
same state is reported against the FP64 form (full orthogonalisation, tol
1e-10; that form matches the CPU oracle to 1e-11 at this size in the GPU
tests) and against the exactly translated wave.  The FP64 form is timed too.
The state (84 MB) and the Krylov vectors exceed the L2 cache; L2 is also
flushed (a 512 MiB write) between timed steps, outside the timed region.

`python bench.py --gpus N --steps K --warmup W [--impl reference]`; for N > 1
launch under torchrun: every rank runs an independent replica of the
workload (the solve has no data-parallel exchange), value = all ranks' units
over the max time.  `--impl reference` times the FP64 CPU oracle on this
host's cores instead (the paper publishes no code), on a bounded sample of
the workload.
"""

import argparse
import hashlib
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
WORKLOAD = ("3D Euler density wave rho=1+0.2sin(x+y+z), u=(1,1,1), p=1, periodic [0,2pi]^3, 32^3 hexes, p=3 LGL, "
            "10,485,760 unknowns, LF flux, EPI2, dt=0.1, Krylov tol 1e-8")
# incomplete orthogonalisation against the latest basis vector only (window 1):
# on this workload the mixed form's FP64 orthogonalisation passes are bound by
# GB300's FP64 pipe, and with window 1 the Krylov dimension hardly grows (37
# steps against 36 with window 2 and 30 with 4) while each step's two passes
# read and multiply one slot instead of two or four: 6.5 ms per step against
# 8.2 (window 2) and 8.8 (window 4), the same error against the FP64 form
CFG = dict(dim=3, p=3, ne=[32, 32, 32], lo=[0.0] * 3, hi=[2 * math.pi] * 3, eq=2, gamma=1.4, scheme=2,
           krylov_tol=1e-8, m_max=64, m_step=5, max_substeps=32, iop=1)
DT = 0.1
# The 2D workload of the paper's vortex experiments (second configuration);
# its vectors stay in L2 and its Arnoldi steps are latency bound.  Window 1
# here too: 29 Krylov steps against 27 with window 4, but 0.78 against 0.90 ms
# per step at the same 1.2e-9 from the FP64 form; the batched and served
# solves use the same window (batched: 0.77 against 0.87-0.95 s).
VORTEX = dict(dim=2, p=4, ne=[64, 64, 1], lo=[0.0, 0.0, 0.0], hi=[10.0, 10.0, 1.0], eq=2, gamma=1.4, scheme=2,
              krylov_tol=1e-8, m_max=64, m_step=5, max_substeps=32, iop=1)
VORTEX_DT = 0.05
# The 1D Burgers solve (192 unknowns, FP64): window 1 as well, 180 against
# 205 us per step through a context and 85.5 against 87.7 us as one resident
# launch, the same 10 Krylov steps and 3e-16 from the oracle.
BURGERS_IOP = 1
CLASSES = ["residual", "jv", "dots", "update", "phi", "combine", "vector"]
# DFMA throughput of this GPU (FP64 FMA per second over all SMs; 1.6 per SM per
# clock at 2070 MHz), measured by the independent-chain throughput probe
# tests/native/alu_rates.cu (tests/test_gpu_alu_rates.py checks it stays so).
FP64_FMA_PER_S = 0.5015e12
# ncu DRAM-traffic records of the dominant kernels, with the hash of the sources
# they were taken from (a record whose sources have changed since is not used)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")
# The CPU oracle's bounded sample of the workload: the same density wave on a
# 16^3 mesh with dt = 0.2 (the same Courant number, the element resolution per
# wavelength halved; with window 1 the oracle's Krylov dimension there is 35,
# the 32^3 workload's 36 on the GPU), one full EPI2 step of 1,310,720 unknowns
# per sample.
SAMPLE_NE, SAMPLE_DT = 16, 0.2
SAMPLE_N = 5 * 64 * SAMPLE_NE ** 3


def max_over_ranks(x, world, device="cpu"):
    """Largest value of x over the ranks (the slowest replica's time)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank, steps, t_max, world):
    """Whole-job throughput of `world` independent replicas: all ranks' units
    over the slowest rank's time (weak scaling: each rank keeps its workload)."""
    return world * units_per_rank * steps / t_max


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def sources_sha(files):
    h = hashlib.sha256()
    for f in sorted(files):
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_record(kernel_class, precision, workload):
    """DRAM bytes per launch of a kernel class from the committed ncu record, or
    None when there is none or its kernel's sources have changed since."""
    try:
        with open(TRAFFIC_FILE) as f:
            recs = json.load(f)
    except Exception:
        return None
    for r in recs.get("records", []):
        if r.get("class") == kernel_class and r.get("precision") == precision and r.get("workload") == workload:
            try:
                if sources_sha(r["sources"]) != r["sources_sha"]:
                    return None
            except Exception:
                return None
            return r
    return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling (every 200 ms) around the timed
    region.  __enter__ returns once the first sample has arrived, so sampling
    is running when the region starts; `extend` keeps the same work running
    after the region until enough samples have been taken."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.rows = []
        self.thread = None

    def _read(self):
        for line in self.proc.stdout:
            if line.count(",") >= 8:
                self.rows.append(line.strip().split(","))

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.time()
        while not self.rows and time.time() - t0 < 10.0 and self.proc.poll() is None:
            time.sleep(0.01)
        return self

    def extend(self, work, min_samples=6, max_s=3.0):
        """Run work() (the timed step, untimed) until min_samples samples exist."""
        t0 = time.time()
        while self.proc is not None and len(self.rows) < min_samples and time.time() - t0 < max_s:
            work()

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.thread is not None:
                self.thread.join(timeout=5)

    def summary(self):
        rows = list(self.rows)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "window": "timed region, then the same steps untimed until 6 samples"}


def host_info():
    """The host the CPU baseline ran on: logical CPUs and the CPU model."""
    import platform
    model = platform.processor() or ""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    arm_parts = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1"}
    return {"nproc": os.cpu_count(), "machine": platform.machine(), "cpu": arm_parts.get(model.lower(), model)}


def rel(a, b):
    import torch
    if isinstance(a, torch.Tensor):
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    a, b = np.asarray(a).reshape(-1), np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ------------------------------------------------------------ CPU oracle ---

def oracle_sample_step():
    """One oracle EPI2 step of the workload's bounded sample (SAMPLE_NE^3,
    dt = SAMPLE_DT, same wave, tol and window): (DOF-steps/s, seconds, m)."""
    from oracle import dg, integrators
    from paper_2011_01316_gb300 import inputs
    ne = SAMPLE_NE
    mesh = dg.Mesh(dim=3, p=3, ne=(ne,) * 3, lo=(0.0,) * 3, hi=(2 * math.pi,) * 3, eq="euler")
    q = inputs.density_wave(dg.node_coords(mesh), 0.0).reshape(-1)
    t0 = time.perf_counter()
    q, st = integrators.step(mesh, q, SAMPLE_DT, tol=CFG["krylov_tol"], m_max=CFG["m_max"], m_step=CFG["m_step"],
                             iop=CFG["iop"])
    t = time.perf_counter() - t0
    return mesh.n_unknowns / t, t, [m for tr in st.traces for (_, m, _) in tr]


SAMPLE_TEXT = (f"one full oracle EPI2 step per sample of the same density wave on a {SAMPLE_NE}^3 mesh "
               f"(1,310,720 unknowns) with dt={SAMPLE_DT} (the workload's Courant number, so about the 32^3 "
               "workload's Krylov dimension), tol 1e-8, window {window}, numpy FP64, single thread")


def oracle_other_rates():
    """Single-thread oracle timings of the other workloads, bounded: the 1D
    Burgers solve (64 elements, p = 2, FP64, tol 1e-10, 50 EPI2 steps of
    dt = 1e-2) in full, and one full EPI2 step of the 2D vortex (64^2, p = 4)."""
    from oracle import dg, integrators
    from paper_2011_01316_gb300 import inputs
    out = {}
    mesh = dg.Mesh(dim=1, p=2, ne=(64,), lo=(0.0,), hi=(2 * math.pi,), eq="burgers")
    q = np.asarray(inputs.burgers_sine(dg.node_coords(mesh)), np.float64).reshape(-1)
    t0 = time.perf_counter()
    for _ in range(50):
        q, _ = integrators.step(mesh, q, 1e-2, tol=1e-10, iop=BURGERS_IOP or None)
    t = time.perf_counter() - t0
    out["burgers1d_64_p2"] = {"us_per_step": 1e6 * t / 50, "dof_steps_per_s": mesh.n_unknowns * 50 / t,
                              "sample": f"50 full EPI2 steps (window {BURGERS_IOP})"}
    mesh = dg.Mesh(dim=2, p=4, ne=(64, 64), lo=(0.0, 0.0), hi=(10.0, 10.0), eq="euler")
    q = inputs.isentropic_vortex(dg.node_coords(mesh), 0.0).reshape(-1)
    t0 = time.perf_counter()
    q, _ = integrators.step(mesh, q, VORTEX_DT, tol=1e-8, iop=VORTEX["iop"] or None)
    t = time.perf_counter() - t0
    out["vortex2d_64_p4"] = {"ms_per_step": 1e3 * t, "dof_steps_per_s": mesh.n_unknowns / t,
                             "sample": f"one full EPI2 step (dt 0.05, tol 1e-8, window {VORTEX['iop']})"}
    return out


def _oracle_solve(job):
    """One bounded oracle solve in a worker process: (unknowns x steps, seconds)."""
    dim, p, ne, hi, eq, q0, dt, steps, iop = job
    from oracle import dg, integrators
    mesh = dg.Mesh(dim=dim, p=p, ne=tuple(ne), lo=(0.0,) * dim, hi=tuple(hi), eq=eq)
    q = np.asarray(q0, np.float64).reshape(-1)
    t0 = time.perf_counter()
    for _ in range(steps):
        q, _ = integrators.step(mesh, q, dt, tol=1e-8, iop=iop)
    return mesh.n_unknowns * steps, time.perf_counter() - t0


def oracle_concurrent(jobs, nproc=None):
    """The oracle on every host core at once: one worker process per core
    (spawned: the parent holds a CUDA context), each taking whole solves from
    `jobs`.  Returns the aggregate DOF-steps/s over the wall time of the pool
    and the worker count."""
    import multiprocessing as mp
    nproc = nproc or os.cpu_count() or 1
    with mp.get_context("spawn").Pool(nproc) as pool:
        pool.map(_oracle_solve, [(1, 1, [4], [1.0], "burgers", np.ones(8), 0.01, 1, 4)] * nproc)  # start-up
        t0 = time.perf_counter()
        out = pool.map(_oracle_solve, jobs, chunksize=1)
        wall = time.perf_counter() - t0
    return sum(u for u, _ in out) / wall, nproc, wall


def _job_of(cfg, q0, dt, steps):
    d = cfg.dim
    return (d, cfg.p, [cfg.ne[k] for k in range(d)], [cfg.hi[k] for k in range(d)],
            "burgers" if cfg.eq == 1 else "euler", q0, dt, steps, cfg.iop or None)


# -------------------------------------------------------------- GPU legs ---

def step_timer(stream, flush):
    import torch

    def timed(c, q, k, dt):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        per, iters = [], []
        for _ in range(k):
            flush.zero_()
            ev0.record(stream)
            st, _ = c.step(q, dt)
            ev1.record(stream)
            ev1.synchronize()
            per.append(ev0.elapsed_time(ev1))
            iters.append(st["krylov_iters"])
        return per, iters
    return timed


def fp64_ops(kclass, prec, bytes_, launches, n_aug):
    """FP64 operations of the incomplete-orthogonalisation passes from their
    algorithmic bytes (per element: FP64 form, window products nwin + 1 for
    (nwin + 1) x 8 bytes, update nwin + 2 for (nwin + 2) x 8; mixed form, window
    products nwin for (nwin + 1/2) x 8 (|w'|^2 in FP32), update nwin for
    (nwin + 2) x 8 (the scale by c_j and the norm in FP32)); None for the
    float-float form."""
    if prec == 2:
        return None
    if prec == 0:
        return bytes_ / 8
    return bytes_ / 8 - launches * n_aug * (0.5 if kclass == "dots" else 2.0)


def kernel_rates(kern, hbm, prec=1, n_aug=None):
    rates = {}
    for k, v in kern.items():
        if v["ms"] > 0 and k in ("residual", "jv", "dots", "update", "combine"):
            gbs = v["bytes"] / (v["ms"] * 1e-3) / 1e9
            rates[k] = {"GB/s": gbs, "frac_of_measured_hbm": gbs / hbm,
                        "us_per_launch": 1e3 * v["ms"] / v["launches"], "launches": v["launches"],
                        "share_of_step": v["ms"] / max(1e-9, sum(x["ms"] for x in kern.values()))}
            if k in ("dots", "update") and n_aug:
                ops = fp64_ops(k, prec, v["bytes"], v["launches"], n_aug)
                if ops is not None:
                    rate = ops / (v["ms"] * 1e-3)
                    rates[k]["fp64_ops_per_s"] = rate
                    rates[k]["frac_of_fp64_pipe"] = rate / FP64_FMA_PER_S
    return rates


def wave3d_form(prec, stream, flush, hbm, steps=3, ne=32, iop=4, ref=None, p=3, tile=0):
    """The workload in one precision form: ms per step (K steps from the same
    state after one warm step), Krylov dimension, per-kernel rates (a second,
    profiled step) and the error of one step against `ref` (a device array)."""
    from paper_2011_01316_gb300 import expdg, inputs
    cfg = {**CFG, "ne": [ne] * 3, "iop": iop, "p": p}
    ctx = expdg.Context(**cfg, prec=prec, tile=tile)
    ctx.set_stream(stream)
    import torch
    q0 = torch.from_numpy(np.ascontiguousarray(inputs.density_wave(ctx.node_coords(), 0.0))).cuda()
    q = q0.clone()
    ctx.step(q, DT)
    err = rel(q, ref) if ref is not None else None
    timed = step_timer(stream, flush)
    q = q0.clone()
    per, iters = timed(ctx, q, steps, DT)
    q = q0.clone()
    ctx.profile_enable(True)
    ctx.step(q, DT)
    kern = ctx.profile_get(reset=True)
    ctx.profile_enable(False)
    n, tile = ctx.n, ctx.tile
    ctx.close()
    ms = float(np.mean(per))
    return {"ms_per_step": ms, "dof_steps_per_s": n / (ms * 1e-3), "krylov_iters_per_step": statistics.mean(iters),
            "jv_tile": {1: "256", 2: "128", 3: "512", 4: "tensor cores 3xTF32", 5: "tensor cores TF32"}.get(tile, "?"),
            "kernels": kernel_rates(kern, hbm, prec, n + 1), "err_vs_fp64_form": err}


def vortex_workload(stream, flush, steps=5):
    """The 2D vortex (64^2, p = 4, 409,600 unknowns: its 3.3 MB vectors stay in
    L2, so launch latency, not HBM, bounds it), EPI2 dt 0.05, tol 1e-8, window
    4, in the mixed and float-float forms, each against the FP64 form (full
    orthogonalisation, tol 1e-10) after one step from the same state."""
    import torch
    from paper_2011_01316_gb300 import expdg, inputs
    ref_ctx = expdg.Context(**{**VORTEX, "iop": 0, "krylov_tol": 1e-10}, prec=expdg.EXPDG_FP64)
    ref_ctx.set_stream(stream)
    q0 = torch.from_numpy(np.ascontiguousarray(inputs.isentropic_vortex(ref_ctx.node_coords(), 0.0))).cuda()
    ref = q0.clone()
    ref_ctx.step(ref, VORTEX_DT)
    ref_ctx.close()
    timed = step_timer(stream, flush)
    out = {"workload": "2D Euler isentropic vortex 64x64, p=4 (409,600 unknowns), EPI2 dt=0.05, tol 1e-8, "
                       f"window {VORTEX['iop']}"}
    for name, prec in (("mixed", expdg.EXPDG_MIXED), ("float_float", expdg.EXPDG_MIXED_FF)):
        ctx = expdg.Context(**VORTEX, prec=prec)
        ctx.set_stream(stream)
        q = q0.clone()
        ctx.step(q, VORTEX_DT)
        err = rel(q, ref)
        for _ in range(3):
            ctx.step(q, VORTEX_DT)
        q = q0.clone()
        per, iters = timed(ctx, q, steps, VORTEX_DT)
        ms = float(np.mean(per))
        out[name] = {"ms_per_step": ms, "dof_steps_per_s": ctx.n / (ms * 1e-3),
                     "krylov_iters_per_step": statistics.mean(iters), "err_vs_fp64_form": err}
        ctx.close()
    return out


def burgers_workload(steps=50, iop=BURGERS_IOP):
    """1D Burgers, 64 elements, p = 2 on the periodic [0, 2 pi] (192
    unknowns), u0 = 0.5 + sin x, LF flux, EPI2 steps of dt = 1e-2 with Krylov
    tol 1e-10, FP64 form: a launch-latency-bound solve.  Reports us per step
    (CUDA events around one expdg_advance of `steps` steps, after 3 warm-up
    steps), DOF-steps/s, and the error after the `steps` steps against the
    oracle's adaptive solve."""
    import torch
    from oracle import dg, integrators
    from paper_2011_01316_gb300 import expdg, inputs
    ctx = expdg.Context(dim=1, p=2, ne=[64, 1, 1], lo=[0.0, 0.0, 0.0], hi=[2 * math.pi, 1.0, 1.0],
                        eq=expdg.EXPDG_BURGERS, scheme=expdg.EXPDG_EPI2, prec=expdg.EXPDG_FP64, krylov_tol=1e-10,
                        m_max=64, m_step=5, max_substeps=32, iop=iop)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream)
    u0 = np.ascontiguousarray(inputs.burgers_sine(ctx.node_coords()))
    q0 = torch.from_numpy(u0).cuda()
    q = q0.clone()
    ctx.advance(q, 1e-2, 3)
    q = q0.clone()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    st = ctx.advance(q, 1e-2, steps)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    mesh = dg.Mesh(dim=1, p=2, ne=(64,), lo=(0.0,), hi=(2 * math.pi,), eq="burgers")
    ref, _ = integrators.advance(mesh, u0.reshape(-1), 1e-2, steps, tol=1e-10, iop=iop or None)
    # the same solve as one resident launch (one CTA, every step inside it;
    # Krylov limit 40, which this solve never reaches: m = 10)
    cfg = expdg.default_config(dim=1, p=2, ne=[64, 1, 1], lo=[0.0, 0.0, 0.0], hi=[2 * math.pi, 1.0, 1.0],
                               eq=expdg.EXPDG_BURGERS, scheme=expdg.EXPDG_EPI2, prec=expdg.EXPDG_FP64,
                               krylov_tol=1e-10, m_max=40, m_step=5, max_substeps=32, iop=iop)
    b = expdg.Batch([cfg])
    qr = q0.clone()
    b.advance([qr], [1e-2], 3)
    qr = q0.clone()
    torch.cuda.synchronize()
    ev0.record(stream)
    st_b = b.advance([qr], [1e-2], steps)
    ev1.record(stream)
    ev1.synchronize()
    ms_r = ev0.elapsed_time(ev1)
    _, rst, _ = b.result(0)
    launches = b.launches()
    b.close()
    ref40, _ = integrators.advance(mesh, u0.reshape(-1), 1e-2, steps, tol=1e-10, m_max=40, iop=iop or None)
    return {"workload": "1D Burgers, 64 elements, p=2, 192 unknowns, u0 = 0.5 + sin x, EPI2 dt=1e-2, tol 1e-10, FP64, "
                        + (f"window {iop} (KIOPS)" if iop else "full orthogonalisation"),
            "steps": steps, "us_per_step": 1e3 * ms / steps, "dof_steps_per_s": ctx.n * steps / (ms * 1e-3),
            "krylov_iters_per_step": st["krylov_iters"] / steps,
            "err_vs_oracle": rel(q.cpu().numpy(), ref), "err_kind": f"oracle, {steps} adaptive steps, same window",
            "resident": {"us_per_step": 1e3 * ms_r / steps, "dof_steps_per_s": ctx.n * steps / (ms_r * 1e-3),
                         "launches": launches, "status": st_b, "krylov_iters_per_step": rst["krylov_iters"] / steps,
                         "err_vs_oracle": rel(qr.cpu().numpy(), ref40),
                         "what": f"expdg_batch_advance: all {steps} steps in one launch of one CTA (FP64)"}}


def exprb32_workload(stream, flush, steps=5):
    """The 2D vortex advanced by EXPRB32 (the paper's third-order scheme,
    Sec. 5.1: two residuals, a stage correction through one operator apply
    and two Krylov solves, the second with phi_3), mixed form, against the
    FP64 form with full orthogonalisation on one step from the same state."""
    import torch
    from paper_2011_01316_gb300 import expdg, inputs
    cfg = {**VORTEX, "scheme": expdg.EXPDG_EXPRB32}
    ctx = expdg.Context(**cfg, prec=expdg.EXPDG_MIXED)
    ctx.set_stream(stream)
    ctx64 = expdg.Context(**{**cfg, "iop": 0, "krylov_tol": 1e-10}, prec=expdg.EXPDG_FP64)
    ctx64.set_stream(stream)
    q0 = torch.from_numpy(np.ascontiguousarray(inputs.isentropic_vortex(ctx.node_coords(), 0.0))).cuda()
    qa, qb = q0.clone(), q0.clone()
    ctx.step(qa, VORTEX_DT)
    ctx64.step(qb, VORTEX_DT)
    err = rel(qa, qb)
    q = q0.clone()
    for _ in range(3):
        ctx.step(q, VORTEX_DT)
    q = q0.clone()
    per, iters = step_timer(stream, flush)(ctx, q, steps, VORTEX_DT)
    ms = float(np.mean(per))
    n = ctx.n
    ctx.close()
    ctx64.close()
    return {"workload": "2D Euler isentropic vortex 64x64, p=4 (409,600 unknowns), EXPRB32, dt=0.05, tol 1e-8, "
                        f"mixed, window {VORTEX['iop']}",
            "ms_per_step": ms, "dof_steps_per_s": n / (ms * 1e-3), "krylov_iters_per_step": statistics.mean(iters),
            "err_vs_fp64_form": err}


def serving_workload(n, seed=1, rate=200.0, workers=8, cpu=False):
    """Poisson stream (mean `rate`/s) of n 2D Euler vortex solves (side 8..128,
    p 2..5, strength U[1,5], centre U(domain), 50 EPI2 steps at Courant 5, tol
    1e-8).  Served: the mixed form, `workers` solves in flight.  Plain: the
    FP64 form, one solve at a time, same requests and the same Krylov window
    (and, for context, with full orthogonalisation).  Reports solves/s,
    p50/p99 arrival-to-completion latency and the largest relative error of a
    served result against the plain FP64 result of the same request."""
    from paper_2011_01316_gb300 import serve
    rng = np.random.default_rng(seed)
    reqs = {"mixed": [], "fp64": [], "fp64_full": []}
    for _ in range(n):
        state = rng.bit_generator.state
        reqs["mixed"].append(serve.vortex_request(rng, 1, iop=VORTEX["iop"]))
        rng.bit_generator.state = state
        reqs["fp64"].append(serve.vortex_request(rng, 0, iop=VORTEX["iop"]))
        rng.bit_generator.state = state
        reqs["fp64_full"].append(serve.vortex_request(rng, 0))
    # warm the kernels of every order once (outside the measured streams)
    warm = serve.Server(workers=1)
    seen = set()
    for r in reqs["mixed"] + reqs["fp64"] + reqs["fp64_full"]:
        key = (r[0].p, r[0].prec, r[0].iop)
        if key not in seen:
            seen.add(key)
            serve.run_stream(warm, [(r[0], r[1], r[2], 1)], 0.0, rng)
    warm.close()
    res, wall = {}, {}
    for name, w in (("mixed", workers), ("fp64", 1), ("fp64_full", 1)):
        if name == "fp64_full" and n > 64:
            continue  # full orthogonalisation one at a time: context for small streams only
        srv = serve.Server(workers=w)
        res[name], wall[name] = serve.run_stream(srv, reqs[name], rate, np.random.default_rng(seed + 1), check=False)
        srv.close()
    both = [(a, b) for a, b in zip(res["mixed"], res["fp64"]) if a[3] == 0 and b[3] == 0]
    err = max((rel(a[0], b[0]) for a, b in both), default=None)
    dofs = sum(r[1].size * r[3] for r, a in zip(reqs["mixed"], res["mixed"]) if a[3] == 0)
    out = {"workload": f"{n} 2D Euler vortex solves, Poisson {rate:g}/s, side 8..128, p 2..5, 50 EPI2 steps, Cr 5",
           "served_mixed": dict(serve.latency_summary(res["mixed"], wall["mixed"]), workers=workers,
                                dof_steps_per_s=dofs / wall["mixed"]),
           "plain_fp64_same_window": dict(serve.latency_summary(res["fp64"], wall["fp64"]), workers=1,
                                          dof_steps_per_s=dofs / wall["fp64"]),
           "max_rel_err_vs_fp64": err,
           "err_kind": "each served result against the plain FP64 form's result of the same request",
           "failed_requests": [{"side": r[0].ne[0], "p": r[0].p, "status_mixed": a[3], "status_fp64": b[3]}
                               for r, a, b in zip(reqs["mixed"], res["mixed"], res["fp64"]) if a[3] != 0 or b[3] != 0]}
    if "fp64_full" in res:
        out["plain_fp64_full_orthogonalisation"] = dict(serve.latency_summary(res["fp64_full"], wall["fp64_full"]),
                                                        workers=1)
    out["speedup_solves_per_s"] = out["served_mixed"]["solves_per_s"] / out["plain_fp64_same_window"]["solves_per_s"]
    if cpu:
        # the oracle on every host core: a seeded sample of 32 of the stream's
        # requests (every request when fewer), 2 of each request's 50 steps
        pick = np.random.default_rng(seed + 7).choice(n, size=min(n, 32), replace=False)
        jobs = [_job_of(reqs["fp64"][i][0], reqs["fp64"][i][1], reqs["fp64"][i][2], 2) for i in pick]
        rate, nproc, wall = oracle_concurrent(jobs)
        per_solve = float(np.mean([reqs["fp64"][i][1].size * 50 for i in range(n)]))
        out["cpu_oracle_all_cores"] = {"dof_steps_per_s": rate, "solves_per_s_equiv": rate / per_solve,
                                       "processes": nproc, "wall_s": wall,
                                       "sample": f"{len(jobs)} seeded requests x 2 of their 50 EPI2 steps, FP64 "
                                                 f"oracle (window {VORTEX['iop']}, tol 1e-8), one process per core at once; "
                                                 "solves/s = DOF-steps/s / mean DOF-steps of a 50-step request"}
    return out


def batched_requests(n, seed, steps, prec):
    from paper_2011_01316_gb300 import expdg, inputs, serve
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        p = int(rng.integers(1, 6))
        if i % 2 == 0:
            ne = int(round(math.exp(rng.uniform(math.log(16), math.log(4096)))))
            cfg = expdg.default_config(dim=1, p=p, ne=[ne, 1, 1], lo=[0, 0, 0], hi=[2 * math.pi, 1, 1],
                                       eq=expdg.EXPDG_BURGERS, prec=prec, krylov_tol=1e-8, iop=VORTEX["iop"])
            X = expdg.config_node_coords(cfg)
            u0, (amp, _) = inputs.fourier_modes(X[0], rng)
            u0 = u0[None]
            umax = float(np.max(np.abs(u0)))
            dx = float(np.min(np.diff(X[0, 0, : p + 1])))
            # smooth until t_shock = 1 / max(-u0'); keep the steps within 0.8 t_shock
            t_shock = 1.0 / max(1e-12, sum((k + 1) * amp[k] for k in range(len(amp))))
            dt = min(5.0 * dx / umax, 0.8 * t_shock / steps)
            reqs.append((cfg, np.ascontiguousarray(u0), dt, steps))
        else:
            side = int(rng.integers(8, 97))
            cfg = expdg.default_config(dim=2, p=p, ne=[side, side, 1], lo=[0, 0, 0], hi=[2 * math.pi] * 2 + [1],
                                       eq=expdg.EXPDG_EULER, prec=prec, krylov_tol=1e-8, iop=VORTEX["iop"])
            X = expdg.config_node_coords(cfg)
            rho, (amp, _) = inputs.fourier_modes(X[0] + X[1], rng)
            if amp.sum() > 0.8:  # keep rho >= 0.2: 1 - sum a_k must stay positive
                rho = 1.0 + (rho - 1.0) * (0.8 / amp.sum())
            q0 = inputs.conservative(rho, [1.0, 1.0], np.ones_like(rho), 1.4)
            reqs.append((cfg, np.ascontiguousarray(q0), serve.courant_dt(cfg, q0, 5.0), steps))
    return reqs


def resident_and_streams(reqs, workers, resident_max):
    """The requests with at most `resident_max` unknowns as one resident batch
    (one launch per class of equal eq, dim, p; Krylov limit 40), the rest
    through the solve server at the same time; returns (results in request
    order as (q, status), wall seconds, resident count, launches)."""
    import threading
    import torch
    from paper_2011_01316_gb300 import expdg, serve
    small = [i for i, r in enumerate(reqs) if r[1].size <= resident_max]
    large = [i for i in range(len(reqs)) if i not in set(small)]
    cfgs = []
    for i in small:
        c = expdg.expdg_config()
        ctypes_copy(c, reqs[i][0])
        c.m_max = min(c.m_max, expdg.BATCH_MAX_KRYLOV)
        cfgs.append(c)
    b = expdg.Batch(cfgs) if small else None
    qs = [torch.from_numpy(reqs[i][1].copy()).cuda() for i in small]
    dts = [reqs[i][2] for i in small]
    if b is not None:  # warm-up (module load), then fresh states
        b.advance([q.clone() for q in qs], dts, 1)
        torch.cuda.synchronize()
    out = [None] * len(reqs)
    box = {}

    def run_small():
        if b is not None:
            box["status"] = b.advance(qs, dts, reqs[small[0]][3])

    srv = serve.Server(workers=workers)
    rng = np.random.default_rng(5)
    t0 = time.perf_counter()
    th = threading.Thread(target=run_small)
    th.start()
    res, _ = serve.run_stream(srv, [reqs[i] for i in large], 0.0, rng, check=False) if large else ([], 0.0)
    th.join()
    wall = time.perf_counter() - t0
    srv.close()
    for k, i in enumerate(large):
        out[i] = (res[k][0], res[k][3])
    for k, i in enumerate(small):
        out[i] = (qs[k].cpu().numpy(), b.result(k)[0])
    launches = b.launches() if b is not None else 0
    if b is not None:
        b.close()
    return out, wall, len(small), launches


def ctypes_copy(dst, src):
    import ctypes
    ctypes.memmove(ctypes.addressof(dst), ctypes.addressof(src), ctypes.sizeof(src))


def batched_workload(n, seed=0, workers=16, steps=20, cpu=False, resident_max=8192):
    """n independent periodic instances (half 1D Burgers with Ne log-uniform in
    [16, 4096], half 2D Euler density waves with side in {8..96}; p uniform in
    {1..5}; initial data 1 + 4 seeded Fourier modes, a_k ~ U[0, 0.3]; dt from
    Courant 5; 20 EPI2 steps; mixed form) run concurrently through the solve
    server, against the same instances run one after another, and every
    result against the FP64 form of the same instance (run concurrently)."""
    from paper_2011_01316_gb300 import serve
    reqs = batched_requests(n, seed, steps, 1)
    rng = np.random.default_rng(seed + 1)
    dofs = sum(r[1].size * r[3] for r in reqs)
    srv = serve.Server(workers=1)
    res1, wall1 = serve.run_stream(srv, reqs, 0.0, rng, check=False)
    srv.close()
    srv = serve.Server(workers=workers)
    resn, walln = serve.run_stream(srv, reqs, 0.0, rng, check=False)
    srv.close()
    same = all(np.array_equal(a[0], b[0]) and a[3] == b[3] for a, b in zip(res1, resn))
    srv = serve.Server(workers=workers)
    res64, _ = serve.run_stream(srv, batched_requests(n, seed, steps, 0), 0.0, rng, check=False)
    srv.close()
    errs = [rel(a[0], b[0]) for a, b in zip(resn, res64) if a[3] == 0 and b[3] == 0]
    resr, wallr, nres, launches = resident_and_streams(reqs, workers, resident_max)
    errs_r = [rel(a[0], b[0]) for a, b in zip(resr, res64) if a[1] == 0 and b[3] == 0]
    cpu_all = None
    if cpu:
        # the oracle on every host core: a seeded sample of 32 instances (half
        # 1D Burgers, half 2D Euler, as the workload), 2 of each one's steps
        r64 = batched_requests(n, seed, steps, 0)
        pick = np.random.default_rng(seed + 7).choice(n, size=min(n, 32), replace=False)
        jobs = [_job_of(r64[i][0], r64[i][1], r64[i][2], 2) for i in pick]
        rate, nproc, wall = oracle_concurrent(jobs)
        cpu_all = {"dof_steps_per_s": rate, "processes": nproc, "wall_s": wall,
                   "sample": f"{len(jobs)} seeded instances x 2 of their {steps} EPI2 steps, FP64 "
                             f"oracle (window {VORTEX['iop']}, tol 1e-8), one process per core at once"}
    return {"workload": f"{n} instances (1D Burgers / 2D Euler, p 1..5, uneven sizes), {steps} EPI2 steps each",
            "cpu_oracle_all_cores": cpu_all,
            "concurrent": {"workers": workers, "wall_s": walln, "dof_steps_per_s": dofs / walln},
            "resident_plus_streams": {"wall_s": wallr, "dof_steps_per_s": dofs / wallr, "resident_instances": nres,
                                      "resident_launches": launches, "streamed_instances": n - nres,
                                      "resident_max_unknowns": resident_max, "failed": sum(1 for a in resr if a[1] != 0),
                                      "max_rel_err_vs_fp64": max(errs_r) if errs_r else None,
                                      "what": "instances with at most resident_max unknowns as one resident batch "
                                              "(one launch per class, one CTA per instance, all steps inside), the "
                                              "rest through the solve server at the same time"},
            "sequential": {"wall_s": wall1, "dof_steps_per_s": dofs / wall1},
            "speedup": wall1 / walln, "identical_results": same,
            "failed": sum(1 for a in resn if a[3] != 0),
            "max_rel_err_vs_fp64": max(errs) if errs else None,
            "err_kind": "each instance's mixed result against the FP64 form of the same instance"}


def k7_workload(stream, flush, hbm, orders=(4, 5, 6, 7, 8), unknowns=5.0e6):
    """The tensor-core trial: the 3D density wave at each order p (about
    `unknowns` unknowns: (unknowns / (5 (p+1)^3))^(1/3) elements per
    direction, dt at the 32^3 p = 3 workload's Courant number), one mixed-form
    EPI2 step (window 2) with the operator's derivative on the FP32 FMA pipes
    (256-thread tile) and on the tensor cores (3xTF32, TF32): microseconds per
    operator apply, Krylov steps and the error against the FP64 form (full
    orthogonalisation, tol 1e-10) after one step from the same state."""
    import torch
    from paper_2011_01316_gb300 import expdg, inputs
    out = []
    for p in orders:
        ne = max(2, int(round((unknowns / (5 * (p + 1) ** 3)) ** (1.0 / 3.0))))
        dt = 0.1 * (32 / ne) * 16.0 / (p + 1) ** 2  # the same dt (p+1)^2 / h as 32^3 p = 3
        cfg = {**CFG, "ne": [ne] * 3, "p": p}
        ref = expdg.Context(**{**cfg, "iop": 0, "krylov_tol": 1e-10}, prec=expdg.EXPDG_FP64)
        ref.set_stream(stream)
        q0 = torch.from_numpy(np.ascontiguousarray(inputs.density_wave(ref.node_coords(), 0.0))).cuda()
        qr = q0.clone()
        ref.step(qr, dt)
        ref.close()
        row = {"p": p, "ne": ne, "unknowns": int(q0.numel()), "dt": dt}
        for name, tile in (("fma", expdg.EXPDG_TILE_256), ("tc_3xtf32", expdg.EXPDG_TILE_TC3),
                           ("tc_tf32", expdg.EXPDG_TILE_TC1)):
            ctx = expdg.Context(**cfg, prec=expdg.EXPDG_MIXED, tile=tile)
            ctx.set_stream(stream)
            q = q0.clone()
            ctx.step(q, dt)
            err = rel(q, qr)
            q = q0.clone()
            ctx.profile_enable(True)
            st, _ = ctx.step(q, dt)
            kern = ctx.profile_get(reset=True)
            ctx.profile_enable(False)
            ctx.close()
            jv = kern["jv"]
            row[name] = {"us_per_jv": 1e3 * jv["ms"] / max(1, jv["launches"]), "krylov_iters": st["krylov_iters"],
                         "err_vs_fp64_form": err, "jv_frac_of_measured_hbm":
                             (jv["bytes"] / max(1, jv["launches"])) / (jv["ms"] / max(1, jv["launches"]) * 1e-3) / 1e9 / hbm}
        out.append(row)
    return {"workload": "3D Euler density wave at p = 4..8, about 5 M unknowns each, mixed form, window 2",
            "orders": out}


def run_reference(args, rank, world):
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample_step()
    times, ms_used = [], []
    for _ in range(args.steps):
        _, t, m = oracle_sample_step()
        times.append(t)
        ms_used += m
    value = len(times) * SAMPLE_N / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "impl": "FP64 CPU oracle (numpy)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": SAMPLE_TEXT.format(window=CFG["iop"]) + f"; Krylov dimensions {sorted(set(ms_used))}"},
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
    ap.add_argument("--serve-requests", type=int, default=48, help="requests of the serving workload (0: skip)")
    ap.add_argument("--serve-workers", type=int, default=8, help="solves in flight in the served form")
    ap.add_argument("--burgers-iop", type=int, default=BURGERS_IOP, help="orthogonalisation window of the Burgers leg (0: full)")
    ap.add_argument("--batch-instances", type=int, default=256, help="instances of the batched workload (0: skip)")
    ap.add_argument("--batch-workers", type=int, default=16, help="instances in flight in the batched workload")
    ap.add_argument("--vortex-iop", type=int, default=VORTEX["iop"],
                    help="orthogonalisation window of the 2D vortex, batched and served workloads")
    ap.add_argument("--resident-max", type=int, default=8192,
                    help="batched workload: instances up to this many unknowns run as one resident batch")
    ap.add_argument("--legs", default="main,wave3d_ff,vortex,burgers,exprb32,serving,batched",
                    help="comma list of legs to run (main = the timed workload; profiling runs pick one)")
    ap.add_argument("--wave3d-ne", type=int, default=32, help="elements per direction of the wave3d legs")
    ap.add_argument("--wave3d-steps", type=int, default=3)
    ap.add_argument("--wave3d-prec", type=int, default=1, help="precision form of a wave3d-only run (1 or 2)")
    ap.add_argument("--wave3d-p", type=int, default=3, help="polynomial order of a wave3d-only run")
    ap.add_argument("--tile", type=int, default=0, help="operator tile class of a wave3d-only run (0: autotuned)")
    ap.add_argument("--iop", type=int, default=CFG["iop"],
                    help="Krylov orthogonalisation window (0: full Arnoldi; k: incomplete, last k vectors)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    CFG["iop"] = args.iop
    VORTEX["iop"] = args.vortex_iop
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

    hbm, peak_kind = peaks()
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    legs = set(args.legs.split(","))
    if "main" not in legs:  # single legs, for profiling runs
        out = {}
        if "wave3d" in legs:
            out["wave3d"] = wave3d_form(args.wave3d_prec, stream, flush, hbm, steps=args.wave3d_steps,
                                        ne=args.wave3d_ne, iop=args.iop, p=args.wave3d_p, tile=args.tile)
        if "vortex" in legs:
            out["vortex"] = vortex_workload(stream, flush)
        if "serving" in legs:
            out["serving"] = serving_workload(args.serve_requests, workers=args.serve_workers,
                                              cpu=not args.no_cpu_baseline)
        if "batched" in legs:
            out["batched"] = batched_workload(args.batch_instances, workers=args.batch_workers,
                                              cpu=not args.no_cpu_baseline, resident_max=args.resident_max)
        if "burgers" in legs:
            out["burgers"] = burgers_workload(iop=args.burgers_iop)
        if "exprb32" in legs:
            out["exprb32"] = exprb32_workload(stream, flush)
        if "k7" in legs:
            out["k7"] = k7_workload(stream, flush, hbm)
        if rank == 0:
            print(json.dumps({"legs": args.legs, **out}), flush=True)
        return

    ctx = expdg.Context(**CFG, prec=expdg.EXPDG_MIXED)
    ctx.set_stream(stream)
    q0 = torch.from_numpy(np.ascontiguousarray(inputs.density_wave(ctx.node_coords(), 0.0))).cuda()
    exact = torch.from_numpy(np.ascontiguousarray(inputs.density_wave(ctx.node_coords(), DT))).cuda()
    N = ctx.n

    # accuracy: one step from the same state against the FP64 form (full
    # orthogonalisation, tol 1e-10) and against the exactly translated wave
    ref_ctx = expdg.Context(**{**CFG, "iop": 0, "krylov_tol": 1e-10}, prec=expdg.EXPDG_FP64)
    ref_ctx.set_stream(stream)
    qref = q0.clone()
    ref_ctx.step(qref, DT)
    ref_ctx.close()
    qa = q0.clone()
    ctx.step(qa, DT)
    err_vs_fp64 = rel(qa, qref)
    err_vs_exact = rel(qa, exact)
    fp64_vs_exact = rel(qref, exact)
    del qa

    timed = step_timer(stream, flush)
    q = q0.clone()
    for _ in range(args.warmup):
        ctx.step(q, DT)
    # timed region: K steps from the initial state, launch counting only
    q = q0.clone()
    ctx.profile_enable(False)
    barrier()
    with ClockSampler(local) as clk:
        per, iters = timed(ctx, q, args.steps, DT)
        barrier()
        launches = sum(v["launches"] for v in ctx.profile_get(reset=True).values())
        qx = q0.clone()
        clk.extend(lambda: (ctx.step(qx, DT), torch.cuda.synchronize()))
    t_local = sum(per) / 1e3
    t_max = max_over_ranks(t_local, world, "cuda")
    value = replica_value(N, args.steps, t_max, world)
    # the same K steps again with a CUDA event pair around every launch
    q = q0.clone()
    ctx.profile_enable(True)
    per_prof, _ = timed(ctx, q, args.steps, DT)
    kern = ctx.profile_get(reset=True)
    ctx.profile_enable(False)

    # roofline of the dominant kernel class over the profiled region
    rates = kernel_rates(kern, hbm, expdg.EXPDG_MIXED, N + 1)
    dom = max(rates, key=lambda k: kern[k]["ms"])
    d = kern[dom]
    achieved = (d["bytes"] / d["launches"]) / (d["ms"] / d["launches"] * 1e-3) / 1e9
    tr = traffic_record(dom, "mixed", "wave3d_32_p3")
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_kind": peak_kind,
                "traffic": tr["dram_bytes_per_launch"] if tr else None, "traffic_unit": "bytes per launch",
                "traffic_source": (tr["capture"] if tr else "no ncu record for the current sources"),
                "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
                "kernel_share": d["ms"] / max(1e-9, sum(v["ms"] for v in kern.values()))}
    if dom in ("dots", "update"):
        roofline["fp64_pipe"] = {"fp64_ops_per_s": rates[dom]["fp64_ops_per_s"], "peak": FP64_FMA_PER_S,
                                 "frac": rates[dom]["frac_of_fp64_pipe"],
                                 "note": ("FP64 operations of the pass (window products and norm in FP64) against the "
                                          "measured DFMA rate")}

    # the FP64 form, same workload and window
    ctx64 = expdg.Context(**CFG, prec=expdg.EXPDG_FP64)
    ctx64.set_stream(stream)
    q = q0.clone()
    ctx64.step(q, DT)
    q = q0.clone()
    per64, it64 = timed(ctx64, q, args.fp64_steps, DT)
    ctx64.close()
    fp64 = {"value": N * len(per64) / (sum(per64) / 1e3), "ms_per_step": sum(per64) / len(per64),
            "steps": len(per64), "krylov_iters_per_step": statistics.mean(it64), "window": CFG["iop"]}

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
    tile = ctx.tile
    ctx.close()

    extra = {}
    if "wave3d_ff" in legs:
        extra["wave3d_float_float"] = wave3d_form(expdg.EXPDG_MIXED_FF, stream, flush, hbm, ref=qref,
                                                  steps=args.wave3d_steps)
    del qref
    if "vortex" in legs:
        extra["vortex"] = vortex_workload(stream, flush)
    if "burgers" in legs:
        extra["burgers"] = burgers_workload(iop=args.burgers_iop)
    if "exprb32" in legs:
        extra["exprb32"] = exprb32_workload(stream, flush)
    cpu_legs = rank == 0 and world == 1 and not args.no_cpu_baseline
    if args.serve_requests > 0 and "serving" in legs:
        extra["serving"] = serving_workload(args.serve_requests, workers=args.serve_workers, cpu=cpu_legs)
    if args.batch_instances > 0 and "batched" in legs:
        extra["batched"] = batched_workload(args.batch_instances, workers=args.batch_workers, cpu=cpu_legs,
                                            resident_max=args.resident_max)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, tt, ms = oracle_sample_step()
        cpu = {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": SAMPLE_TEXT.format(window=CFG["iop"]) + f" ({tt:.1f} s; Krylov dimension {ms})", "host": host_info(),
               "other_workloads": oracle_other_rates()}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD,
                           "precision": ("mixed: Jv in FP32 (FP32 accumulation); R in float-float (48-bit "
                                         "significand) delivered in FP64; FP64 Krylov basis, inner products, "
                                         "orthogonalisation, phi(H) and update"),
                           "krylov": (f"incomplete orthogonalisation, window {CFG['iop']} (KIOPS)" if CFG["iop"]
                                      else "full Arnoldi (DCGS2)"),
                           "l2": "inputs larger than L2 (84 MB state, 84 MB per Krylov vector); also flushed "
                                 "between timed steps (512 MiB write)",
                           "jv_tile": {1: "256", 2: "128", 3: "512"}.get(tile, "?") + " threads per CTA (autotuned)",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "err_vs_fp64": err_vs_fp64,
                "err_kind": ("relative L2 after one step against the FP64 form (full orthogonalisation, tol 1e-10), "
                             "which matches the CPU oracle to 1e-11 at this size in the GPU tests"),
                "err_vs_exact": err_vs_exact, "fp64_form_err_vs_exact": fp64_vs_exact,
                "fp64_form": fp64, "e2e": e2e, "gpu_launches": launches,
                "roofline": roofline, "kernels": kern, "kernel_rates": rates, "cpu_baseline": cpu,
                "clocks": clk.summary(),
                "ms_per_step_min": min(per), "ms_per_step_median": statistics.median(per),
                "krylov_iters_per_step": statistics.mean(iters),
                "jv_per_s": sum(iters) / (sum(per) / 1e3),
                "ms_per_step_profiled": sum(per_prof) / len(per_prof), **extra}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
