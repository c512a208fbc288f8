"""Serving client: the expdg_server_* C-ABI (continuous batching of solves),
a Poisson request stream of 2D Euler vortex solves, and latency statistics.

All solve work runs in libexpdg; this module only submits requests, polls,
fetches results and measures arrival-to-completion latency.
"""

import ctypes
import math
import time

import numpy as np

from . import expdg, inputs


class Server:
    """One expdg_server: `workers` solves in flight, contexts within `hbm_budget` bytes."""

    def __init__(self, workers=8, hbm_budget=0):
        cfg = expdg.expdg_server_config(hbm_budget, workers)
        h = ctypes.c_void_p()
        st = expdg.lib.expdg_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != expdg.EXPDG_OK:
            raise expdg.ExpdgError(st, "expdg_server_create failed")
        self.h = h
        self._shapes = {}

    def close(self):
        if getattr(self, "h", None):
            expdg.lib.expdg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, cfg, q0, dt, nsteps):
        q0 = np.ascontiguousarray(q0, dtype=np.float64)
        rid = ctypes.c_int64(0)
        st = expdg.lib.expdg_server_submit(self.h, ctypes.byref(cfg), q0.ctypes.data, float(dt), int(nsteps),
                                           ctypes.byref(rid))
        if st != expdg.EXPDG_OK:
            raise expdg.ExpdgError(st, "expdg_server_submit failed")
        self._shapes[rid.value] = q0.shape
        return rid.value

    def poll(self, cap=256):
        ids = (ctypes.c_int64 * cap)()
        n = ctypes.c_int(0)
        expdg.lib.expdg_server_poll(self.h, ids, cap, ctypes.byref(n))
        return [ids[i] for i in range(n.value)]

    def fetch(self, rid, check=True):
        """(final state, stats dict, (queueing, service, latency) seconds, status).
        With check=True a failed solve raises ExpdgError."""
        q = np.empty(self._shapes.pop(rid))
        stt = expdg.expdg_stats()
        times = (ctypes.c_double * 3)()
        st = expdg.lib.expdg_server_fetch(self.h, rid, q.ctypes.data, ctypes.byref(stt), times)
        if check and st != expdg.EXPDG_OK:
            raise expdg.ExpdgError(st, f"solve {rid} failed")
        return q, stt.as_dict(), tuple(times), st

    def info(self):
        used = ctypes.c_size_t(0)
        pend = ctypes.c_int(0)
        run = ctypes.c_int(0)
        expdg.lib.expdg_server_info(self.h, ctypes.byref(used), ctypes.byref(pend), ctypes.byref(run))
        return {"used_bytes": used.value, "pending": pend.value, "running": run.value}


def courant_dt(cfg, q, courant):
    """dt = Cr dx_min / c_max with dx_min the smallest LGL node spacing and
    c_max = max |u.n| + a over the nodes (the paper's Courant number, Sec. 5)."""
    gamma = cfg.gamma
    rho = q[0]
    dim = cfg.dim
    u = [q[1 + d] / rho for d in range(dim)]
    p = (gamma - 1.0) * (q[dim + 1] - 0.5 * rho * sum(x * x for x in u))
    a = np.sqrt(gamma * p / rho)
    c = max(float(np.max(np.abs(x) + a)) for x in u)
    # smallest gap between neighbouring nodes along x (uniform mesh, same in every direction)
    X = expdg.config_node_coords(cfg)[0]
    gaps = np.diff(X[0, : cfg.p + 1])
    dx = float(np.min(gaps))
    return courant * dx / c


def vortex_request(rng, prec, courant=5.0, sides=(8, 128), orders=(2, 5), steps=50, iop=0):
    """One request of the serving workload: 2D Euler isentropic vortex on the
    periodic [0,10]^2, side ~ U{8..128} elements, p ~ U{2..5}, strength
    ~ U[1, 5], centre ~ U(domain), free stream (1, 1), EPI2 at Courant 5;
    iop = Krylov orthogonalisation window (0: full)."""
    side = int(rng.integers(sides[0], sides[1] + 1))
    p = int(rng.integers(orders[0], orders[1] + 1))
    strength = float(rng.uniform(1.0, 5.0))
    center = (float(rng.uniform(0, 10)), float(rng.uniform(0, 10)))
    cfg = expdg.default_config(dim=2, p=p, ne=[side, side, 1], lo=[0, 0, 0], hi=[10, 10, 1], eq=expdg.EXPDG_EULER,
                               prec=prec, krylov_tol=1e-8, iop=iop)
    X = expdg.config_node_coords(cfg)
    q0 = inputs.isentropic_vortex(X, 0.0, strength=strength, center=center)
    dt = courant_dt(cfg, q0, courant)
    return cfg, np.ascontiguousarray(q0), dt, steps


def run_stream(server, requests, rate, rng, poll_interval=2e-4, check=True):
    """Submit `requests` [(cfg, q0, dt, nsteps)] with Poisson arrivals of mean
    `rate` per second (rate <= 0: all at once); return per-request results
    (q, stats, times, status) in submission order and the wall time from first
    arrival to last completion.  check=False keeps failed solves as results."""
    n = len(requests)
    gaps = rng.exponential(1.0 / rate, n) if rate > 0 else np.zeros(n)
    arrivals = np.cumsum(gaps) - gaps[0]
    ids = [None] * n
    out = [None] * n
    where = {}
    t0 = time.perf_counter()
    k = 0
    done = 0
    while done < n:
        now = time.perf_counter() - t0
        while k < n and arrivals[k] <= now:
            cfg, q0, dt, steps = requests[k]
            ids[k] = server.submit(cfg, q0, dt, steps)
            where[ids[k]] = k
            k += 1
        for rid in server.poll():
            i = where.pop(rid)
            out[i] = server.fetch(rid, check=check)
            done += 1
        if done < n:
            time.sleep(poll_interval)
    wall = time.perf_counter() - t0
    return out, wall


def latency_summary(results, wall):
    """Throughput and latency over the successful solves (failures counted)."""
    ok = [r for r in results if r[3] == expdg.EXPDG_OK]
    lat = np.array([r[2][2] for r in ok]) if ok else np.array([float("nan")])
    return {"solves": len(ok), "failed": len(results) - len(ok), "wall_s": wall, "solves_per_s": len(ok) / wall,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_queue_ms": 1e3 * float(np.mean([r[2][0] for r in ok])) if ok else None,
            "mean_service_ms": 1e3 * float(np.mean([r[2][1] for r in ok])) if ok else None}
