"""The solve server (continuous batching) on the GPU: every result is the
same alone and in a concurrent mix of differently sized Burgers and Euler
solves, admission respects the device-memory budget, and oversize requests
are refused."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_01316_gb300 import expdg, inputs, serve
    return expdg, inputs, serve


def _requests(expdg, inputs, serve, n, seed, prec):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        if i % 3 == 0:
            ne = int(rng.integers(16, 200))
            p = int(rng.integers(1, 6))
            cfg = expdg.default_config(dim=1, p=p, ne=[ne, 1, 1], lo=[0, 0, 0], hi=[2 * math.pi, 1, 1],
                                       eq=expdg.EXPDG_BURGERS, prec=prec, krylov_tol=1e-8)
            X = expdg.config_node_coords(cfg)
            q0 = inputs.fourier_modes(X[0], rng, mean=1.0)[0][None]
            reqs.append((cfg, np.ascontiguousarray(q0), 0.2 * (2 * math.pi / ne) / p, 3))
        else:
            cfg, q0, dt, _ = serve.vortex_request(rng, prec, sides=(8, 40), orders=(2, 5))
            reqs.append((cfg, q0, dt, 3))
    return reqs


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_same_result_alone_and_in_the_mix(mods, prec):
    expdg, inputs, serve = mods
    reqs = _requests(expdg, inputs, serve, 12, 3 + prec, prec)
    alone = []
    s1 = serve.Server(workers=1)
    for r in reqs:
        res, wall = serve.run_stream(s1, [r], 0.0, np.random.default_rng(0))
        alone.append(res[0][0])
    s1.close()
    s8 = serve.Server(workers=6)
    mix, wall = serve.run_stream(s8, reqs, 0.0, np.random.default_rng(0))
    info = s8.info()
    s8.close()
    for (q_mix, st, times, status), q_alone in zip(mix, alone):
        # deterministic kernels and reductions: identical bits alone and in the mix
        np.testing.assert_array_equal(q_mix, q_alone)
        assert times[2] >= times[1] > 0.0
    assert info["pending"] == 0 and info["running"] == 0


def test_fresh_contexts_under_concurrency(mods):
    """Many fresh contexts created and run at once on non-blocking worker
    streams (as under load): every result equals its single-stream result."""
    expdg, inputs, serve = mods
    rng = np.random.default_rng(5)
    reqs = [serve.vortex_request(rng, 1, sides=(20, 90), orders=(2, 5), steps=3) for _ in range(16)]
    s = serve.Server(workers=8)
    mix, _ = serve.run_stream(s, reqs, 0.0, rng)
    s.close()
    for (cfg, q0, dt, n), (q_mix, st, times, status) in zip(reqs, mix):
        ctx = expdg.Context(cfg)
        q = q0.copy()
        ctx.advance(q, dt, n)
        ctx.close()
        np.testing.assert_array_equal(q_mix, q)


def test_budget_admission_and_refusal(mods):
    expdg, inputs, serve = mods
    reqs = _requests(expdg, inputs, serve, 6, 11, 1)
    biggest = max(expdg.context_bytes(r[0]) for r in reqs)
    s = serve.Server(workers=4, hbm_budget=biggest)  # at most one context resident
    res, wall = serve.run_stream(s, reqs, 0.0, np.random.default_rng(0))
    assert s.info()["used_bytes"] <= biggest
    s.close()
    s2 = serve.Server(workers=2)
    ref, _ = serve.run_stream(s2, reqs, 0.0, np.random.default_rng(0))
    s2.close()
    for a, b in zip(res, ref):
        np.testing.assert_array_equal(a[0], b[0])
    tiny = serve.Server(workers=1, hbm_budget=biggest // 4)
    with pytest.raises(expdg.ExpdgError) as ei:
        tiny.submit(*reqs[[expdg.context_bytes(r[0]) for r in reqs].index(biggest)])
    assert ei.value.status == expdg.EXPDG_ENOMEM
    tiny.close()


def test_server_matches_context_advance(mods):
    expdg, inputs, serve = mods
    rng = np.random.default_rng(21)
    cfg, q0, dt, _ = serve.vortex_request(rng, 1, sides=(16, 16), orders=(3, 3))
    s = serve.Server(workers=2)
    res, _ = serve.run_stream(s, [(cfg, q0, dt, 4)], 0.0, rng)
    s.close()
    ctx = expdg.Context(cfg)
    q = q0.copy()
    ctx.advance(q, dt, 4)
    np.testing.assert_array_equal(res[0][0], q)


@pytest.mark.parametrize("prec", [1, 2])
def test_served_sample_against_oracle(mods, prec):
    """The serving workload's CPU-oracle check: a seeded 5 % sample (3 of the
    48 requests of the bench's stream, seed 1: sides 112, 23 and 57 at p = 4,
    3, 3) served in the mixed (or float-float) form through the server,
    against the oracle's FP64 solve of the same request (tol 1e-10, full
    Arnoldi).  Two of each request's 50 EPI2 steps (the oracle's time)."""
    from oracle import dg, integrators
    from tests.test_gpu_parity import TOL_MIXED, rel
    expdg, inputs, serve = mods
    rng = np.random.default_rng(1)
    reqs = [serve.vortex_request(rng, prec, iop=4) for _ in range(48)]
    pick = np.random.default_rng(7).choice(48, size=3, replace=False)
    sub = [(reqs[i][0], reqs[i][1], reqs[i][2], 2) for i in pick]
    srv = serve.Server(workers=3)
    res, _ = serve.run_stream(srv, sub, 0.0, np.random.default_rng(2), check=False)
    srv.close()
    for (cfg, q0, dt, nsteps), r in zip(sub, res):
        assert r[3] == 0
        side = cfg.ne[0]
        mesh = dg.Mesh(dim=2, p=cfg.p, ne=(side, side), lo=(0.0, 0.0), hi=(10.0, 10.0), eq="euler")
        ref = q0.copy()
        for _ in range(nsteps):
            ref, _ = integrators.step(mesh, ref, dt, tol=1e-10)
        assert rel(r[0], ref) <= TOL_MIXED, (side, cfg.p)
