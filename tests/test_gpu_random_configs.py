"""Seeded random configurations across the supported space (dimension,
order, uneven meshes, both equations, LF / Roe fluxes, viscosity, the three
schemes, orthogonalisation window, CTA tile): one step of the FP64 form with
the oracle's decisions replayed (1e-11) and one adaptive step of each of the
mixed and float-float forms against the oracle (1e-6, those forms' bar)."""
import math

import numpy as np
import pytest

from oracle import dg, integrators
from paper_2011_01316_gb300 import inputs
from tests.test_gpu_parity import MIXED_PRECS, TOL_MIXED, TOL_STEP64, _replay_from, rel

pytestmark = pytest.mark.gpu


def draw(seed):
    rng = np.random.default_rng(1000 + seed)
    eq = int(rng.integers(1, 3))
    dim = 1 if eq == 1 else int(rng.integers(1, 4))
    pmax = {1: 8, 2: 6, 3: 4}[dim]
    p = int(rng.integers(1, pmax + 1))
    nmax = {1: 40, 2: 9, 3: 4}[dim]
    ne = tuple(int(rng.integers(1, nmax + 1)) for _ in range(dim))
    hi = tuple(float(rng.uniform(3.0, 7.0)) for _ in range(dim))
    viscous = eq == 1 and rng.random() < 0.4
    cfg = dict(eq=eq, dim=dim, p=p, ne=ne, hi=hi, scheme=int(rng.integers(2, 5)), iop=int(rng.choice([0, 2, 4, 8])),
               tile=int(rng.integers(0, 4)), flux=int(eq == 2 and rng.random() < 0.3),
               kappa=float(rng.uniform(0.01, 0.05)) if viscous else 0.0,
               bc=int(viscous and rng.random() < 0.5))
    return cfg, rng


def make(E, cfg, prec):
    d = cfg["dim"]
    ctx = E.Context(eq=cfg["eq"], dim=d, p=cfg["p"], ne=list(cfg["ne"]) + [1] * (3 - d),
                    lo=[0.0] * 3, hi=list(cfg["hi"]) + [1.0] * (3 - d), prec=prec, scheme=cfg["scheme"],
                    krylov_tol=1e-10, m_max=64, m_step=5, max_substeps=32, gamma=1.4, iop=cfg["iop"],
                    tile=cfg["tile"], flux=cfg["flux"], kappa=cfg["kappa"], bc=cfg["bc"])
    mesh = dg.Mesh(dim=d, p=cfg["p"], ne=cfg["ne"], lo=(0.0,) * d, hi=cfg["hi"],
                   eq="burgers" if cfg["eq"] == 1 else "euler", flux="roe" if cfg["flux"] else "lf",
                   kappa=cfg["kappa"], bc="dirichlet" if cfg["bc"] else "periodic")
    return ctx, mesh


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_01316_gb300 import expdg
    return expdg


@pytest.mark.parametrize("seed", range(60))
def test_random_config_step(E, seed):
    cfg, rng = draw(seed)
    ctx, mesh = make(E, cfg, 0)
    X = dg.node_coords(mesh)
    if cfg["eq"] == 1:
        q = inputs.fourier_modes(X[0], rng, mean=0.5)[0][None].copy()
        if cfg["bc"]:  # zero Dirichlet ends: a state that vanishes there
            q = q * np.sin(math.pi * X[0] / cfg["hi"][0])[None]
    else:
        q = inputs.random_euler_state(mesh.dim, mesh.n_elem, mesh.n_node, rng)
    q = np.ascontiguousarray(q)
    dt = 0.02 if cfg["eq"] == 1 else 0.03
    iop = cfg["iop"] or None
    ref, st = integrators.step(mesh, q, dt, scheme=cfg["scheme"], tol=1e-10, iop=iop)
    got = q.copy()
    ctx.step(got, dt, replay=_replay_from(st))
    assert rel(got, ref) <= TOL_STEP64, cfg
    ctx.close()
    for prec in MIXED_PRECS:
        ctxm, _ = make(E, cfg, prec)
        gotm = q.copy()
        ctxm.step(gotm, dt)
        ctxm.close()
        assert rel(gotm, ref) <= TOL_MIXED, (prec, rel(gotm, ref), cfg)
