"""Viscous Burgers (Sec. 3.1 with kappa > 0, central fluxes, zero Dirichlet
ends, manufactured forcing) on the CUDA path against the oracle.

FP64 form: operators 1e-12, steps with the oracle's decisions replayed 1e-11.
Mixed and float-float forms: 1e-6 per step (their bar).  The manufactured-solution run of
Sec. 5.1 (EXPRB32, dt = 5e-5 to t = 0.01) reproduces the oracle's error."""
import math

import numpy as np
import pytest

from oracle import dg, integrators
from tests.test_gpu_parity import MIXED_PRECS, TOL_MIXED, TOL_OP64, TOL_STEP64, _replay_from, rel
from tests.test_oracle_viscous import manufactured

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_01316_gb300 import expdg
    return expdg


CASES = {
    "dirichlet_p2": dict(p=2, ne=20, bc="dirichlet", kappa=0.03),
    "dirichlet_p5": dict(p=5, ne=13, bc="dirichlet", kappa=0.03),
    "periodic_p3": dict(p=3, ne=17, bc="periodic", kappa=0.05),
    "dirichlet_p1": dict(p=1, ne=40, bc="dirichlet", kappa=0.2),
}


def make(E, case, prec=0, scheme=3, iop=0, tol=1e-10):
    c = CASES[case]
    ctx = E.Context(dim=1, p=c["p"], ne=[c["ne"], 1, 1], lo=[0.0, 0.0, 0.0], hi=[1.0, 1.0, 1.0], eq=E.EXPDG_BURGERS,
                    prec=prec, scheme=scheme, krylov_tol=tol, m_max=64, m_step=5, max_substeps=32, iop=iop,
                    kappa=c["kappa"], bc=E.EXPDG_BC_DIRICHLET if c["bc"] == "dirichlet" else E.EXPDG_BC_PERIODIC)
    mesh0 = dg.Mesh(dim=1, p=c["p"], ne=(c["ne"],), lo=(0.0,), hi=(1.0,), eq="burgers", kappa=c["kappa"], bc=c["bc"])
    x = dg.node_coords(mesh0)[0]
    u, s = manufactured(x, c["kappa"])
    mesh = dg.Mesh(dim=1, p=c["p"], ne=(c["ne"],), lo=(0.0,), hi=(1.0,), eq="burgers", kappa=c["kappa"],
                   bc=c["bc"], source=s[None])
    ctx.set_source(np.ascontiguousarray(s[None]))
    return ctx, mesh, np.ascontiguousarray((u + 0.3 * np.sin(7 * x) * x * (1 - x))[None])


@pytest.mark.parametrize("case", list(CASES))
def test_viscous_residual_and_jv_fp64(E, case):
    ctx, mesh, q = make(E, case)
    assert rel(ctx.residual(q), dg.residual(mesh, q)) <= TOL_OP64
    rng = np.random.default_rng(80)
    v = np.ascontiguousarray(rng.standard_normal(q.shape))
    assert rel(ctx.jv(q, v), dg.jv(mesh, q, v)) <= TOL_OP64


@pytest.mark.parametrize("prec", MIXED_PRECS)
@pytest.mark.parametrize("case", list(CASES))
def test_viscous_residual_mixed(E, case, prec):
    """The mixed form's residual (the FP64 kernel) and the float-float one,
    relative to the size of the terms they sum: 1e-13 (a few hundred units of
    2^-48)."""
    ctx, mesh, q = make(E, case, prec=prec)
    ref = dg.residual(mesh, q)
    scale = np.max(np.abs(ref)) + mesh.kappa * (2.0 / mesh.h[0]) ** 2 * (mesh.p + 1) ** 4 * np.max(np.abs(q))
    assert np.max(np.abs(ctx.residual(q) - ref)) <= 1e-13 * scale


@pytest.mark.parametrize("iop", [0, 4])
@pytest.mark.parametrize("scheme", [2, 3])
@pytest.mark.parametrize("case", list(CASES))
def test_viscous_step_fp64_replayed(E, case, scheme, iop):
    ctx, mesh, q = make(E, case, scheme=scheme, iop=iop)
    dt = 2e-3
    ref, st = integrators.step(mesh, q, dt, scheme=scheme, tol=1e-10, iop=iop or None)
    got = q.copy()
    ctx.step(got, dt, replay=_replay_from(st))
    assert rel(got, ref) <= TOL_STEP64


@pytest.mark.parametrize("prec", MIXED_PRECS)
@pytest.mark.parametrize("scheme", [2, 3])
@pytest.mark.parametrize("case", ["dirichlet_p2", "periodic_p3"])
def test_viscous_step_mixed(E, case, scheme, prec):
    ctx, mesh, q = make(E, case, prec=prec, scheme=scheme, iop=4)
    dt = 2e-3
    ref, _ = integrators.step(mesh, q, dt, scheme=scheme, tol=1e-10)
    got = q.copy()
    ctx.step(got, dt)
    assert rel(got, ref) <= TOL_MIXED


def test_manufactured_solution_run_matches_oracle(E):
    """Sec. 5.1's manufactured problem at k = 2, h = 1/20: EXPRB32, dt = 5e-5,
    200 steps from the nodal interpolant; the GPU FP64 form (adaptive) ends
    where the oracle ends, and its L2 error against the exact solution is the
    oracle's."""
    p, ne, kappa = 2, 20, 0.03
    ctx = E.Context(dim=1, p=p, ne=[ne, 1, 1], lo=[0.0, 0.0, 0.0], hi=[1.0, 1.0, 1.0], eq=E.EXPDG_BURGERS, prec=0,
                    scheme=3, krylov_tol=1e-12, m_max=64, m_step=5, max_substeps=32, kappa=kappa,
                    bc=E.EXPDG_BC_DIRICHLET)
    mesh0 = dg.Mesh(dim=1, p=p, ne=(ne,), lo=(0.0,), hi=(1.0,), eq="burgers", kappa=kappa, bc="dirichlet")
    x = dg.node_coords(mesh0)[0]
    u0, s = manufactured(x, kappa)
    mesh = dg.Mesh(dim=1, p=p, ne=(ne,), lo=(0.0,), hi=(1.0,), eq="burgers", kappa=kappa, bc="dirichlet",
                   source=s[None])
    ctx.set_source(np.ascontiguousarray(s[None]))
    got = np.ascontiguousarray(u0[None].copy())
    ctx.advance(got, 5e-5, 200)
    ref = u0[None].reshape(-1)
    for _ in range(200):
        ref, _ = integrators.step(mesh, ref, 5e-5, scheme=integrators.EXPRB32, tol=1e-12)
    assert rel(got, ref) <= 1e-10
    err_gpu = math.sqrt(np.sum((got[0] - u0) ** 2 * dg.mass_weights(mesh)))
    err_ref = math.sqrt(np.sum((ref.reshape(u0.shape) - u0) ** 2 * dg.mass_weights(mesh)))
    assert abs(err_gpu - err_ref) <= 1e-6 * err_ref


def test_invalid_viscous_configs(E):
    for bad in (dict(kappa=-1.0, eq=1, dim=1), dict(kappa=0.1), dict(bc=1), dict(bc=7, eq=1, dim=1)):
        with pytest.raises(E.ExpdgError) as ei:
            E.Context(**bad)
        assert ei.value.status == E.EXPDG_EINVAL
