"""The Roe flux (Sec. 3.2) on the CUDA path against the oracle.

FP64 form: operators 1e-12, steps with the oracle's decisions replayed 1e-11;
FP32 and float-float operators within the forward-error bounds of
tests/test_gpu_parity.py (the mixed form's residual is the FP64 one: 1e-12);
mixed and float-float steps 1e-6."""
import numpy as np
import pytest

from oracle import dg, integrators
from tests.test_gpu_parity import (C_JV32, C_RFX, CASES, MIXED_PRECS, PRECS, TOL_MIXED, TOL_OP64, TOL_STEP64, _replay_from,
                                   flux_scale, rel, state)

pytestmark = pytest.mark.gpu

EULER_CASES = ["euler1d_p3", "euler2d_p4", "euler2d_p1", "euler2d_p7", "euler3d_p3", "euler3d_p2"]


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_01316_gb300 import expdg
    return expdg


def make(E, case, prec=0, scheme=2, iop=0, tol=1e-10):
    c = CASES[case]
    ctx = E.Context(eq=c["eq"], dim=c["dim"], p=c["p"], ne=list(c["ne"]) + [1] * (3 - c["dim"]),
                    lo=list(c["lo"]) + [0.0] * (3 - c["dim"]), hi=list(c["hi"]) + [1.0] * (3 - c["dim"]),
                    prec=prec, scheme=scheme, krylov_tol=tol, m_max=64, m_step=5, max_substeps=32, gamma=1.4,
                    iop=iop, flux=E.EXPDG_FLUX_ROE)
    mesh = dg.Mesh(dim=c["dim"], p=c["p"], ne=c["ne"], lo=c["lo"], hi=c["hi"], eq="euler", flux="roe")
    return ctx, mesh


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", EULER_CASES)
def test_roe_residual_and_jv_parity(E, case, prec):
    rng = np.random.default_rng(95)
    ctx, mesh = make(E, case, prec=prec)
    for smooth in (True, False):
        q = np.ascontiguousarray(state(mesh, rng, smooth))
        R, Rref = ctx.residual(q), dg.residual(mesh, q)
        v = np.ascontiguousarray(rng.standard_normal(q.shape))
        Lv, Lref = ctx.jv(q, v), dg.jv(mesh, q, v)
        amp = (mesh.p + 1) ** 2
        if prec in MIXED_PRECS:
            assert np.linalg.norm(R - Rref) <= C_RFX * amp * flux_scale(mesh, q)
        else:
            assert rel(R, Rref) <= TOL_OP64
        if prec == 0:
            assert rel(Lv, Lref) <= TOL_OP64
        else:
            assert np.linalg.norm(Lv - Lref) <= C_JV32 * amp * flux_scale(mesh, q, v)


@pytest.mark.parametrize("iop", [0, 4])
@pytest.mark.parametrize("scheme", [2, 3])
@pytest.mark.parametrize("case", ["euler1d_p3", "euler2d_p4", "euler3d_p3"])
def test_roe_step_fp64_replayed(E, case, scheme, iop):
    rng = np.random.default_rng(96)
    ctx, mesh = make(E, case, scheme=scheme, iop=iop)
    q = np.ascontiguousarray(state(mesh, rng))
    ref, st = integrators.step(mesh, q, 0.05, scheme=scheme, tol=1e-10, iop=iop or None)
    got = q.copy()
    ctx.step(got, 0.05, replay=_replay_from(st))
    assert rel(got, ref) <= TOL_STEP64
    np.testing.assert_allclose(dg.totals(mesh, got), dg.totals(mesh, q), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("prec", MIXED_PRECS)
@pytest.mark.parametrize("scheme", [2, 3])
@pytest.mark.parametrize("case", ["euler2d_p4", "euler3d_p3"])
def test_roe_step_mixed(E, case, scheme, prec):
    rng = np.random.default_rng(97)
    ctx, mesh = make(E, case, prec=prec, scheme=scheme, iop=4)
    q = np.ascontiguousarray(state(mesh, rng))
    ref, _ = integrators.step(mesh, q, 0.05, scheme=scheme, tol=1e-10)
    got = q.copy()
    ctx.step(got, 0.05)
    assert rel(got, ref) <= TOL_MIXED


def test_roe_rejected_for_burgers(E):
    with pytest.raises(E.ExpdgError) as ei:
        E.Context(eq=1, dim=1, flux=E.EXPDG_FLUX_ROE)
    assert ei.value.status == E.EXPDG_EINVAL
