"""The tensor-core trial of the operator's derivative contraction (tile
classes EXPDG_TILE_TC3 and EXPDG_TILE_TC1: sum_j D_ij F_j as warp-level
m16n8k8 TF32 matrix products, FP32 accumulation) against the oracle.

Operator, forward-error bound as in tests/test_gpu_parity.py,
||Lv - L64 v|| <= c (p+1)^2 S: TC3 (operands split into two TF32 parts,
three products; each operand carried to about 21 of FP32's 24 significant
bits) c = 1e-6; TC1 (one product of 11-bit TF32 significands, u = 2^-11)
c = 2e-3.  Steps: TC3 within the mixed form's 1e-6 bar."""
import math

import numpy as np
import pytest

from oracle import dg, integrators
from paper_2011_01316_gb300 import inputs
from tests.test_gpu_parity import TOL_MIXED, flux_scale, rel

pytestmark = pytest.mark.gpu

C_TC3, C_TC1 = 1e-6, 2e-3
CASES = {
    "euler2d_p4": dict(dim=2, p=4, ne=(7, 5)),
    "euler2d_p7": dict(dim=2, p=7, ne=(3, 4)),
    "euler3d_p4": dict(dim=3, p=4, ne=(3, 2, 3)),
    "euler3d_p5": dict(dim=3, p=5, ne=(2, 3, 2)),
    "euler3d_p7": dict(dim=3, p=7, ne=(2, 2, 1)),
    "euler3d_p8": dict(dim=3, p=8, ne=(1, 2, 2)),
}


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_01316_gb300 import expdg
    return expdg


def make(E, case, tile, scheme=2):
    c = CASES[case]
    d = c["dim"]
    hi = (2 * math.pi,) * d
    ctx = E.Context(eq=2, dim=d, p=c["p"], ne=list(c["ne"]) + [1] * (3 - d), lo=[0.0] * 3, hi=list(hi) + [1.0] * (3 - d),
                    prec=E.EXPDG_MIXED, scheme=scheme, krylov_tol=1e-10, m_max=64, m_step=5, max_substeps=32,
                    gamma=1.4, iop=4, tile=tile)
    mesh = dg.Mesh(dim=d, p=c["p"], ne=c["ne"], lo=(0.0,) * d, hi=hi, eq="euler")
    return ctx, mesh


@pytest.mark.parametrize("tile", [4, 5])
@pytest.mark.parametrize("case", list(CASES))
def test_tensor_core_operator_parity(E, case, tile):
    rng = np.random.default_rng(120)
    ctx, mesh = make(E, case, tile)
    assert ctx.tile == tile
    for smooth in (True, False):
        X = dg.node_coords(mesh)
        q = inputs.density_wave(X, 0.0) if smooth else inputs.random_euler_state(mesh.dim, mesh.n_elem,
                                                                                  mesh.n_node, rng)
        q = np.ascontiguousarray(q)
        v = np.ascontiguousarray(rng.standard_normal(q.shape))
        Lv, Lref = ctx.jv(q, v), dg.jv(mesh, q, v)
        bound = (C_TC3 if tile == 4 else C_TC1) * (mesh.p + 1) ** 2 * flux_scale(mesh, q, v)
        assert np.linalg.norm(Lv - Lref) <= bound, (np.linalg.norm(Lv - Lref) / bound)
    ctx.close()


@pytest.mark.parametrize("case", ["euler2d_p4", "euler3d_p4", "euler3d_p7"])
def test_tensor_core_step_within_bar(E, case):
    ctx, mesh = make(E, case, 4)
    q = np.ascontiguousarray(inputs.density_wave(dg.node_coords(mesh), 0.0))
    ref, _ = integrators.step(mesh, q, 0.05, tol=1e-10)
    got = q.copy()
    ctx.step(got, 0.05)
    ctx.close()
    assert rel(got, ref) <= TOL_MIXED
