"""The allocation-free residual entry point, through the C-ABI.

expdg_residual_noalloc serves callers that cannot allocate device memory
(their GPU memory belongs to their own pool allocator, or cudaMalloc's
implicit synchronisation is not acceptable on their path).  Its scratch is a
fixed static device array shared by all calls, so each check makes two calls
in a row and compares both with the context-based expdg_residual, at the
tolerance the operator parity tests use for the FP64 form (relative 1e-12;
both paths run the same kernels, so the results should agree exactly), and
with the CPU oracle's residual at the operator parity tests' bars (the FP64
residual of the FP64 and mixed forms 1e-12; the float-float one within its
forward-error bound).

This file is named to be collected last: it must pass alone in a fresh
process and after every other test.
"""
import ctypes
import math

import numpy as np
import pytest

from oracle import dg
from tests.test_gpu_parity import C_RFX, TOL_OP64, flux_scale

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_01316_gb300 import expdg, inputs
    return torch, expdg, inputs


def _state(expdg, inputs, ctx, kind):
    X = ctx.node_coords()
    if kind == "vortex":
        return inputs.isentropic_vortex(X, 0.0, center=(4.0, 6.0))
    if kind == "burgers":
        return inputs.burgers_sine(X)
    return inputs.density_wave(X, 0.0)


CASES = [
    ("vortex", dict(dim=2, p=4, ne=[16, 12, 1], lo=[0, 0, 0], hi=[10, 10, 1], eq=2)),
    ("burgers", dict(dim=1, p=2, ne=[64, 1, 1], lo=[0, 0, 0], hi=[2 * math.pi, 1, 1], eq=1)),
    ("wave3d", dict(dim=3, p=3, ne=[6, 5, 4], lo=[0, 0, 0], hi=[2 * math.pi] * 3, eq=2)),
]


def _mesh(cfg):
    d = cfg.dim
    return dg.Mesh(dim=d, p=cfg.p, ne=tuple(cfg.ne[:d]), lo=tuple(cfg.lo[:d]), hi=tuple(cfg.hi[:d]),
                   eq="burgers" if cfg.eq == 1 else "euler")


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("kind,kw", CASES)
def test_noalloc_residual_matches_context_residual(env, kind, kw, prec):
    torch, expdg, inputs = env
    cfg = expdg.default_config(**kw, prec=prec)
    ctx = expdg.Context(cfg)
    qh = np.ascontiguousarray(_state(expdg, inputs, ctx, kind))
    q = torch.from_numpy(qh).cuda()
    ref = torch.empty_like(q)
    ctx.residual(q, ref)
    mesh = _mesh(cfg)
    oracle = dg.residual(mesh, qh)
    for _ in range(2):
        out = torch.full_like(q, float("nan"))
        st = expdg.lib.expdg_residual_noalloc(ctypes.byref(cfg), ctypes.c_void_p(q.data_ptr()),
                                              ctypes.c_void_p(out.data_ptr()), None)
        assert st == expdg.EXPDG_OK
        err = float(torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref))
        assert err <= TOL, err
        got = out.cpu().numpy()
        if prec != 0:
            assert np.linalg.norm(got - oracle) <= C_RFX * (mesh.p + 1) ** 2 * flux_scale(mesh, qh)
        else:
            assert np.linalg.norm(got - oracle) <= TOL_OP64 * np.linalg.norm(oracle)
    ctx.close()


def test_noalloc_rejects_oversize_and_host_pointers(env):
    torch, expdg, inputs = env
    small = torch.zeros(8, dtype=torch.float64, device="cuda")
    for prec in (1, 2):   # the forms that use the static float-float scratch
        big = expdg.default_config(dim=3, p=3, ne=[32, 32, 32], lo=[0, 0, 0], hi=[1, 1, 1], eq=2, prec=prec)
        st = expdg.lib.expdg_residual_noalloc(ctypes.byref(big), ctypes.c_void_p(small.data_ptr()),
                                              ctypes.c_void_p(small.data_ptr()), None)
        assert st == expdg.EXPDG_EINVAL
    cfg = expdg.default_config(dim=1, p=2, ne=[4, 1, 1], lo=[0, 0, 0], hi=[1, 1, 1], eq=1)
    h = np.zeros(12)
    st = expdg.lib.expdg_residual_noalloc(ctypes.byref(cfg), ctypes.c_void_p(h.ctypes.data),
                                          ctypes.c_void_p(h.ctypes.data), None)
    assert st == expdg.EXPDG_EINVAL


def test_noalloc_reports_nonphysical_state(env):
    torch, expdg, inputs = env
    cfg = expdg.default_config(dim=2, p=2, ne=[4, 4, 1], lo=[0, 0, 0], hi=[10, 10, 1], eq=2)
    ctx = expdg.Context(cfg)
    q = torch.from_numpy(np.ascontiguousarray(_state(expdg, inputs, ctx, "vortex"))).cuda()
    q[0, 2, 3] = -1.0
    out = torch.empty_like(q)
    st = expdg.lib.expdg_residual_noalloc(ctypes.byref(cfg), ctypes.c_void_p(q.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), None)
    assert st == expdg.EXPDG_ENONPHYSICAL
    q[0, 2, 3] = 1.0
    st = expdg.lib.expdg_residual_noalloc(ctypes.byref(cfg), ctypes.c_void_p(q.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), None)
    assert st == expdg.EXPDG_OK   # the flag of the previous call was cleared
    ctx.close()


def test_noalloc_and_context_reject_another_devices_memory(env):
    """Memory of a GPU other than the current one is refused (EXPDG_EINVAL), not
    dereferenced: the kernels would fault without peer access.  Needs two GPUs."""
    torch, expdg, inputs = env
    if torch.cuda.device_count() < 2:
        pytest.skip("needs a second GPU")
    cfg = expdg.default_config(dim=1, p=2, ne=[8, 1, 1], lo=[0, 0, 0], hi=[1, 1, 1], eq=1)
    other = torch.zeros(24, dtype=torch.float64, device="cuda:1")
    mine = torch.zeros(24, dtype=torch.float64, device="cuda:0")
    with torch.cuda.device(0):
        st = expdg.lib.expdg_residual_noalloc(ctypes.byref(cfg), ctypes.c_void_p(other.data_ptr()),
                                              ctypes.c_void_p(mine.data_ptr()), None)
        assert st == expdg.EXPDG_EINVAL
        ctx = expdg.Context(cfg)
        with pytest.raises(expdg.ExpdgError) as ei:
            ctx.residual(other, mine)
        assert ei.value.status == expdg.EXPDG_EINVAL
        ctx.close()
