"""Resident batch (expdg_batch_*): one launch per class of small EPI2 solves,
one CTA per instance, against the FP64 oracle.

* FP64 form: the same decisions as the oracle's Krylov solver (checks at the
  multiples of m_step, Saad's estimate, the same sub-step rule), so several
  steps agree to rounding: 1e-11 relative, as the replayed FP64 tests of the
  context path.
* Mixed form (FP32 operator, float-float residual, FP64 Krylov): 1e-6
  relative to the oracle, the mixed-form bar.
* An instance gives the same bits alone and in a batch of other classes and
  sizes; a non-physical instance fails alone; bad configurations and
  pointers are rejected.
"""
import math

import numpy as np
import pytest

from oracle import dg, integrators
from paper_2011_01316_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_STEP64 = 1e-11
TOL_MIXED = 1e-6


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_01316_gb300 import expdg
    return torch, expdg


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def burgers(E, ne, p, prec=0, iop=4, tol=1e-10, m_max=40):
    cfg = E.default_config(eq=1, dim=1, p=p, ne=[ne, 1, 1], lo=[0.0, 0, 0], hi=[2 * math.pi, 1, 1], prec=prec,
                           scheme=2, krylov_tol=tol, m_max=m_max, m_step=5, max_substeps=32, iop=iop)
    mesh = dg.Mesh(dim=1, p=p, ne=(ne,), lo=(0.0,), hi=(2 * math.pi,), eq="burgers")
    q = inputs.burgers_sine(dg.node_coords(mesh))
    return cfg, mesh, np.ascontiguousarray(q)


def wave2d(E, side, p, prec=1, iop=4, tol=1e-8, m_max=40):
    L = 2 * math.pi
    cfg = E.default_config(eq=2, dim=2, p=p, ne=[side, side, 1], lo=[0.0, 0.0, 0], hi=[L, L, 1], prec=prec,
                           scheme=2, krylov_tol=tol, m_max=m_max, m_step=5, max_substeps=32, iop=iop, gamma=1.4)
    mesh = dg.Mesh(dim=2, p=p, ne=(side, side), lo=(0.0, 0.0), hi=(L, L), eq="euler")
    q = inputs.density_wave(dg.node_coords(mesh), 0.0)
    return cfg, mesh, np.ascontiguousarray(q)


def run(torch, E, items, dts, nsteps):
    """Advance the (cfg, mesh, q) items as one batch; returns (states, batch)."""
    b = E.Batch([c for c, _, _ in items])
    qs = [torch.from_numpy(q.copy()).cuda() for _, _, q in items]
    st = b.advance(qs, dts, nsteps)
    return [x.cpu().numpy() for x in qs], b, st


def test_burgers_c0_fp64_matches_oracle(env):
    """The 1D Burgers workload (64 elements, p = 2, u0 = 0.5 + sin x, EPI2,
    dt 1e-2, tol 1e-10, window 4) in one launch against the oracle."""
    torch, E = env
    cfg, mesh, q = burgers(E, 64, 2)
    got, b, st = run(torch, E, [(cfg, mesh, q)], [1e-2], 10)
    assert st == E.EXPDG_OK and b.launches() == 1
    ref, sts = integrators.advance(mesh, q, 1e-2, 10, tol=1e-10, m_max=40, m_step=5, iop=4)
    assert rel(got[0], ref) <= TOL_STEP64
    status, stats, done = b.result(0)
    assert status == E.EXPDG_OK and done == 10
    assert stats["krylov_iters"] == sum(s.krylov_iters for s in sts)   # the oracle's decisions
    b.close()


@pytest.mark.parametrize("iop", [0, 1, 4])
@pytest.mark.parametrize("ne,p", [(16, 1), (37, 3), (128, 5)])
def test_burgers_fp64_windows_and_orders(env, ne, p, iop):
    torch, E = env
    cfg, mesh, q = burgers(E, ne, p, iop=iop)
    got, b, st = run(torch, E, [(cfg, mesh, q)], [2e-2], 4)
    assert st == E.EXPDG_OK
    ref, _ = integrators.advance(mesh, q, 2e-2, 4, tol=1e-10, m_max=40, m_step=5, iop=iop or None)
    assert rel(got[0], ref) <= TOL_STEP64
    b.close()


def test_burgers_substeps_fp64(env):
    """A step large enough that m_max = 10 forces halved sub-steps."""
    torch, E = env
    cfg, mesh, q = burgers(E, 32, 3, m_max=10)
    got, b, st = run(torch, E, [(cfg, mesh, q)], [0.2], 2)
    assert st == E.EXPDG_OK
    ref, sts = integrators.advance(mesh, q, 0.2, 2, tol=1e-10, m_max=10, m_step=5, iop=4)
    assert sum(s.rejected for s in sts) > 0
    assert rel(got[0], ref) <= TOL_STEP64
    _, stats, _ = b.result(0)
    assert stats["rejected"] == sum(s.rejected for s in sts)
    b.close()


@pytest.mark.parametrize("side,p", [(6, 1), (8, 2), (5, 4)])
def test_euler2d_mixed_and_fp64_match_oracle(env, side, p):
    torch, E = env
    cfgm, mesh, q = wave2d(E, side, p, prec=1)
    cfg64, _, _ = wave2d(E, side, p, prec=0)
    dt = 0.5 * (2 * math.pi / side) / (p + 1)
    got, b, st = run(torch, E, [(cfgm, mesh, q), (cfg64, mesh, q)], [dt, dt], 3)
    assert st == E.EXPDG_OK and b.launches() == 2
    ref, _ = integrators.advance(mesh, q, dt, 3, tol=1e-8, m_max=40, m_step=5, iop=4)
    assert rel(got[1], ref) <= TOL_STEP64
    assert rel(got[0], ref) <= TOL_MIXED
    # conservation of the cell totals (periodic mesh): to rounding in the FP64
    # form; in the mixed form each FP32 operator output's total is zero only
    # to FP32 rounding, so the totals move by about 1e-10 over these steps
    np.testing.assert_allclose(dg.totals(mesh, got[1]), dg.totals(mesh, q), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dg.totals(mesh, got[0]), dg.totals(mesh, q), rtol=1e-8, atol=1e-8)
    b.close()


def test_same_bits_alone_and_in_a_batch(env):
    torch, E = env
    rng = np.random.default_rng(41)
    items, dts = [], []
    for k in range(7):
        if k % 2 == 0:
            cfg, mesh, _ = burgers(E, int(rng.integers(8, 200)), int(rng.integers(1, 6)), prec=k % 3 == 0)
            q = np.ascontiguousarray(inputs.fourier_modes(dg.node_coords(mesh)[0], rng)[0][None])
            dts.append(0.01)
        else:
            cfg, mesh, q = wave2d(E, int(rng.integers(3, 9)), int(rng.integers(1, 6)), prec=1 if k != 3 else 0)
            dts.append(0.05)
        items.append((cfg, mesh, q))
    together, b, st = run(torch, E, items, dts, 3)
    assert st == E.EXPDG_OK
    assert b.launches() == len({(c.eq, c.dim, c.p, c.prec) for c, _, _ in items})
    b.close()
    for i, item in enumerate(items):
        alone, b1, st1 = run(torch, E, [item], [dts[i]], 3)
        assert st1 == E.EXPDG_OK
        assert np.array_equal(alone[0], together[i]), i
        b1.close()


def test_nonphysical_instance_fails_alone(env):
    torch, E = env
    cfg, mesh, q = wave2d(E, 4, 2, prec=1)
    bad = q.copy()
    bad[0, 3, 2] = -1.0
    cfgb, meshb, qb = burgers(E, 20, 2, prec=1)
    got, b, st = run(torch, E, [(cfg, mesh, bad), (cfgb, meshb, qb)], [0.05, 0.01], 2)
    assert st == E.EXPDG_ENONPHYSICAL
    s0, _, done0 = b.result(0)
    s1, _, done1 = b.result(1)
    assert s0 == E.EXPDG_ENONPHYSICAL and done0 == 0
    assert s1 == E.EXPDG_OK and done1 == 2
    np.testing.assert_array_equal(got[0], bad)   # stopped at the start of the failing step
    b.close()


def test_bad_configurations_and_pointers_rejected(env):
    torch, E = env
    cfg, mesh, q = burgers(E, 16, 2)
    for bad in (dict(scheme=3), dict(p=6), dict(m_max=41), dict(prec=2)):
        c = E.default_config(eq=1, dim=1, p=2, ne=[16, 1, 1], lo=[0, 0, 0], hi=[1, 1, 1], m_max=40)
        for k, v in bad.items():
            setattr(c, k, v)
        with pytest.raises(E.ExpdgError) as ei:
            E.Batch([c])
        assert ei.value.status == E.EXPDG_EINVAL
    c3 = E.default_config(eq=2, dim=3, p=1, ne=[2, 2, 2], lo=[0, 0, 0], hi=[1, 1, 1], m_max=40)
    with pytest.raises(E.ExpdgError):
        E.Batch([c3])
    b = E.Batch([cfg])
    host = q.copy()
    assert b.advance([host], [0.01], 1) == E.EXPDG_EINVAL   # host memory
    dev = torch.from_numpy(q.copy()).cuda()
    assert b.advance([dev], [0.0], 1) == E.EXPDG_EINVAL     # dt must be positive
    b.close()


@pytest.mark.parametrize("bc,kappa,prec", [("dirichlet", 0.03, 0), ("periodic", 0.05, 0), ("dirichlet", 0.03, 1)])
def test_viscous_burgers_resident(env, bc, kappa, prec):
    """Viscous Burgers (central fluxes for the diffusion, zero Dirichlet ends or
    periodic; no forcing) through the resident solve against the oracle."""
    torch, E = env
    ne, p = 24, 3
    cfg = E.default_config(eq=1, dim=1, p=p, ne=[ne, 1, 1], lo=[0.0, 0, 0], hi=[1.0, 1, 1], prec=prec, scheme=2,
                           krylov_tol=1e-10, m_max=40, m_step=5, max_substeps=32, iop=4, kappa=kappa,
                           bc=E.EXPDG_BC_DIRICHLET if bc == "dirichlet" else E.EXPDG_BC_PERIODIC)
    mesh = dg.Mesh(dim=1, p=p, ne=(ne,), lo=(0.0,), hi=(1.0,), eq="burgers", kappa=kappa, bc=bc)
    x = dg.node_coords(mesh)[0]
    q = np.ascontiguousarray((np.sin(2 * math.pi * x) * (0.5 + x * (1 - x)))[None])
    got, b, st = run(torch, E, [(cfg, mesh, q)], [2e-3], 3)
    assert st == E.EXPDG_OK
    ref, _ = integrators.advance(mesh, q, 2e-3, 3, tol=1e-10, m_max=40, m_step=5, iop=4)
    assert rel(got[0], ref) <= (TOL_STEP64 if prec == 0 else TOL_MIXED)
    b.close()
