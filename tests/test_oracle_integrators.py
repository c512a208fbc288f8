"""Pins for the oracle's exponential steps: the method-of-characteristics
Burgers solution (before the shock time t = 1), exact translation of the
isentropic vortex and of the Euler density wave, conservation of the
quadrature totals, the Euler identity EPI2 = exp(dt L) q^n, and the temporal
orders 2 (EPI2), 3 (EXPRB32) and 4 (EXPRB42) of the paper's schemes."""
import math

import numpy as np
import pytest

from oracle import dg, integrators, krylov
from paper_2011_01316_gb300 import inputs


def burgers_mesh(ne=64, p=2):
    return dg.Mesh(dim=1, p=p, ne=(ne,), lo=(0.0,), hi=(2 * math.pi,), eq="burgers")


def l2_rel(mesh, a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(dg.l2_norm(mesh, a - b)) / np.linalg.norm(dg.l2_norm(mesh, b)))


def test_burgers_c0_matches_characteristics():
    """64 elements, p = 2, u0 = 0.5 + sin x, EPI2, tol 1e-10, dt = 1e-2 to
    t = 0.5 (the small Burgers workload)."""
    mesh = burgers_mesh()
    x = dg.node_coords(mesh)
    u = inputs.burgers_sine(x).reshape(-1)
    tot0 = dg.totals(mesh, u)
    u, sts = integrators.advance(mesh, u, 1e-2, 50, scheme=integrators.EPI2, tol=1e-10)
    exact = inputs.burgers_characteristics(x[0], 0.5)
    err = l2_rel(mesh, u, exact[None])
    assert err < 3e-4, err   # spatial error at h = 2 pi/64, p = 2 (same at dt/4)
    assert abs(dg.totals(mesh, u)[0] - tot0[0]) < 1e-13 * abs(tot0[0]) + 1e-14
    assert all(s.substeps == 1 for s in sts)


def test_burgers_spatial_rate():
    """h-refinement at small dt: error against characteristics falls at
    about h^(p+1)."""
    p = 3
    errs = []
    for ne in (16, 32, 64):
        mesh = burgers_mesh(ne, p)
        x = dg.node_coords(mesh)
        u = inputs.burgers_sine(x).reshape(-1)
        u, _ = integrators.advance(mesh, u, 0.0125, 16, scheme=integrators.EXPRB32, tol=1e-12)
        errs.append(l2_rel(mesh, u, inputs.burgers_characteristics(x[0], 0.2)[None]))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > p) and rates[-1] > p + 0.5, (errs, rates)


@pytest.mark.parametrize("scheme,order", [(integrators.EPI2, 2), (integrators.EXPRB32, 3),
                                          (integrators.EXPRB42, 4)])
def test_temporal_order(scheme, order):
    """Order from three step sizes dt, dt/2, dt/4 on a fixed DG space
    (40 elements, p = 4, as in the paper's Burgers temporal study):
    log2(|q_dt - q_dt/2| / |q_dt/2 - q_dt/4|) ~ order."""
    mesh = burgers_mesh(40, 4)
    x = dg.node_coords(mesh)
    u0 = inputs.burgers_sine(x).reshape(-1)
    T = 0.4
    sols = []
    for n in (4, 8, 16):
        u, _ = integrators.advance(mesh, u0, T / n, n, scheme=scheme, tol=1e-13)
        sols.append(u)
    r = math.log2(np.linalg.norm(sols[0] - sols[1]) / np.linalg.norm(sols[1] - sols[2]))
    assert r > order - 0.35, r


def vortex_mesh(ne, p):
    return dg.Mesh(dim=2, p=p, ne=(ne, ne), lo=(0.0, 0.0), hi=(10.0, 10.0), eq="euler")


def test_vortex_translation_and_conservation():
    mesh = vortex_mesh(16, 3)
    X = dg.node_coords(mesh)
    q = inputs.isentropic_vortex(X, 0.0).reshape(-1)
    tot0 = dg.totals(mesh, q)
    q, sts = integrators.advance(mesh, q, 0.1, 5, scheme=integrators.EPI2, tol=1e-10)
    exact = inputs.isentropic_vortex(X, 0.5)
    err = l2_rel(mesh, q, exact)
    assert err < 5e-3, err
    assert np.all(np.abs(dg.totals(mesh, q) - tot0) <= 1e-13 * np.abs(tot0))


def test_euler_epi2_is_exponential_of_state():
    """For Euler N(q^n) = R(q^n) - L(q^n) q^n = 0 (F(q) = A(q) q), so the EPI2
    step equals exp(dt L) q^n; the two Krylov sums agree to the tolerance."""
    mesh = vortex_mesh(6, 2)
    X = dg.node_coords(mesh)
    q = inputs.isentropic_vortex(X, 0.0).reshape(-1)
    dt = 0.2
    q1, _ = integrators.step(mesh, q, dt, scheme=integrators.EPI2, tol=1e-12)
    w, _ = krylov.phi_sum(lambda x: dt * dg.jv(mesh, q, x).reshape(-1), [q], tol=1e-12)
    assert np.max(np.abs(q1 - w)) <= 1e-9 * np.max(np.abs(q))


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 3)])
def test_density_wave_spatial_rate(dim, p):
    """Exact periodic Euler solution rho = 1 + 0.2 sin(x + y - 2t); error under
    refinement at rate >= p + 1/2 (the paper observes k + 1/2 for the
    vortex, Table expo-euler-isentropic-sconv-uni)."""
    errs = []
    for ne in (8, 16, 32):
        mesh = dg.Mesh(dim=dim, p=p, ne=(ne,) * dim, lo=(0.0,) * dim, hi=(2 * math.pi,) * dim, eq="euler")
        X = dg.node_coords(mesh)
        q = inputs.density_wave(X, 0.0).reshape(-1)
        q, _ = integrators.advance(mesh, q, 0.05, 4, scheme=integrators.EXPRB42, tol=1e-12)
        errs.append(l2_rel(mesh, q, inputs.density_wave(X, 0.2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > p) and rates[-1] > p + 0.5, (errs, rates)


def test_density_wave_3d_one_step():
    mesh = dg.Mesh(dim=3, p=2, ne=(4, 4, 4), lo=(0.0,) * 3, hi=(2 * math.pi,) * 3, eq="euler")
    X = dg.node_coords(mesh)
    q = inputs.density_wave(X, 0.0).reshape(-1)
    tot0 = dg.totals(mesh, q)
    q, st = integrators.step(mesh, q, 0.1, scheme=integrators.EPI2, tol=1e-8)
    assert l2_rel(mesh, q, inputs.density_wave(X, 0.1)) < 5e-3
    assert np.all(np.abs(dg.totals(mesh, q) - tot0) <= 1e-13 * np.abs(tot0))


def test_replayed_step_is_identical():
    mesh = vortex_mesh(4, 2)
    X = dg.node_coords(mesh)
    q = inputs.isentropic_vortex(X, 0.0).reshape(-1)
    for scheme in (integrators.EPI2, integrators.EXPRB32, integrators.EXPRB42):
        q1, st = integrators.step(mesh, q, 0.3, scheme=scheme, tol=1e-10, m_max=10)
        q2, st2 = integrators.step(mesh, q, 0.3, scheme=scheme, replay=st.traces)
        np.testing.assert_array_equal(q1, q2)
