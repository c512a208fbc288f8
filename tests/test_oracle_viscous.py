"""Pins for the oracle's viscous Burgers operator (Sec. 3.1 with kappa > 0,
central fluxes, zero Dirichlet boundaries): exactness on polynomials, the
symmetry and sign of the central-flux diffusion operator, complex-step
Jacobians, the heat equation's exact decay, and the paper's manufactured-
solution table (Sec. 5.1)."""
import math
import os

import numpy as np
import pytest

from oracle import dg, integrators

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "viscous_burgers_mms_lf.txt")


def vmesh(p, ne, kappa=0.03, bc="dirichlet", lo=0.0, hi=1.0, source=None):
    return dg.Mesh(dim=1, p=p, ne=(ne,), lo=(lo,), hi=(hi,), eq="burgers", kappa=kappa, bc=bc, source=source)


def nodes(mesh):
    return dg.node_coords(mesh)[0]          # [e, n]


@pytest.mark.parametrize("p", [2, 3, 5])
def test_gradient_and_diffusion_exact_on_polynomials(p):
    """u = x (1 - x) vanishes at both ends and is a global polynomial: every
    jump and boundary correction is zero, so q = u' = 1 - 2x and the diffusion
    part is kappa u'' = -2 kappa exactly (p >= 2)."""
    mesh = vmesh(p, 5, kappa=0.7)
    x = nodes(mesh)
    U = mesh.to_grid((x * (1 - x))[None])
    np.testing.assert_allclose(dg.gradient(mesh, U)[0], 1 - 2 * x, atol=1e-12)
    np.testing.assert_allclose(dg._viscous(mesh, U)[0], -2 * 0.7 * np.ones_like(x), atol=1e-11)


def _matrix(mesh, qt):
    n = qt.size
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = dg.jv(mesh, qt, e).reshape(-1)
    return A


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("p,ne", [(1, 4), (3, 3), (4, 5)])
def test_central_diffusion_symmetric_negative(bc, p, ne):
    """With u~ = 0 only the diffusion part remains: the central-flux operator
    is symmetric in the LGL mass inner product and negative semidefinite,
    M L = -kappa B^T M B (central fluxes can leave null modes besides the
    constants, e.g. p = 1 with Dirichlet ends, so no definiteness)."""
    mesh = vmesh(p, ne, kappa=0.25, bc=bc)
    A = _matrix(mesh, np.zeros(mesh.n_unknowns))
    M = np.diag(dg.mass_weights(mesh).reshape(-1))
    S = M @ A
    np.testing.assert_allclose(S, S.T, atol=1e-12 * np.max(np.abs(S)))
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    assert np.max(ev) <= 1e-12 * np.max(np.abs(ev))
    if bc == "periodic":                    # constants are in the null space
        assert abs(np.max(ev)) <= 1e-12 * np.max(np.abs(ev))


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_viscous_jv_equals_complex_step(bc):
    rng = np.random.default_rng(70)
    mesh = vmesh(3, 4, kappa=0.05, bc=bc)
    qt = rng.uniform(-1.0, 1.5, mesh.n_unknowns)
    lam = dg.face_lambda(mesh, qt)
    A = _matrix(mesh, qt)
    h = 1e-30
    for j in range(qt.size):
        z = qt.astype(complex)
        z[j] += 1j * h
        col = np.imag(dg.residual(mesh, z, lam=lam)).reshape(-1) / h
        np.testing.assert_allclose(A[:, j], col, rtol=1e-12, atol=1e-12 * np.max(np.abs(A)))


def test_heat_equation_decay():
    """A tiny amplitude makes the convection negligible (relative size ~ the
    amplitude): u = eps sin(pi x) on [0, 1] with zero Dirichlet data decays as
    exp(-kappa pi^2 t) (the heat equation's exact solution)."""
    eps, kappa, t_end, dt = 1e-7, 0.1, 0.5, 0.05
    mesh = vmesh(6, 8, kappa=kappa)
    x = nodes(mesh)
    q = (eps * np.sin(np.pi * x))[None].reshape(-1)
    for _ in range(int(round(t_end / dt))):
        q, _ = integrators.step(mesh, q, dt, scheme=integrators.EXPRB32, tol=1e-13)
    exact = eps * math.exp(-kappa * math.pi ** 2 * t_end) * np.sin(np.pi * x)
    err = np.max(np.abs(q.reshape(x.shape) - exact)) / (eps * math.exp(-kappa * math.pi ** 2 * t_end))
    assert err < 1e-6


def manufactured(x, kappa=0.03):
    """u = sin(x^2) x (x - 1) and its source u u' - kappa u'' (Sec. 5.1)."""
    u = np.sin(x ** 2) * x * (x - 1)
    du = 2 * x * np.cos(x ** 2) * x * (x - 1) + np.sin(x ** 2) * (2 * x - 1)
    ddu = ((6 * x ** 2 - 4 * x) * np.cos(x ** 2) - 4 * x ** 3 * (x - 1) * np.sin(x ** 2)
           + 2 * x * np.cos(x ** 2) * (2 * x - 1) + 2 * np.sin(x ** 2))
    return u, u * du - kappa * ddu


def mms_error(p, ne, dt=5e-5, t_end=0.01, kappa=0.03):
    """EXPRB32 from the nodal interpolant of the manufactured solution to
    t_end; L2 error of the DG polynomial against u, by (p + 6)-point Gauss
    quadrature per element."""
    mesh0 = vmesh(p, ne, kappa=kappa)
    x = nodes(mesh0)
    u0, s = manufactured(x, kappa)
    mesh = vmesh(p, ne, kappa=kappa, source=s[None])
    q = u0[None].reshape(-1)
    for _ in range(int(round(t_end / dt))):
        q, _ = integrators.step(mesh, q, dt, scheme=integrators.EXPRB32, tol=1e-12)
    U = q.reshape(ne, p + 1)
    g, gw = np.polynomial.legendre.leggauss(p + 6)
    r = mesh.r
    V = np.array([[np.prod([(gg - r[m]) / (r[j] - r[m]) for m in range(p + 1) if m != j]) for j in range(p + 1)]
                  for gg in g])
    h = 1.0 / ne
    xg = (np.arange(ne)[:, None] + (g[None, :] + 1) / 2) * h
    ue, _ = manufactured(xg, kappa)
    return math.sqrt(np.sum((U @ V.T - ue) ** 2 * gw[None, :] * h / 2))


def golden():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, h, err, _ = line.split()
            rows.append((int(k), int(h.split("/")[1]), float(err)))
    return rows


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_manufactured_solution_table(k):
    """The paper's LF column at h = 1/20, 1/40: the observed order between
    them is within 0.3 of the printed order (optimal k + 1 for even k,
    sub-optimal for odd k, as the paper observes), and each error within a
    factor 0.75 .. 2.6 of the printed one: this collocated LGL form
    (diagonal mass, nodal source and initial data) is not the paper's own
    quadrature, whose choice the paper does not state (a reading)."""
    ref = {(kk, ne): e for kk, ne, e in golden() if kk == k}
    e20, e40 = mms_error(k, 20), mms_error(k, 40)
    rate, rate_paper = math.log2(e20 / e40), math.log2(ref[(k, 20)] / ref[(k, 40)])
    assert abs(rate - rate_paper) <= 0.3, (rate, rate_paper)
    for e, ne in ((e20, 20), (e40, 40)):
        assert 0.75 <= e / ref[(k, ne)] <= 2.6, (k, ne, e, ref[(k, ne)])
