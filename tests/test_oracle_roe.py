"""Pins for the oracle's Roe flux (Sec. 3.2 and its Roe-average footnote):
|A| against an eigen-decomposition of the paper's printed flux Jacobian,
Roe's property of the average, complex-step Jacobians, homogeneity,
free-stream preservation, conservation and consistency with the PDE."""
import numpy as np
import pytest

from oracle import dg
from paper_2011_01316_gb300 import inputs
from tests.test_oracle_dg import paper_A, random_state

TINY = [(1, 3, (3,)), (2, 2, (2, 2)), (2, 1, (3, 2)), (3, 1, (2, 2, 2)), (3, 2, (2, 1, 2))]


def rmesh(dim, p, ne):
    return dg.Mesh(dim=dim, p=p, ne=ne, lo=(0.0,) * dim, hi=tuple(1.0 + 0.5 * d for d in range(dim)),
                   eq="euler", flux="roe")


def roe_state(qL, qR, dim, gamma):
    """A conservative state with the Roe average's velocity and enthalpy (the
    flux Jacobian depends on u and H only); density sqrt(rho_L rho_R)."""
    def uH(q):
        rho, u = q[0], q[1:1 + dim] / q[0]
        p = (gamma - 1) * (q[dim + 1] - 0.5 * rho * u @ u)
        return rho, u, (q[dim + 1] + p) / rho
    rl, ul, Hl = uH(qL)
    rr, ur, Hr = uH(qR)
    sl, sr = np.sqrt(rl), np.sqrt(rr)
    u = (sl * ul + sr * ur) / (sl + sr)
    H = (sl * Hl + sr * Hr) / (sl + sr)
    rho = sl * sr
    a2 = (gamma - 1) * (H - 0.5 * u @ u)
    E = H - a2 / gamma                     # p / rho = a^2 / gamma
    return np.concatenate([[rho], rho * u, [rho * E]])


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_roe_dissipation_is_abs_of_paper_jacobian(dim):
    """|A(q*_Roe)| dq = R |Lambda| R^-1 dq with (Lambda, R) the eigen-pairs of
    the Jacobian exactly as printed (Sec. 3.2), evaluated at the Roe average."""
    rng = np.random.default_rng(90)
    mesh = rmesh(dim, 1, (1,) * dim)
    for _ in range(25):
        qL = inputs.random_euler_state(dim, 1, 1, rng)[:, 0, 0]
        qR = inputs.random_euler_state(dim, 1, 1, rng)[:, 0, 0]
        dq = rng.standard_normal(dim + 2)
        qs = roe_state(qL, qR, dim, mesh.gamma)
        for d in range(dim):
            n = np.zeros(dim)
            n[d] = 1.0
            lam, R = np.linalg.eig(paper_A(qs, n, mesh.gamma))
            absA = np.real(R @ np.diag(np.abs(np.real(lam))) @ np.linalg.inv(R))
            got = dg.roe_dissipation(mesh, qL.reshape(-1, 1), qR.reshape(-1, 1), dq.reshape(-1, 1), d)[:, 0]
            np.testing.assert_allclose(got, absA @ dq, rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_roe_average_property(dim):
    """Roe's defining property: A(q*_Roe) (q_R - q_L) = F(q_R) - F(q_L)."""
    rng = np.random.default_rng(91)
    mesh = rmesh(dim, 1, (1,) * dim)
    for _ in range(25):
        qL = inputs.random_euler_state(dim, 1, 1, rng)[:, 0, 0]
        qR = inputs.random_euler_state(dim, 1, 1, rng)[:, 0, 0]
        qs = roe_state(qL, qR, dim, mesh.gamma)
        for d in range(dim):
            n = np.zeros(dim)
            n[d] = 1.0
            dF = dg.flux(mesh, qR.reshape(-1, 1), d)[:, 0] - dg.flux(mesh, qL.reshape(-1, 1), d)[:, 0]
            np.testing.assert_allclose(paper_A(qs, n, mesh.gamma) @ (qR - qL), dF, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dim,p,ne", TINY)
def test_roe_jv_equals_complex_step(dim, p, ne):
    rng = np.random.default_rng(92)
    mesh = rmesh(dim, p, ne)
    qt = random_state(mesh, rng).reshape(-1)
    frozen = dg.face_dissipation(mesh, qt)
    n = qt.size
    h = 1e-30
    scale = 0.0
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        jv = dg.jv(mesh, qt, e).reshape(-1)
        z = qt.astype(complex)
        z[j] += 1j * h
        cs = np.imag(dg.residual(mesh, z, lam=frozen)).reshape(-1) / h
        cols.append((jv, cs))
        scale = max(scale, np.max(np.abs(jv)))
    for jv, cs in cols:
        np.testing.assert_allclose(jv, cs, rtol=1e-12, atol=1e-12 * scale)


@pytest.mark.parametrize("dim,p,ne", [(1, 3, (5,)), (2, 2, (3, 4)), (3, 1, (2, 3, 2))])
def test_roe_homogeneity_free_stream_conservation(dim, p, ne):
    """F(q) = A(q) q and the same |A| on both sides: L(q) q = R(q); constant
    states are steady; the totals of R and L v vanish (periodic mesh)."""
    rng = np.random.default_rng(93)
    mesh = rmesh(dim, p, ne)
    q = random_state(mesh, rng).reshape(-1)
    R = dg.residual(mesh, q).reshape(-1)
    assert np.max(np.abs(R - dg.jv(mesh, q, q).reshape(-1))) <= 1e-13 * np.max(np.abs(R))
    const = inputs.conservative(np.full((mesh.n_elem, mesh.n_node), 1.3), [0.4, -0.2, 0.1][:dim],
                                np.full((mesh.n_elem, mesh.n_node), 0.9), mesh.gamma)
    assert np.max(np.abs(dg.residual(mesh, const))) < 1e-13
    Rg = dg.residual(mesh, q.reshape(mesh.m, mesh.n_elem, mesh.n_node))
    scale = np.sum(np.abs(Rg.reshape(mesh.m, -1)) * dg.mass_weights(mesh).reshape(1, -1), axis=1)
    assert np.all(np.abs(dg.totals(mesh, Rg)) <= 1e-13 * scale)


def test_roe_differs_from_lf_only_in_dissipation():
    """On a continuous state (no jumps) the two fluxes agree; on a random one
    they differ (the dissipation term is active)."""
    rng = np.random.default_rng(94)
    lf = dg.Mesh(dim=2, p=3, ne=(4, 4), lo=(0.0, 0.0), hi=(2 * np.pi,) * 2, eq="euler")
    roe = dg.Mesh(dim=2, p=3, ne=(4, 4), lo=(0.0, 0.0), hi=(2 * np.pi,) * 2, eq="euler", flux="roe")
    X = dg.node_coords(lf)
    smooth = inputs.density_wave(X, 0.0)
    # continuous across faces only up to the polynomial representation: compare
    # against the size of the residual
    q = random_state(lf, rng)
    assert np.max(np.abs(dg.residual(lf, q) - dg.residual(roe, q))) > 1e-3
    assert (np.max(np.abs(dg.residual(lf, smooth) - dg.residual(roe, smooth)))
            <= 1e-2 * np.max(np.abs(dg.residual(lf, smooth))))


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 3)])
def test_roe_residual_consistent_with_pde(dim, p):
    """R(q) -> dq/dt of the exact density wave at rate >= p."""
    errs = []
    for ne in (4, 8, 16):
        mesh = dg.Mesh(dim=dim, p=p, ne=(ne,) * dim, lo=(0.0,) * dim, hi=(2 * np.pi,) * dim, eq="euler",
                       flux="roe")
        X = dg.node_coords(mesh)
        dt = 1e-6
        q0 = inputs.density_wave(X, 0.0)
        dqdt = (inputs.density_wave(X, dt) - inputs.density_wave(X, -dt)) / (2 * dt)
        errs.append(np.max(np.abs(dg.residual(mesh, q0) - dqdt)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > p - 0.3), (errs, rates)


@pytest.mark.parametrize("dim,p,ne", [(1, 2, (4,)), (2, 2, (3, 3)), (3, 2, (3, 2, 2))])
def test_roe_face_matrix_from_operator(dim, p, ne):
    """On a state that is constant per element, the face dissipation matrix
    read off the linear operator at a face node (whose other indices are
    interior: the volume term cancels the lifted own-side flux there) is
    R |Lambda| R^-1 of the printed Jacobian at the Roe average of the two
    elements' states, column by column."""
    from tests.test_oracle_dg import _face_column, _face_probe_node, _neighbour, _piecewise_constant_state
    rng = np.random.default_rng(95)
    mesh = rmesh(dim, p, ne)
    qt = _piecewise_constant_state(dim, ne, p, rng, mesh.gamma)
    for d in range(dim):
        nvec = np.zeros(dim)
        nvec[d] = 1.0
        for side in (0, 1):
            n = _face_probe_node(mesh, d, side)
            e = int(rng.integers(mesh.n_elem))
            qs = roe_state(qt[:, e, 0], qt[:, _neighbour(mesh, e, d, side), 0], dim, mesh.gamma)
            lam, R = np.linalg.eig(paper_A(qs, nvec, mesh.gamma))
            absA = np.real(R @ np.diag(np.abs(np.real(lam))) @ np.linalg.inv(R))
            for f in range(mesh.m):
                np.testing.assert_allclose(_face_column(mesh, qt, f, e, n, d), absA[:, f], rtol=1e-10,
                                           atol=1e-11 * np.max(np.abs(absA)))
