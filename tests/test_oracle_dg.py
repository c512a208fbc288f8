"""Pins for the oracle's DG operator R(q) and linear operator L(q~)v:
complex-step derivatives, the paper's printed flux Jacobian, homogeneity of
the Euler flux, free-stream preservation, conservation, and consistency
with the PDE on smooth data."""
import numpy as np
import pytest

from oracle import dg
from paper_2011_01316_gb300 import inputs

TINY = [
    ("burgers", 1, 2, (3,)),
    ("burgers", 1, 4, (4,)),
    ("euler", 1, 3, (3,)),
    ("euler", 2, 2, (2, 2)),
    ("euler", 2, 1, (3, 2)),
    ("euler", 3, 1, (2, 2, 2)),
    ("euler", 3, 2, (2, 1, 2)),
]


def make_mesh(eq, dim, p, ne):
    return dg.Mesh(dim=dim, p=p, ne=ne, lo=(0.0,) * dim, hi=tuple(1.0 + 0.5 * d for d in range(dim)), eq=eq)


def random_state(mesh, rng):
    if mesh.eq == "burgers":
        return rng.uniform(-1.0, 1.5, (1, mesh.n_elem, mesh.n_node))
    return inputs.random_euler_state(mesh.dim, mesh.n_elem, mesh.n_node, rng)


@pytest.mark.parametrize("eq,dim,p,ne", TINY)
def test_jv_equals_complex_step_jacobian(eq, dim, p, ne):
    """Assemble L(q~) column by column from Jv and from the complex-step
    derivative of the frozen-lambda residual; the two agree to rounding."""
    rng = np.random.default_rng(1)
    mesh = make_mesh(eq, dim, p, ne)
    qt = random_state(mesh, rng).reshape(-1)
    lam = dg.face_lambda(mesh, qt)
    n = qt.size
    h = 1e-30
    J_cs = np.zeros((n, n))
    J_jv = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        J_cs[:, j] = np.imag(dg.residual(mesh, qt + 1j * h * e, lam=lam).reshape(-1)) / h
        J_jv[:, j] = dg.jv(mesh, qt, e).reshape(-1)
    scale = np.max(np.abs(J_cs))
    assert np.max(np.abs(J_cs - J_jv)) <= 1e-13 * scale


def paper_A(q, nvec, gamma):
    """The Euler flux Jacobian A = dF.n/dq exactly as printed in Sec. 3.2."""
    dim = len(nvec)
    rho, mom, E = q[0], q[1:1 + dim], q[dim + 1]
    u = mom / rho
    gm = gamma - 1.0
    p = gm * (E - 0.5 * rho * u @ u)
    H = (E + p) / rho
    un = nvec @ u
    phi = 0.5 * gm * (u @ u)
    A = np.zeros((dim + 2, dim + 2))
    A[0, 1:1 + dim] = nvec
    A[1:1 + dim, 0] = phi * nvec - u * un
    A[1:1 + dim, 1:1 + dim] = np.outer(u, nvec) - gm * np.outer(nvec, u) + un * np.eye(dim)
    A[1:1 + dim, dim + 1] = gm * nvec
    A[dim + 1, 0] = (phi - H) * un
    A[dim + 1, 1:1 + dim] = H * nvec - gm * u * un
    A[dim + 1, dim + 1] = gamma * un
    return A


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_flux_jacobian_matches_paper_matrix(dim):
    rng = np.random.default_rng(2)
    mesh = make_mesh("euler", dim, 1, (1,) * dim)
    for _ in range(20):
        q = inputs.random_euler_state(dim, 1, 1, rng)[:, 0, 0]
        v = rng.standard_normal(dim + 2)
        for d in range(dim):
            n = np.zeros(dim)
            n[d] = 1.0
            ref = paper_A(q, n, mesh.gamma) @ v
            got = dg.flux_jacobian_apply(mesh, q.reshape(-1, 1), v.reshape(-1, 1), d)[:, 0]
            np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dim,p,ne", [(1, 3, (5,)), (2, 2, (3, 4)), (3, 1, (2, 3, 2))])
def test_euler_homogeneity(dim, p, ne):
    """F(q) = A(q) q for the Euler flux, so L(q) q = R(q) (with lambda
    computed from q on both sides)."""
    rng = np.random.default_rng(3)
    mesh = make_mesh("euler", dim, p, ne)
    q = random_state(mesh, rng).reshape(-1)
    R = dg.residual(mesh, q).reshape(-1)
    Lq = dg.jv(mesh, q, q).reshape(-1)
    assert np.max(np.abs(R - Lq)) <= 1e-13 * np.max(np.abs(R))


@pytest.mark.parametrize("eq,dim,p,ne", TINY + [("euler", 2, 4, (3, 3))])
def test_free_stream_and_conservation(eq, dim, p, ne):
    rng = np.random.default_rng(4)
    mesh = make_mesh(eq, dim, p, ne)
    if eq == "burgers":
        const = np.full((1, mesh.n_elem, mesh.n_node), 0.7)
    else:
        const = inputs.conservative(np.full((mesh.n_elem, mesh.n_node), 1.3),
                                    [0.4, -0.2, 0.1][:dim], np.full((mesh.n_elem, mesh.n_node), 0.9),
                                    mesh.gamma)
    assert np.max(np.abs(dg.residual(mesh, const))) < 1e-13
    assert np.max(np.abs(dg.jv(mesh, const, const))) < 1e-13 or eq == "burgers"
    q = random_state(mesh, rng)
    R = dg.residual(mesh, q)
    tot = dg.totals(mesh, R)
    scale = np.sum(np.abs(R.reshape(mesh.m, -1)) * dg.mass_weights(mesh).reshape(1, -1), axis=1)
    assert np.all(np.abs(tot) <= 1e-13 * scale)
    v = rng.standard_normal(q.shape)
    Lv = dg.jv(mesh, q, v)
    tot = dg.totals(mesh, Lv)
    scale = np.sum(np.abs(Lv.reshape(mesh.m, -1)) * dg.mass_weights(mesh).reshape(1, -1), axis=1)
    assert np.all(np.abs(tot) <= 1e-13 * scale)


def test_burgers_residual_consistent_with_pde():
    """R(u) -> -(u^2/2)_x for smooth u under refinement, at rate >= p."""
    errs = []
    p = 3
    for ne in (8, 16, 32):
        mesh = dg.Mesh(dim=1, p=p, ne=(ne,), lo=(0.0,), hi=(2 * np.pi,), eq="burgers")
        x = dg.node_coords(mesh)
        u = inputs.burgers_sine(x)
        R = dg.residual(mesh, u)
        exact = -(u * np.cos(x[0]))
        errs.append(np.max(np.abs(R - exact)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > p - 0.3), rates


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 3), (3, 1)])
def test_euler_residual_consistent_with_pde(dim, p):
    """R(q) -> dq/dt of the exact density wave, at rate >= p."""
    errs = []
    for ne in (4, 8, 16) if dim == 2 else (4, 8):
        mesh = dg.Mesh(dim=dim, p=p, ne=(ne,) * dim, lo=(0.0,) * dim, hi=(2 * np.pi,) * dim, eq="euler")
        X = dg.node_coords(mesh)
        dt = 1e-6
        q0 = inputs.density_wave(X, 0.0)
        dqdt = (inputs.density_wave(X, dt) - inputs.density_wave(X, -dt)) / (2 * dt)
        R = dg.residual(mesh, q0)
        errs.append(np.max(np.abs(R - dqdt)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > p - 0.3), (errs, rates)


def test_node_coords_layout():
    mesh = dg.Mesh(dim=3, p=2, ne=(3, 2, 4), lo=(0, 1, 2), hi=(3, 3, 6), eq="euler")
    X = dg.node_coords(mesh)
    # element e = ex + ne_x (ey + ne_y ez), node n = i + 3 (j + 3 k)
    e = 1 + 3 * (1 + 2 * 2)
    n = 2 + 3 * (0 + 3 * 1)
    r = mesh.r
    assert X[0, e, n] == pytest.approx(0 + 1.0 * (1 + (r[2] + 1) / 2))
    assert X[1, e, n] == pytest.approx(1 + 1.0 * (1 + (r[0] + 1) / 2))
    assert X[2, e, n] == pytest.approx(2 + 1.0 * (2 + (r[1] + 1) / 2))


@pytest.mark.parametrize("c,p,ne", [(0.8, 2, 5), (-1.3, 4, 3), (0.5, 1, 7)])
def test_linear_advection_energy_dissipation(c, p, ne):
    """Burgers L(u~) at constant u~ = c is DG linear advection with the LF
    flux; with LGL/SBP its energy rate is exactly
    v^T M L v = -1/2 |c| sum_faces (v^- - v^+)^2 (dissipation only through
    the lambda = |c| jump term; a wrong sign or lift factor breaks it)."""
    rng = np.random.default_rng(5)
    mesh = dg.Mesh(dim=1, p=p, ne=(ne,), lo=(0.0,), hi=(1.7,), eq="burgers")
    ut = np.full((1, mesh.n_elem, mesh.n_node), c)
    v = rng.standard_normal((1, mesh.n_elem, mesh.n_node))
    Lv = dg.jv(mesh, ut, v)
    M = dg.mass_weights(mesh)
    lhs = np.sum(v[0] * M * Lv[0])
    jumps = v[0, :, p] - np.roll(v[0, :, 0], -1)
    rhs = -0.5 * abs(c) * np.sum(jumps ** 2)
    assert abs(lhs - rhs) <= 1e-13 * max(1.0, abs(rhs))


# ---- the Lax-Friedrichs coefficient of the Euler operator (Sec. 3.2, Sec. 5.1) ----
# The dissipation coefficient lambda of the Euler LF flux multiplies the jump
# only, so free stream, conservation, homogeneity and the complex-step pin
# (which freeze the same lambda on both sides) cannot see it.  These pins fix
# its value from the paper's printed flux Jacobian (Sec. 3.2): lambda at a face
# node pair is the larger spectral radius of A_n(q^-) and A_n(q^+).

def _spectral_radius(q, d, gamma):
    n = np.zeros(len(q) - 2)
    n[d] = 1.0
    return float(np.max(np.abs(np.linalg.eigvals(paper_A(q, n, gamma)))))


def _piecewise_constant_state(dim, ne, p, rng, gamma=1.4):
    """Euler states constant on each element, drawn per element: rho and p in
    [0.6, 1.6], every velocity component in [-1, 1] (both signs of u.n)."""
    nel, nn = int(np.prod(ne)), (p + 1) ** dim
    rho = rng.uniform(0.6, 1.6, (nel, 1))
    pr = rng.uniform(0.6, 1.6, (nel, 1))
    vel = [rng.uniform(-1.0, 1.0, (nel, 1)) for _ in range(dim)]
    return np.ascontiguousarray(np.broadcast_to(inputs.conservative(rho, vel, pr, gamma), (dim + 2, nel, nn)))


def _face_probe_node(mesh, d, side):
    """Node index with i_d = 0 (side 0) or p (side 1) and every other index
    interior (1), so only the face normal to x_d touches it."""
    idx = [1] * mesh.dim
    idx[d] = 0 if side == 0 else mesh.p
    n, mult = 0, 1
    for k in range(mesh.dim):
        n += idx[k] * mult
        mult *= mesh.p + 1
    return n


def _neighbour(mesh, e, d, side):
    ec, t = [], e
    for k in range(mesh.dim):
        ec.append(t % mesh.ne[k])
        t //= mesh.ne[k]
    ec[d] = (ec[d] + (1 if side else -1)) % mesh.ne[d]
    out, mult = 0, 1
    for k in range(mesh.dim):
        out += ec[k] * mult
        mult *= mesh.ne[k]
    return out


def _face_column(mesh, qt, f, e, n, d):
    """-(h_d w_0) L(q~) e_{f,e,n} at node (e, n): at a face node whose other
    indices are interior, the volume term (D_pp = 1/(2 w_0), SBP) cancels the
    lifted own-side flux, so this is the face's dissipation matrix applied to
    e_f: lambda e_f for LF, |A(q*_Roe)| e_f for Roe."""
    v = np.zeros((mesh.m, mesh.n_elem, mesh.n_node))
    v[f, e, n] = 1.0
    Lv = dg.jv(mesh, qt, v)
    return -mesh.h[d] * mesh.w[0] * Lv[:, e, n]


@pytest.mark.parametrize("dim,p,ne", [(1, 2, (4,)), (2, 2, (3, 3)), (2, 3, (3, 2)), (3, 2, (3, 3, 2))])
def test_euler_lf_coefficient_is_larger_spectral_radius(dim, p, ne):
    """On a state that is constant per element but jumps between elements, the
    LF coefficient read off the operator at every probed face node equals
    max(rho(A_n(q^-)), rho(A_n(q^+))), rho the spectral radius of the printed
    Jacobian (its eigenvalues u.n - a, u.n, u.n + a: so |u.n| + a, the max
    over the two sides, not a mean and not |u.n| alone)."""
    rng = np.random.default_rng(11)
    mesh = make_mesh("euler", dim, p, ne)
    qt = _piecewise_constant_state(dim, ne, p, rng, mesh.gamma)
    elems = rng.choice(mesh.n_elem, size=min(3, mesh.n_elem), replace=False)
    nprobe = 0
    for d in range(dim):
        for side in (0, 1):
            n = _face_probe_node(mesh, d, side)
            for e in elems:
                e = int(e)
                en = _neighbour(mesh, e, d, side)
                lam = max(_spectral_radius(qt[:, e, 0], d, mesh.gamma), _spectral_radius(qt[:, en, 0], d, mesh.gamma))
                for f in range(mesh.m):
                    col = _face_column(mesh, qt, f, e, n, d)
                    ref = np.zeros(mesh.m)
                    ref[f] = lam
                    np.testing.assert_allclose(col, ref, rtol=1e-12, atol=1e-12 * lam)
                    nprobe += 1
    assert nprobe == 2 * dim * len(elems) * mesh.m


@pytest.mark.parametrize("dim,d", [(1, 0), (2, 0), (2, 1), (3, 2)])
def test_euler_lf_characteristic_energy(dim, d):
    """Linearised about a constant state and applied to data that varies along
    x_d only, L splits in the characteristic variables w = R^-1 v of the
    printed Jacobian A_{e_d} into scalar LF advections with speeds Lambda_k and
    the common coefficient lambda = max_k |Lambda_k|; with the LGL (SBP) mass
    each satisfies w_k^T M (R^-1 L v)_k = -1/2 lambda sum_faces |face| [w_k]^2
    (the energy-rate identity of the Burgers pin above, per characteristic
    field)."""
    rng = np.random.default_rng(12)
    p, ne = 3, (4, 3, 2)[:dim]
    mesh = make_mesh("euler", dim, p, ne)
    qc = inputs.conservative(np.array(1.1), [0.7, -0.4, 0.3][:dim], np.array(0.8), mesh.gamma)
    qt = np.broadcast_to(qc.reshape(-1, 1, 1), (mesh.m, mesh.n_elem, mesh.n_node)).copy()
    nvec = np.zeros(dim)
    nvec[d] = 1.0
    Lam, Rv = np.linalg.eig(paper_A(qc, nvec, mesh.gamma))
    Lam, Rv = np.real(Lam), np.real(Rv)
    lam = np.max(np.abs(Lam))
    # w: random along x_d (element index along d and node index along d), constant otherwise
    Q = mesh.to_grid(np.zeros((mesh.m, mesh.n_elem, mesh.n_node)))
    eax, nax = mesh.elem_axis(d), mesh.node_axis(d)
    prof = rng.standard_normal((mesh.m, mesh.ne[d], p + 1))
    shp = [mesh.m] + [1] * (2 * dim)
    shp[eax], shp[nax] = mesh.ne[d], p + 1
    W = np.broadcast_to(prof.reshape(shp), Q.shape)
    V = np.einsum("ij,j...->i...", Rv, W)
    Lv = mesh.to_grid(dg.jv(mesh, qt, mesh.from_grid(V)))
    Wl = np.einsum("ij,j...->i...", np.linalg.inv(Rv), Lv)
    M = mesh.to_grid(np.broadcast_to(dg.mass_weights(mesh)[None], (1, mesh.n_elem, mesh.n_node)), m=1)[0]
    face = float(np.prod([mesh.hi[k] - mesh.lo[k] for k in range(dim) if k != d]))
    for k in range(mesh.m):
        lhs = float(np.sum(W[k] * M * Wl[k]))
        jumps = prof[k, :, p] - np.roll(prof[k, :, 0], -1)
        rhs = -0.5 * lam * face * float(np.sum(jumps ** 2))
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs)), (k, Lam[k], lhs, rhs)
