"""Pins for the oracle's dense exponential, scalar phi-functions and the
augmented-Krylov phi-sum: a library Pade expm, quadrature of the paper's
integral definition of phi_i, diagonal operators (closed forms), tiny
assembled operators (dense expm of the augmented matrix), and linear
advection at full size (exact exponential by Bloch/FFT block
diagonalisation)."""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

from oracle import dg, expm, krylov


@pytest.mark.parametrize("n,scale", [(1, 0.3), (5, 0.1), (12, 3.0), (30, 40.0), (64, 12.0)])
def test_expm_matches_library_pade(n, scale):
    rng = np.random.default_rng(n)
    H = np.triu(rng.standard_normal((n, n)), -1) * scale / math.sqrt(n)   # upper Hessenberg
    E = expm.expm(H)
    ref = scipy.linalg.expm(H)
    assert np.max(np.abs(E - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_expm_closed_forms():
    d = np.array([-3.0, -0.5, 0.0, 0.7, 2.0])
    np.testing.assert_allclose(expm.expm(np.diag(d)), np.diag(np.exp(d)), rtol=1e-14)
    J = np.diag(np.ones(4), 1) * 2.0     # nilpotent: exp = sum_k J^k/k!
    ref = sum(np.linalg.matrix_power(J, k) / math.factorial(k) for k in range(5))
    np.testing.assert_allclose(expm.expm(J), ref, rtol=1e-14, atol=1e-14)
    th = 7.3                               # rotation generator
    R = expm.expm(np.array([[0.0, -th], [th, 0.0]]))
    np.testing.assert_allclose(R, [[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]], atol=1e-13)


@pytest.mark.parametrize("i", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("z", [-40.0, -3.0, -0.7, -1e-3, 0.0, 0.4, 2.5, 1.5 + 2.0j])
def test_phi_scalar_integral_definition(i, z):
    """phi_i(z) = int_0^1 e^{(1-t) z} t^{i-1}/(i-1)! dt (Sec. 2.3), phi_0 = e^z."""
    got = expm.phi_scalar(i, z)
    if i == 0:
        ref = np.exp(z)
    else:
        f = lambda t, part: (np.exp((1 - t) * z) * t ** (i - 1) / math.factorial(i - 1)).__getattribute__(part)  # noqa
        ref = (scipy.integrate.quad(f, 0, 1, args=("real",), epsabs=1e-14, epsrel=1e-13, limit=200)[0]
               + 1j * scipy.integrate.quad(f, 0, 1, args=("imag",), epsabs=1e-14, epsrel=1e-13, limit=200)[0])
    assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref))
    if z == 0.0:
        assert abs(got - 1.0 / math.factorial(i)) < 1e-15


@pytest.mark.parametrize("P", [0, 1, 2, 3])
def test_phi_sum_diagonal_operator(P):
    """Diagonal A: sum_i phi_i(A) c_i is the scalar closed form per entry."""
    rng = np.random.default_rng(10 + P)
    N = 60
    a = rng.uniform(-6.0, 0.5, N)
    c = [rng.standard_normal(N) for _ in range(P + 1)]
    w, st = krylov.phi_sum(lambda x: a * x, c, tol=1e-12, m_max=64)
    ref = np.array([sum((expm.phi_scalar(i, a[k]) * c[i][k]).real for i in range(P + 1)) for k in range(N)])
    assert np.max(np.abs(w - ref)) <= 1e-10 * np.max(np.abs(ref))


def _assembled(mesh, qt):
    n = qt.size
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = dg.jv(mesh, qt, e).reshape(-1)
    return A


def _augmented_dense(A, c):
    """exp of the (N+P)-square augmented matrix, built densely."""
    P = len(c) - 1
    N = A.shape[0]
    M = np.zeros((N + P, N + P))
    M[:N, :N] = A
    for k in range(1, P + 1):          # column N+k-1 holds c_{P+1-k}
        M[:N, N + k - 1] = c[P + 1 - k]
    for k in range(P - 1):
        M[N + k, N + k + 1] = 1.0
    start = np.concatenate([c[0], np.zeros(P)])
    if P:
        start[N + P - 1] = 1.0
    return (scipy.linalg.expm(M) @ start)[:N]


@pytest.mark.parametrize("P", [0, 1, 3])
@pytest.mark.parametrize("eq,dim,p,ne", [("burgers", 1, 2, (3,)), ("euler", 2, 1, (2, 2))])
def test_phi_sum_tiny_mesh_dense_expm(P, eq, dim, p, ne):
    """m reaching N + P gives the exact result: compare with a dense expm
    (library Pade) of the assembled augmented matrix."""
    from tests.test_oracle_dg import make_mesh, random_state
    rng = np.random.default_rng(20 + P)
    mesh = make_mesh(eq, dim, p, ne)
    qt = random_state(mesh, rng).reshape(-1)
    dt = 0.05
    A = dt * _assembled(mesh, qt)
    c = [rng.standard_normal(qt.size) for _ in range(P + 1)]
    ref = _augmented_dense(A, c)
    w, st = krylov.phi_sum(lambda x: A @ x, c, tol=1e-14, m_max=qt.size + P + 1)
    assert np.max(np.abs(w - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("P", [1, 2, 3])
def test_phi_sum_substepping_and_replay(P):
    """Forcing a small m_max makes the solver sub-step; the result is still the
    dense one, and replaying the recorded trace reproduces it exactly."""
    from tests.test_oracle_dg import make_mesh, random_state
    rng = np.random.default_rng(30)
    mesh = make_mesh("burgers", 1, 4, (4,))
    qt = random_state(mesh, rng).reshape(-1)
    A = 1.5 * _assembled(mesh, qt)
    c = [rng.standard_normal(qt.size) for _ in range(P + 1)]
    ref = _augmented_dense(A, c)
    w, st = krylov.phi_sum(lambda x: A @ x, c, tol=1e-12, m_max=10, m_step=5)
    assert st.substeps > 1 and st.rejected >= 1
    assert abs(sum(s for s, _, _ in st.trace) - 1.0) == 0.0
    assert np.max(np.abs(w - ref)) <= 1e-9 * np.max(np.abs(ref))
    w2, st2 = krylov.phi_sum(lambda x: A @ x, c, replay=st.trace)
    np.testing.assert_array_equal(w, w2)
    assert st2.trace == st.trace


def _bloch_exp_advection(c, p, ne, length, dt, v):
    """exp(dt L) v for DG linear advection on a uniform periodic 1D mesh.
    L is block-circulant: (L v)_e = B_-1 v_{e-1} + B_0 v_e + B_+1 v_{e+1};
    blocks read off one oracle Jv on a 3-element periodic mesh of the same
    element size (every block sees the same neighbours), then each Bloch
    symbol B(theta) = sum_k B_k e^{i k theta} is exponentiated densely
    (library Pade) and the result assembled by FFT."""
    h = length / ne
    small = dg.Mesh(dim=1, p=p, ne=(3,), lo=(0.0,), hi=(3 * h,), eq="burgers")
    n = p + 1
    ut = np.full((1, 3, n), c)
    B = {k: np.zeros((n, n)) for k in (-1, 0, 1)}
    for j in range(n):
        e = np.zeros((1, 3, n))
        e[0, 1, j] = 1.0                  # unit vector in the middle element
        col = dg.jv(small, ut, e)[0]
        B[0][:, j] = col[1]
        B[1][:, j] = col[0]               # element 0 sees element 1 as its +1 neighbour
        B[-1][:, j] = col[2]              # element 2 sees element 1 as its -1 neighbour
    V = np.fft.fft(v.reshape(ne, n), axis=0)          # V_k = sum_e v_e e^{-i theta_k e}
    out = np.zeros_like(V)
    for k in range(ne):
        th = 2 * np.pi * k / ne
        sym = B[0] + B[-1] * np.exp(-1j * th) + B[1] * np.exp(1j * th)
        out[k] = scipy.linalg.expm(dt * sym) @ V[k]
    return np.real(np.fft.ifft(out, axis=0)).reshape(-1)


@pytest.mark.parametrize("c,p,ne,dt", [(1.0, 4, 64, 0.05), (-0.6, 3, 128, 0.1), (1.0, 2, 256, 0.02)])
def test_linear_advection_exponential_full_size(c, p, ne, dt):
    """N = 0 (linear problem): the phi-sum with c = [v] is exp(dt L) v, which
    the Bloch/FFT construction gives exactly."""
    rng = np.random.default_rng(40)
    length = 2 * np.pi
    mesh = dg.Mesh(dim=1, p=p, ne=(ne,), lo=(0.0,), hi=(length,), eq="burgers")
    ut = np.full((1, mesh.n_elem, mesh.n_node), c)
    x = dg.node_coords(mesh)[0]
    v = (np.sin(x) + 0.3 * np.cos(3 * x) + 0.1 * rng.standard_normal(x.shape)).reshape(-1)
    ref = _bloch_exp_advection(c, p, ne, length, dt, v)
    w, st = krylov.phi_sum(lambda y: dt * dg.jv(mesh, ut, y).reshape(-1), [v], tol=1e-12, m_max=64)
    assert np.max(np.abs(w - ref)) <= 1e-9 * np.max(np.abs(ref))


# ---- incomplete orthogonalisation (KIOPS's replacement for Arnoldi, Sec. 1) ----

def _recorded_basis(A, c0, iop, m):
    """Vectors v_0..v_{m-1} the solver feeds to the operator (P = 0, so they
    are the whole basis vectors), with a fixed m and no acceptance test."""
    seen = []

    def apply(x):
        seen.append(np.array(x))
        return A @ x
    krylov.phi_sum(apply, [c0], replay=[(1.0, m, 1.0)], iop=iop)
    return np.array(seen)


@pytest.mark.parametrize("iop", [1, 2, 3, 5])
def test_iom_orthogonality_pattern(iop):
    """v_{j+1} is orthogonalised against v_{j-iop+1..j}: each basis vector is
    orthogonal to exactly the iop vectors before it.  Inner products inside
    that window vanish to rounding, those outside it do not (non-symmetric
    operator)."""
    rng = np.random.default_rng(50)
    n, m = 80, 14
    A = rng.standard_normal((n, n)) / math.sqrt(n) - 0.3 * np.eye(n)
    V = _recorded_basis(A, rng.standard_normal(n), iop, m)
    G = V @ V.T
    np.testing.assert_allclose(np.diag(G), 1.0, rtol=1e-13)
    for j in range(m):
        for i in range(max(0, j - iop), j):
            assert abs(G[i, j]) < 1e-12
        if j - iop - 1 >= 0:
            assert abs(G[j - iop - 1, j]) > 1e-6


def test_iom_window_covering_m_is_full_arnoldi():
    rng = np.random.default_rng(51)
    n = 50
    A = rng.standard_normal((n, n)) / math.sqrt(n) - np.eye(n)
    c = [rng.standard_normal(n), rng.standard_normal(n)]
    w0, s0 = krylov.phi_sum(lambda x: A @ x, c, tol=1e-12, m_max=40)
    w1, s1 = krylov.phi_sum(lambda x: A @ x, c, tol=1e-12, m_max=40, iop=40)
    np.testing.assert_array_equal(w0, w1)
    assert s0.trace == s1.trace


def test_iom_symmetric_operator_is_lanczos():
    """Symmetric A (P = 0): Arnoldi reduces to the three-term Lanczos
    recurrence, so a window of 2 spans the same space with the same H as
    full orthogonalisation; the phi-sums agree to rounding and with the
    dense exponential."""
    rng = np.random.default_rng(52)
    n = 120
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Q * rng.uniform(-8.0, 0.0, n)) @ Q.T
    A = 0.5 * (A + A.T)
    c0 = rng.standard_normal(n)
    ref = scipy.linalg.expm(A) @ c0
    wf, _ = krylov.phi_sum(lambda x: A @ x, [c0], tol=1e-13, m_max=40, m_step=5)
    wl, _ = krylov.phi_sum(lambda x: A @ x, [c0], tol=1e-13, m_max=40, m_step=5, iop=2)
    assert np.max(np.abs(wl - ref)) <= 1e-11 * np.max(np.abs(ref))
    assert np.max(np.abs(wl - wf)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("iop", [2, 4])
@pytest.mark.parametrize("P", [1, 3])
def test_iom_tiny_mesh_dense_expm(iop, P):
    """With incomplete orthogonalisation the accepted result still meets the
    tolerance against the dense augmented exponential (Euler, 2x2, p = 2)."""
    from tests.test_oracle_dg import make_mesh, random_state
    rng = np.random.default_rng(53 + P)
    mesh = make_mesh("euler", 2, 2, (2, 2))
    qt = random_state(mesh, rng).reshape(-1)
    A = 0.05 * _assembled(mesh, qt)
    c = [np.zeros(qt.size)] + [rng.standard_normal(qt.size) for _ in range(P)]
    ref = _augmented_dense(A, c)
    tol = 1e-10
    w, st = krylov.phi_sum(lambda x: A @ x, c, tol=tol, m_max=64, iop=iop)
    assert st.substeps >= 1
    assert np.max(np.abs(w - ref)) <= 10 * tol * np.linalg.norm(ref)
