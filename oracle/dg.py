"""Collocated nodal DG operator R(q) and its frozen-flux linearisation L(q~)v.

Plain FP64 numpy, one whole-mesh array operation per term, in the order the
paper writes the terms.  Test infrastructure only (see ``oracle/__init__``).

Discretisation (Sec. 2.2, Eq. EXPO-SemiDiscretizedForm_ode; Sec. 3):

* Mesh: uniform periodic tensor mesh of ``ne[d]`` elements per direction on
  [lo_d, hi_d], element size h_d = (hi_d - lo_d) / ne[d].  Each element holds
  (p+1)^dim LGL nodes (tensor product).
* Canonical array layout ``q[f, e, n]``: field f, element
  e = ex + ne_x (ey + ne_y ez), node n = i + (p+1)(j + (p+1) k) with i the
  x-index.  Fields: Burgers ``u``; Euler ``rho, rho u_1..rho u_dim, rho E``.
* Semi-discrete right-hand side dq/dt = R(q) in strong collocated form.  With
  LGL collocation (diagonal mass, SBP) this is algebraically the weak forms of
  Sec. 3.1 / 3.2 (Sec. 4 notes LGL quadrature; no over-integration):

    R = - sum_d (2/h_d) D^(d) F_d(q)
        - sum_faces (2/h_d) (1/w_0) (F*.n - F(q^-).n)   at face nodes,

  with the Lax-Friedrichs numerical flux
    F*.n^- = 1/2 (F(q^-) + F(q^+)).n^- + 1/2 lambda (q^- - q^+),
  which is the paper's {F} + 1/2 max|.| [[q]] written for the minus side
  ([[q]].n^- = q^- - q^+ with [[v]] := 2{v.n}, Sec. 2.1).
  - Burgers (Sec. 3.1): f = u^2/2, lambda = max(|u^-|, |u^+|).
  - Euler (Sec. 3.2 fluxes; LF per Sec. 5.1 "we use Lax-Friedrichs flux for
    Euler equations"): lambda = max(|u^-.n| + a^-, |u^+.n| + a^+) per face node
    pair, a = sqrt(gamma p / rho).
* Linear operator L(q~) (Sec. 2.2, Eq. linearflux; Burgers (u~ u)* of
  Sec. 3.1; Euler (A~ q)* of Sec. 3.2): same form with F_d replaced by
  A_d(q~) v and lambda computed from q~ and then held fixed ("frozen"; the
  continuous-level split of Eq. split-goveq-continuous avoids differentiating
  the stabilisation parameter).  Equivalently L(q~) v is the derivative of R
  at q~ with lambda frozen; ``residual(..., lam=face_lambda(q~))`` is that
  frozen-lambda residual, used by the complex-step pin.
* Viscous Burgers (Sec. 3.1, Eq. pde-burgers-eq with kappa > 0; weak forms
  Eq. gov-burgers1d / Burger): the auxiliary q = du/dx with the central flux
  u** = {u} (Eq. gov-burgers1d-gradu), and the total flux u^2/2 - kappa q with
  the central flux q** = {q} for the diffusion part.  In strong collocated form
    q = (2/h) D u + (2/h)(1/w_0) n (u** - u^-)            at face nodes,
    R = R_convective + kappa [ (2/h) D q + (2/h)(1/w_0) n (q** - q^-) ].
  The diffusion part is linear, so L(u~) v carries the same term with q(v).
  Zero Dirichlet boundaries (the paper's footnote to Sec. 4): u^+ = u_D = 0 in
  the convective fluxes (u~u)* and (u^2/2)*, u** = u_D = 0, q** = q^-.
* A time-independent forcing (``Mesh.source``, canonical layout) is added to R,
  as the manufactured-solution experiment of Sec. 5.1 adds its source term.
* Roe flux for Euler (Sec. 3.2, ``Mesh.flux = "roe"``): the LF term
  1/2 lambda (q^- - q^+) becomes 1/2 |A(q*_Roe)| (q^- - q^+), |A| = R |Lambda| R^-1
  of the flux Jacobian in the face normal at the Roe average of the two
  traces (rho* = sqrt(rho^- rho^+), u* and H* weighted by sqrt(rho), a* from
  H* and u*).  The linear operator uses the Roe average of the linearisation
  state's traces, frozen like lambda.
"""

from dataclasses import dataclass, field
import numpy as np

from . import lgl


@dataclass
class Mesh:
    dim: int
    p: int
    ne: tuple
    lo: tuple
    hi: tuple
    eq: str = "euler"          # "burgers" (dim 1) or "euler"
    gamma: float = 1.4
    kappa: float = 0.0         # viscosity (Burgers only)
    bc: str = "periodic"       # "periodic" or "dirichlet" (u_D = 0 at both ends; Burgers only)
    source: object = None      # optional forcing added to R (canonical layout)
    flux: str = "lf"           # numerical flux: "lf" (Lax-Friedrichs) or "roe" (Euler)
    r: np.ndarray = field(init=False, repr=False)
    w: np.ndarray = field(init=False, repr=False)
    D: np.ndarray = field(init=False, repr=False)

    def __post_init__(self):
        self.ne = tuple(int(x) for x in self.ne)
        self.lo = tuple(float(x) for x in self.lo)
        self.hi = tuple(float(x) for x in self.hi)
        assert len(self.ne) == self.dim == len(self.lo) == len(self.hi)
        if self.eq == "burgers" and self.dim != 1:
            raise ValueError("Burgers is one-dimensional (Sec. 3.1)")
        if self.bc not in ("periodic", "dirichlet"):
            raise ValueError("bc must be 'periodic' or 'dirichlet'")
        if (self.kappa != 0.0 or self.bc != "periodic") and self.eq != "burgers":
            raise ValueError("viscosity and Dirichlet boundaries are defined for Burgers (Sec. 3.1)")
        if self.flux not in ("lf", "roe") or (self.flux == "roe" and self.eq != "euler"):
            raise ValueError("flux must be 'lf', or 'roe' for Euler (Sec. 3.2)")
        self.r = lgl.nodes(self.p)
        self.w = lgl.weights(self.p)
        self.D = lgl.diff_matrix(self.p)

    @property
    def h(self):
        return tuple((self.hi[d] - self.lo[d]) / self.ne[d] for d in range(self.dim))

    @property
    def m(self):
        return 1 if self.eq == "burgers" else self.dim + 2

    @property
    def n_elem(self):
        return int(np.prod(self.ne))

    @property
    def n_node(self):
        return (self.p + 1) ** self.dim

    @property
    def n_unknowns(self):
        return self.m * self.n_elem * self.n_node

    # grid form: (m, ne_{dim-1}, ..., ne_0, p+1 (index dim-1), ..., p+1 (index 0))
    def grid_shape(self, m=None):
        m = self.m if m is None else m
        return (m,) + tuple(reversed(self.ne)) + (self.p + 1,) * self.dim

    def elem_axis(self, d):
        return 1 + (self.dim - 1 - d)

    def node_axis(self, d):
        return 1 + self.dim + (self.dim - 1 - d)

    def to_grid(self, q, m=None):
        return np.asarray(q).reshape(self.grid_shape(m))

    def from_grid(self, Q):
        m = Q.shape[0]
        return Q.reshape(m, self.n_elem, self.n_node)


def node_coords(mesh):
    """Physical node coordinates x_d = lo_d + h_d (e_d + (r_i + 1)/2), in the
    canonical layout [d, e, n]."""
    X = np.zeros(mesh.grid_shape(mesh.dim))
    for d in range(mesh.dim):
        e_idx = np.arange(mesh.ne[d], dtype=np.float64)
        shp_e = [1] * (2 * mesh.dim)
        shp_e[mesh.elem_axis(d) - 1] = mesh.ne[d]
        shp_n = [1] * (2 * mesh.dim)
        shp_n[mesh.node_axis(d) - 1] = mesh.p + 1
        X[d] = mesh.lo[d] + mesh.h[d] * (e_idx.reshape(shp_e) + (mesh.r.reshape(shp_n) + 1.0) / 2.0)
    return mesh.from_grid(X)


def _at(ndim, axis, idx):
    s = [slice(None)] * ndim
    s[axis] = idx
    return tuple(s)


# ---------------------------------------------------------------- physics ---

def pressure(mesh, Q):
    """Ideal gas p = (gamma-1)(rho E - 1/2 |rho u|^2 / rho)  (Sec. 3.2)."""
    rho = Q[0]
    mom = Q[1:1 + mesh.dim]
    return (mesh.gamma - 1.0) * (Q[mesh.dim + 1] - 0.5 * np.sum(mom * mom, axis=0) / rho)


def flux(mesh, Q, d):
    """Physical flux component F_d(q).  Burgers f = u^2/2 (Sec. 3.1);
    Euler F_d = (rho u_d, rho u u_d + p e_d, rho u_d H) (Sec. 3.2,
    Eq. euler-gov), rho u_d H = (rho E + p) u_d."""
    if mesh.eq == "burgers":
        return 0.5 * Q * Q
    dim = mesh.dim
    rho = Q[0]
    mom = Q[1:1 + dim]
    E = Q[dim + 1]
    p = pressure(mesh, Q)
    ud = mom[d] / rho
    F = np.empty_like(Q)
    F[0] = mom[d]
    for k in range(dim):
        F[1 + k] = mom[k] * ud + (p if k == d else 0.0)
    F[dim + 1] = (E + p) * ud
    return F


def flux_jacobian_apply(mesh, Qt, V, d):
    """A_d(q~) v: the flux Jacobian dF_d/dq at q~ (Sec. 3.2, matrix A with
    n = e_d; Burgers A = u~, Sec. 3.1) applied to v, written as the
    directional derivative of F_d."""
    if mesh.eq == "burgers":
        return Qt * V
    dim = mesh.dim
    g1 = mesh.gamma - 1.0
    rho = Qt[0]
    mom = Qt[1:1 + dim]
    E = Qt[dim + 1]
    u = mom / rho
    p = pressure(mesh, Qt)
    drho = V[0]
    dmom = V[1:1 + dim]
    dE = V[dim + 1]
    du = (dmom - u * drho) / rho
    dp = g1 * (dE - np.sum(u * dmom, axis=0) + 0.5 * np.sum(u * u, axis=0) * drho)
    out = np.empty_like(V)
    out[0] = dmom[d]
    for k in range(dim):
        out[1 + k] = dmom[k] * u[d] + mom[k] * du[d] + (dp if k == d else 0.0)
    out[dim + 1] = (dE + dp) * u[d] + (E + p) * du[d]
    return out


def wave_speed(mesh, Q, d):
    """|u.n| + a for Euler (a = sqrt(gamma p / rho)); |u| for Burgers."""
    if mesh.eq == "burgers":
        return np.abs(Q[0])
    rho = Q[0]
    un = Q[1 + d] / rho
    a = np.sqrt(mesh.gamma * pressure(mesh, Q) / rho)
    return np.abs(un) + a


def face_traces(mesh, Q, d):
    """Traces on the two faces normal to x_d of every element:
    returns (own_left, nbr_left, own_right, nbr_right); 'nbr_left' is the
    right-end trace of element e-1 (periodic), 'nbr_right' the left-end trace
    of element e+1.  With zero Dirichlet boundaries the outside trace of the
    first and last element is u_D = 0."""
    nd = Q.ndim
    eax, nax, p = mesh.elem_axis(d), mesh.node_axis(d), mesh.p
    own_left = Q[_at(nd, nax, 0)]
    own_right = Q[_at(nd, nax, p)]
    nbr_left = np.roll(Q, 1, axis=eax)[_at(nd, nax, p)]
    nbr_right = np.roll(Q, -1, axis=eax)[_at(nd, nax, 0)]
    if mesh.bc == "dirichlet":
        nbr_left = nbr_left.copy()
        nbr_right = nbr_right.copy()
        nbr_left[_at(nd - 1, eax, 0)] = 0.0
        nbr_right[_at(nd - 1, eax, mesh.ne[d] - 1)] = 0.0
    return own_left, nbr_left, own_right, nbr_right


def _boundary_mask(mesh, trace, d, side):
    """True on the traces of the domain boundary face (side 0: left end of
    element 0, side 1: right end of the last element) of a Dirichlet mesh."""
    mask = np.zeros(trace.shape, dtype=bool)
    if mesh.bc == "dirichlet":
        mask[_at(trace.ndim, mesh.elem_axis(d), 0 if side == 0 else mesh.ne[d] - 1)] = True
    return mask


def gradient(mesh, U):
    """Auxiliary variable q = du/dx of the viscous Burgers equation (grid
    form in, grid form out): Eq. gov-burgers1d-gradu in strong collocated form,
    q = (2/h) D u + (2/h)(1/w_0) n (u** - u^-) at face nodes, with the central
    flux u** = {u} and u** = u_D = 0 on a Dirichlet boundary."""
    d, hd = 0, mesh.h[0]
    nd, nax = U.ndim, mesh.node_axis(0)
    lift = 1.0 / lgl.endpoint_weight(mesh.p)
    G = (2.0 / hd) * _apply_D(mesh, U, d)
    ol, nl, orr, nr = face_traces(mesh, U, d)
    us_l = np.where(_boundary_mask(mesh, ol, d, 0), 0.0, 0.5 * (ol + nl))
    us_r = np.where(_boundary_mask(mesh, orr, d, 1), 0.0, 0.5 * (orr + nr))
    G[_at(nd, nax, 0)] += (2.0 / hd) * lift * (-1.0) * (us_l - ol)
    G[_at(nd, nax, mesh.p)] += (2.0 / hd) * lift * (+1.0) * (us_r - orr)
    return G


def _viscous(mesh, U):
    """kappa [ (2/h) D q + (2/h)(1/w_0) n (q** - q^-) ] with q = gradient(u)
    and the central flux q** = {q} (q** = q^- on a Dirichlet boundary): the
    diffusion part of R (Sec. 3.1, Eq. Burger), linear in u."""
    d, hd = 0, mesh.h[0]
    nd, nax = U.ndim, mesh.node_axis(0)
    lift = 1.0 / lgl.endpoint_weight(mesh.p)
    Qg = gradient(mesh, U)
    R = (2.0 / hd) * _apply_D(mesh, Qg, d)
    ol, nl, orr, nr = face_traces(mesh, Qg, d)
    qs_l = np.where(_boundary_mask(mesh, ol, d, 0), ol, 0.5 * (ol + nl))
    qs_r = np.where(_boundary_mask(mesh, orr, d, 1), orr, 0.5 * (orr + nr))
    R[_at(nd, nax, 0)] += (2.0 / hd) * lift * (-1.0) * (qs_l - ol)
    R[_at(nd, nax, mesh.p)] += (2.0 / hd) * lift * (+1.0) * (qs_r - orr)
    return mesh.kappa * R


def roe_dissipation(mesh, QL, QR, dQ, d):
    """|A(q*_Roe)| dQ for the flux Jacobian in direction e_d (Sec. 3.2 and its
    footnote): the Roe average of the states QL, QR (traces, field-major), then
    the eigen-decomposition of A at (u*, H*) written as waves: acoustic
    u_n -+ a with strengths (dp -+ a (dm_n - u_n drho)) / (2 a^2), entropy u_n
    with drho - dp / a^2, shear u_n with dm_t - u_t drho, where
    dp = (gamma - 1)(dE - u.dm + |u|^2 drho / 2) and the right eigenvectors
    (1, u -+ a e_d, H -+ u_n a), (1, u, |u|^2/2), (0, e_t, u_t)."""
    dim, g1 = mesh.dim, mesh.gamma - 1.0
    rl, rr = QL[0], QR[0]
    sl, sr = np.sqrt(rl), np.sqrt(rr)
    ul, ur = QL[1:1 + dim] / rl, QR[1:1 + dim] / rr
    Hl = (QL[dim + 1] + pressure(mesh, QL)) / rl
    Hr = (QR[dim + 1] + pressure(mesh, QR)) / rr
    u = (sl * ul + sr * ur) / (sl + sr)
    H = (sl * Hl + sr * Hr) / (sl + sr)
    uu = np.sum(u * u, axis=0)
    a2 = g1 * (H - 0.5 * uu)
    a = np.sqrt(a2)
    un = u[d]
    dr, dm, dE = dQ[0], dQ[1:1 + dim], dQ[dim + 1]
    dp = g1 * (dE - np.sum(u * dm, axis=0) + 0.5 * uu * dr)
    dun = dm[d] - un * dr
    am = (dp - a * dun) / (2.0 * a2)
    ap = (dp + a * dun) / (2.0 * a2)
    a0 = dr - dp / a2
    lm, l0, lp = np.abs(un - a), np.abs(un), np.abs(un + a)
    out = np.empty_like(dQ)
    out[0] = lm * am + l0 * a0 + lp * ap
    shear_E = 0.0
    for k in range(dim):
        if k == d:
            out[1 + k] = lm * am * (u[k] - a) + l0 * a0 * u[k] + lp * ap * (u[k] + a)
        else:
            st = dm[k] - u[k] * dr
            out[1 + k] = lm * am * u[k] + l0 * (a0 * u[k] + st) + lp * ap * u[k]
            shear_E = shear_E + u[k] * st
    out[dim + 1] = lm * am * (H - un * a) + l0 * (a0 * 0.5 * uu + shear_E) + lp * ap * (H + un * a)
    return out


def face_dissipation(mesh, q):
    """Frozen data of the face dissipation, per direction: the LF coefficients
    (lam_left, lam_right) of ``face_lambda``, or for the Roe flux the state
    traces (own_left, nbr_left, own_right, nbr_right) that define |A|."""
    if mesh.flux == "roe":
        Q = mesh.to_grid(q)
        return [("roe",) + face_traces(mesh, Q, d) for d in range(mesh.dim)]
    return face_lambda(mesh, q)


def _dissipate(mesh, data, side, dq, d):
    """The dissipation term of a face: lambda dq (LF) or |A(q*_Roe)| dq (Roe)."""
    if len(data) == 5:
        _, ol, nl, orr, nr = data
        ql, qr = (ol, nl) if side == 0 else (orr, nr)
        return roe_dissipation(mesh, ql, qr, dq, d)
    return (data[0] if side == 0 else data[1]) * dq


def face_lambda(mesh, q):
    """LF dissipation coefficient lambda per face-node pair, for each
    direction: [(lam_left, lam_right) for d] (Sec. 3.1 max|u^+-|;
    Sec. 5.1 LF for Euler with |u.n| + a)."""
    Q = mesh.to_grid(q)
    out = []
    for d in range(mesh.dim):
        ol, nl, orr, nr = face_traces(mesh, Q, d)
        lam_l = np.maximum(wave_speed(mesh, ol, d), wave_speed(mesh, nl, d))
        lam_r = np.maximum(wave_speed(mesh, orr, d), wave_speed(mesh, nr, d))
        out.append((lam_l, lam_r))
    return out


def _apply_D(mesh, F, d):
    """(D^(d) F)_i = sum_j D_ij F_j along the node axis of direction d."""
    nax = mesh.node_axis(d)
    Fm = np.moveaxis(F, nax, -1)
    G = Fm @ mesh.D.T
    return np.moveaxis(G, -1, nax)


def _operator(mesh, Q, fluxfn, lam):
    """Shared strong-form assembly: volume derivative plus LF face lift.
    ``fluxfn(S, d)`` gives the (physical or linearised) flux of a state S,
    ``Q`` supplies the jump term, ``lam`` the per-face coefficients."""
    R = np.zeros_like(Q)
    nd = Q.ndim
    lift = 1.0 / lgl.endpoint_weight(mesh.p)
    for d in range(mesh.dim):
        hd = mesh.h[d]
        nax = mesh.node_axis(d)
        # volume term  -(2/h_d) D^(d) F_d
        R -= (2.0 / hd) * _apply_D(mesh, fluxfn(Q, d), d)
        ol, nl, orr, nr = face_traces(mesh, Q, d)
        # left face, outward normal n = -e_d:
        #   F*.n = 1/2 (F(q-) + F(q+)).n + 1/2 D (q- - q+),  D = lam (LF) or |A| (Roe)
        Fm, Fp = fluxfn(ol, d), fluxfn(nl, d)
        fstar_n = 0.5 * (Fm + Fp) * (-1.0) + 0.5 * _dissipate(mesh, lam[d], 0, ol - nl, d)
        R[_at(nd, nax, 0)] -= (2.0 / hd) * lift * (fstar_n - Fm * (-1.0))
        # right face, outward normal n = +e_d
        Fm, Fp = fluxfn(orr, d), fluxfn(nr, d)
        fstar_n = 0.5 * (Fm + Fp) * (+1.0) + 0.5 * _dissipate(mesh, lam[d], 1, orr - nr, d)
        R[_at(nd, nax, mesh.p)] -= (2.0 / hd) * lift * (fstar_n - Fm * (+1.0))
    return R


def residual(mesh, q, lam=None):
    """R(q), the semi-discrete right-hand side dq/dt (Sec. 2.2,
    Eq. EXPO-SemiDiscretizedForm_ode with R = Lq + N(q)).  ``lam`` (as
    returned by ``face_lambda``) freezes the LF coefficient; by default it is
    computed from q itself.  Works for complex q when ``lam`` is given."""
    Q = mesh.to_grid(q)
    if lam is None:
        lam = face_dissipation(mesh, q)
    R = _operator(mesh, Q, lambda S, d: flux(mesh, S, d), lam)
    if mesh.kappa != 0.0:
        R = R + _viscous(mesh, Q)
    R = mesh.from_grid(R)
    if mesh.source is not None:
        R = R + np.asarray(mesh.source).reshape(R.shape)
    return R


def jv(mesh, qt, v):
    """L(q~) v: the DG linear operator built from the linear flux
    F_L = A(q~) v (Eq. linearflux) with the linear LF flux
    (A~v)* = {A~v} + 1/2 lambda~ [[v]], lambda~ from q~ (Sec. 3.1 (u~u)*,
    Sec. 3.2 (A~q)*)."""
    Qt = mesh.to_grid(qt)
    V = mesh.to_grid(v)
    lam = face_dissipation(mesh, qt)
    # the face traces of the linearisation point travel with those of v:
    # apply the operator to the stacked pair and use only the v half.
    m = mesh.m

    def lin_flux(S, d):
        return np.concatenate([np.zeros_like(S[:m]), flux_jacobian_apply(mesh, S[:m], S[m:], d)])

    S = np.concatenate([Qt, V])
    R = np.zeros_like(V)
    nd = V.ndim
    lift = 1.0 / lgl.endpoint_weight(mesh.p)
    for d in range(mesh.dim):
        hd = mesh.h[d]
        nax = mesh.node_axis(d)
        R -= (2.0 / hd) * _apply_D(mesh, flux_jacobian_apply(mesh, Qt, V, d), d)
        ol, nl, orr, nr = face_traces(mesh, S, d)
        Fm = flux_jacobian_apply(mesh, ol[:m], ol[m:], d)
        Fp = flux_jacobian_apply(mesh, nl[:m], nl[m:], d)
        fstar_n = 0.5 * (Fm + Fp) * (-1.0) + 0.5 * _dissipate(mesh, lam[d], 0, ol[m:] - nl[m:], d)
        R[_at(nd, nax, 0)] -= (2.0 / hd) * lift * (fstar_n - Fm * (-1.0))
        Fm = flux_jacobian_apply(mesh, orr[:m], orr[m:], d)
        Fp = flux_jacobian_apply(mesh, nr[:m], nr[m:], d)
        fstar_n = 0.5 * (Fm + Fp) * (+1.0) + 0.5 * _dissipate(mesh, lam[d], 1, orr[m:] - nr[m:], d)
        R[_at(nd, nax, mesh.p)] -= (2.0 / hd) * lift * (fstar_n - Fm * (+1.0))
    del lin_flux
    if mesh.kappa != 0.0:
        R = R + _viscous(mesh, V)
    return mesh.from_grid(R)


def mass_weights(mesh):
    """Diagonal LGL mass per node, prod_d w_{i_d} h_d/2, in layout [e, n]
    (broadcast over fields)."""
    W = np.ones((mesh.p + 1,) * mesh.dim)
    for d in range(mesh.dim):
        shp = [1] * mesh.dim
        shp[mesh.dim - 1 - d] = mesh.p + 1
        W = W * (mesh.w.reshape(shp) * mesh.h[d] / 2.0)
    return np.broadcast_to(W.reshape(1, -1), (mesh.n_elem, mesh.n_node))


def totals(mesh, q):
    """Quadrature total of each field over the mesh, sum_K (q, 1)_K."""
    Q = np.asarray(q).reshape(mesh.m, mesh.n_elem, mesh.n_node)
    return np.sum(Q * mass_weights(mesh)[None], axis=(1, 2))


def l2_norm(mesh, q):
    """Broken L2 norm with the LGL mass, sqrt(sum_K (q, q)_K) per field."""
    Q = np.asarray(q).reshape(mesh.m, mesh.n_elem, mesh.n_node)
    return np.sqrt(np.sum(Q * Q * mass_weights(mesh)[None], axis=(1, 2)))


def max_wave_speed(mesh, q):
    """max over nodes and directions of |u.n| + a (Euler) or |u| (Burgers):
    the c of the paper's Courant number (Sec. 5 footnote)."""
    Q = mesh.to_grid(q)
    return float(max(np.max(wave_speed(mesh, Q, d)) for d in range(mesh.dim)))
