"""Exponential time steps of the paper, FP64 (test infrastructure only).

R(q) = L q + N(q) is the DG right-hand side (``dg.residual``) and
L = L(q^n) the frozen-flux linear operator at the current state
(``dg.jv``; the footnotes write L = dR/dq at q^n, the body of Sec. 2.2
builds it from the linear flux with the stabilisation frozen - this oracle
uses the body's operator, N(q) := R(q) - L q).

* EPI2 (Sec. 5.1 footnote, Tokman):
    q^{n+1} = q^n + dt phi_1(dt L) R^n.
* EXPRB32 (Sec. 5.1 footnote, Hochbruck & Ostermann):
    q^(2)   = q^n + dt phi_1(dt L) R^n,
    q^{n+1} = q^n + dt phi_1(dt L) R^n + 2 dt phi_3(dt L) D_{n,2},
    D_{n,2} = N(q^(2)) - N(q^n) = R(q^(2)) - R^n - L (q^(2) - q^n).
* EXPRB42 (Sec. 5.2 footnote, Luan):
    q^(2)   = q^n + 3/4 dt phi_1(3/4 dt L) R^n,
    q^{n+1} = q^n + dt phi_1(dt L) R^n + 32/9 dt phi_3(dt L) D_{n,2}.

Each phi-combination is one call of ``krylov.phi_sum`` with
c = [c_0, ..., c_P].
"""

from dataclasses import dataclass, field
import numpy as np

from . import dg
from .krylov import phi_sum

EPI2, EXPRB32, EXPRB42 = 2, 3, 4


@dataclass
class StepStats:
    krylov_iters: int = 0
    substeps: int = 0
    rejected: int = 0
    jv_applies: int = 0
    residual_applies: int = 0
    err_est: float = 0.0
    traces: list = field(default_factory=list)   # one (sigma, m, eta) list per Krylov solve


def step(mesh, q, dt, scheme=EPI2, tol=1e-10, m_max=64, m_step=5, max_substeps=64, replay=None, iop=None):
    """One exponential step from q^n; returns (q^{n+1}, StepStats).
    ``replay`` is an optional list (one entry per Krylov solve of the step)
    of (sigma, m, eta) traces to follow; ``iop`` the incomplete
    orthogonalisation window of the Krylov solves (None: full Arnoldi)."""
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    st = StepStats()
    Rn = dg.residual(mesh, q).reshape(-1)
    st.residual_applies += 1

    def L(x):
        st.jv_applies += 1
        return dg.jv(mesh, q, x).reshape(-1)

    zero = np.zeros_like(q)
    solve_id = [0]

    def krylov(A, c):
        rp = None if replay is None else replay[solve_id[0]]
        solve_id[0] += 1
        w, ks = phi_sum(A, c, tol=tol, m_max=m_max, m_step=m_step,
                        max_substeps=max_substeps, replay=rp, iop=iop)
        st.krylov_iters += ks.iterations
        st.substeps += ks.substeps
        st.rejected += ks.rejected
        st.err_est = max(st.err_est, ks.err_est)
        st.traces.append(ks.trace)
        return w

    dtL = lambda x: dt * L(x)  # noqa: E731
    if scheme == EPI2:
        w = krylov(dtL, [zero, dt * Rn])
        return q + w, st
    if scheme == EXPRB32:
        w1 = krylov(dtL, [zero, dt * Rn])
        q2 = q + w1
        D = dg.residual(mesh, q2).reshape(-1) - Rn - L(q2 - q)
        st.residual_applies += 1
        w2 = krylov(dtL, [zero, zero, zero, 2.0 * dt * D])
        return q2 + w2, st
    if scheme == EXPRB42:
        a = 0.75 * dt
        w1 = krylov(lambda x: a * L(x), [zero, a * Rn])
        q2 = q + w1
        D = dg.residual(mesh, q2).reshape(-1) - Rn - L(q2 - q)
        st.residual_applies += 1
        w2 = krylov(dtL, [zero, dt * Rn, zero, (32.0 / 9.0) * dt * D])
        return q + w2, st
    raise ValueError("unknown scheme")


def advance(mesh, q, dt, nsteps, **kw):
    """nsteps exponential steps of size dt; returns (q, [StepStats])."""
    allst = []
    for _ in range(nsteps):
        q, st = step(mesh, q, dt, **kw)
        allst.append(st)
    return q, allst
