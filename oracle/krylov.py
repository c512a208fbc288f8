"""Krylov evaluation of the phi-function sum, FP64.

Computes  w = sum_{i=0}^{P} phi_i(A) c_i  (the sum of
Eq. linear_combination_of_phifunctions, Sec. 2.3, with the factors
dt^i folded into c_i) for a linear operator A given only through x -> A x.

Construction (Sec. 2.3: "an augmented matrix is constructed and projected
onto a small Krylov subspace"; refs. Sidje, Al-Mohy & Higham, Niesen &
Wright, KIOPS):

  A_hat = [[A, eta W], [0, J]],  W = [c_P, c_{P-1}, ..., c_1],
  J = P x P upper shift (ones on the superdiagonal),
  top block of exp(A_hat) [c_0; e_P / eta]  =  sum_i phi_i(A) c_i.

The paper runs KIOPS with "empirically determined" parameters (Sec. 2.3
footnote) and prints no algorithm, so this oracle fixes the following
reading (shared, decision for decision, with the GPU path):

* Arnoldi with modified Gram-Schmidt on A_hat, Euclidean inner product over
  all N + P entries, start vector b = [c_0; e_P/eta], beta = ||b||.
* Or, with a window iop >= 1, the incomplete orthogonalisation procedure that
  KIOPS puts in place of Arnoldi (Sec. 1): step j orthogonalises A_hat v_j
  (modified Gram-Schmidt) against v_{j-iop+1}, ..., v_j only, so H_m is
  banded upper Hessenberg and V_m is orthonormal only within each window.
  The projected approximation and the error estimate below are used
  unchanged.  iop >= m_max is full Arnoldi.
* Projected approximation exp(A_hat) b ~ beta V_m exp(H_m) e_1, checked at
  m = m_step, 2 m_step, ..., m_max with Saad's estimate
  err = beta h_{m+1,m} |e_m^T exp(H_m) e_1|; accepted when err <= tol beta.
  A happy breakdown (h_{m+1,m} <= 1e-13 ||A_hat v_m||) is accepted at once.
* Sub-stepping when m_max is reached: the recurrence behind
  b_i = sum_j (t^n)^j/j! v_{i+j} (Sec. 2.3) applied to
  w(s) = sum_i s^i phi_i(s A) c_i, which solves
  w' = A w + sum_{j<P} s^j/j! c_{j+1}, w(0) = c_0, gives
    w(s + sigma) = sum_i sigma^i phi_i(sigma A) chat_i,
    chat_0 = w(s),  chat_i = sum_{j=0}^{P-i} s^j/j! c_{i+j}.
  A rejected attempt halves sigma; after an accepted sub-step with
  m <= m_max/2, sigma doubles; sigma never passes 1 - s.  All sigma are
  powers of two, so s reaches 1 exactly.
* Tail scale eta = 2^(-round(log2 max_i ||sigma^i chat_i||)) (1 if all are 0):
  a power of two, so the scaling is exact; the result does not depend on it.

Every accepted sub-step is recorded as (sigma, m, eta); ``phi_sum`` can
replay such a trace (no decisions taken) for decision-free comparisons.

Test infrastructure only (see ``oracle/__init__``).
"""

import math
from dataclasses import dataclass, field
import numpy as np

from .expm import expm

BREAKDOWN_REL = 1e-13


class KrylovError(RuntimeError):
    pass


@dataclass
class KrylovStats:
    iterations: int = 0          # Arnoldi iterations (= operator applies), incl. rejected attempts
    substeps: int = 0            # accepted sub-steps
    rejected: int = 0            # attempts that reached m_max without acceptance
    err_est: float = 0.0         # error estimate of the last accepted sub-step
    trace: list = field(default_factory=list)   # [(sigma, m, eta)] accepted sub-steps


def tail_scale(vecs):
    nrm = max((float(np.linalg.norm(v)) for v in vecs), default=0.0)
    if nrm == 0.0 or not math.isfinite(nrm):
        return 1.0
    return 2.0 ** (-round(math.log2(nrm)))


def _arnoldi_expm(apply_A, b, sigma, eta, m_max, m_step, tol, fixed_m=None, iop=None):
    """One Krylov attempt for exp(A_hat) [b_0; e_P/eta] with A_hat built on
    sigma*A and W = [b_P, ..., b_1] (b = [b_0, b_1, ..., b_P], b_i already
    carrying sigma^i); iop: orthogonalisation window (None: full Arnoldi).
    Returns (accepted, m, top, err, iterations)."""
    P = len(b) - 1
    N = b[0].shape[0]
    n_aug = N + P
    start = np.zeros(n_aug)
    start[:N] = b[0]
    if P > 0:
        start[N + P - 1] = 1.0 / eta
    beta = float(np.linalg.norm(start))
    if beta == 0.0:
        return True, 0, np.zeros(N), 0.0, 0
    limit = m_max if fixed_m is None else fixed_m
    V = np.zeros((limit + 1, n_aug))
    H = np.zeros((limit + 1, limit))
    V[0] = start / beta
    iters = 0
    for j in range(limit):
        x, y = V[j, :N], V[j, N:]
        w = np.zeros(n_aug)
        # A_hat [x; y] = [sigma A x + eta sum_k y_k b_{P+1-k}; J y]
        w[:N] = sigma * apply_A(x)
        for k in range(1, P + 1):
            w[:N] += eta * y[k - 1] * b[P + 1 - k]
        if P > 0:
            w[N:N + P - 1] = y[1:]
        iters += 1
        wnorm0 = float(np.linalg.norm(w))
        lo = 0 if iop is None else max(0, j - iop + 1)
        for i in range(lo, j + 1):           # modified Gram-Schmidt
            H[i, j] = float(np.dot(V[i], w))
            w = w - H[i, j] * V[i]
        H[j + 1, j] = float(np.linalg.norm(w))
        m = j + 1
        breakdown = H[j + 1, j] <= BREAKDOWN_REL * wnorm0
        if not breakdown:
            V[j + 1] = w / H[j + 1, j]
        if fixed_m is not None:
            if m < fixed_m:
                if breakdown:
                    raise KrylovError("breakdown before the replayed m")
                continue
            E = expm(H[:m, :m])
            y1 = E[:, 0]
            err = 0.0 if breakdown else beta * H[m, m - 1] * abs(y1[m - 1])
            top = beta * (V[:m, :N].T @ y1)
            return True, m, top, err, iters
        if breakdown or m % m_step == 0 or m == m_max:
            E = expm(H[:m, :m])
            y1 = E[:, 0]
            err = 0.0 if breakdown else beta * H[m, m - 1] * abs(y1[m - 1])
            if breakdown or err <= tol * beta:
                top = beta * (V[:m, :N].T @ y1)
                return True, m, top, err, iters
    return False, m_max, None, float("inf"), iters


def phi_sum(apply_A, c, tol=1e-10, m_max=64, m_step=5, max_substeps=64, replay=None, iop=None):
    """w = sum_{i=0}^{P} phi_i(A) c_i by the augmented Krylov method above.

    apply_A : x -> A x (FP64 vectors of length N)
    c       : [c_0, ..., c_P]; c_0 may be all zeros
    replay  : optional list of (sigma, m, eta) to follow instead of deciding
    iop     : incomplete-orthogonalisation window (None or 0: full Arnoldi)
    Returns (w, KrylovStats)."""
    if iop is not None and iop <= 0:
        iop = None
    c = [np.asarray(ci, dtype=np.float64) for ci in c]
    P = len(c) - 1
    stats = KrylovStats()
    s = 0.0
    sigma = 1.0
    w = c[0].copy()
    k_replay = 0
    while s < 1.0:
        if replay is not None:
            if k_replay >= len(replay):
                raise KrylovError("replay trace ended before s = 1")
            sigma, m_fix, eta = replay[k_replay]
            k_replay += 1
        chat = [w] + [sum((s ** j) / math.factorial(j) * c[i + j] for j in range(P - i + 1))
                      for i in range(1, P + 1)]
        b = [chat[0]] + [(sigma ** i) * chat[i] for i in range(1, P + 1)]
        if replay is None:
            eta = tail_scale(b[1:])
            ok, m, top, err, iters = _arnoldi_expm(apply_A, b, sigma, eta, m_max, m_step, tol, iop=iop)
        else:
            ok, m, top, err, iters = _arnoldi_expm(apply_A, b, sigma, eta, m_max, m_step, tol,
                                                   fixed_m=m_fix, iop=iop)
        stats.iterations += iters
        if not ok:
            stats.rejected += 1
            if stats.rejected > max_substeps:
                raise KrylovError("no convergence within the sub-step budget")
            sigma *= 0.5
            continue
        w = top
        s += sigma
        stats.substeps += 1
        stats.err_est = err
        stats.trace.append((sigma, m, eta))
        if replay is None:
            if m <= m_max // 2:
                sigma *= 2.0
            sigma = min(sigma, 1.0 - s)
    return w, stats
