"""Legendre-Gauss-Lobatto (LGL) reference-element tables, FP64.

The paper evaluates its DG integrals with LGL quadrature (Sec. 4, first
paragraph) on nodal tensor-product elements.  The formulas below are the
textbook ones for LGL collocation:

* nodes r_0 < ... < r_p: the endpoints -1, +1 and the p-1 roots of P_p'(r);
* weights w_i = 2 / (p (p+1) P_p(r_i)^2);
* differentiation matrix of the Lagrange basis on those nodes,
  D_ij = P_p(r_i) / (P_p(r_j) (r_i - r_j)) for i != j,
  D_00 = -p(p+1)/4, D_pp = +p(p+1)/4, other diagonal entries 0.

Test infrastructure only (see ``oracle/__init__``).
"""

import math
import numpy as np


def legendre(p, r):
    """P_p(r) and P_{p-1}(r) by the three-term recurrence
    (n+1) P_{n+1} = (2n+1) r P_n - n P_{n-1}."""
    r = np.asarray(r, dtype=np.float64)
    pm1 = np.ones_like(r)
    if p == 0:
        return pm1, np.zeros_like(r)
    pn = r.copy()
    for n in range(1, p):
        pm1, pn = pn, ((2 * n + 1) * r * pn - n * pm1) / (n + 1)
    return pn, pm1


def nodes(p):
    """LGL nodes on [-1, 1], ascending.  Interior nodes are the roots of
    P_p'; found by Newton's method on P_p' with P_p'' taken from Legendre's
    differential equation, started from the Chebyshev-Gauss-Lobatto points."""
    if p < 1:
        raise ValueError("LGL needs p >= 1")
    r = -np.cos(np.pi * np.arange(p + 1) / p)
    interior = r[1:-1].copy()
    for _ in range(100):
        pn, pm1 = legendre(p, interior)
        d1 = p * (interior * pn - pm1) / (interior ** 2 - 1.0)      # P_p'
        d2 = (2.0 * interior * d1 - p * (p + 1) * pn) / (1.0 - interior ** 2)  # P_p''
        step = d1 / d2
        interior = interior - step
        if np.max(np.abs(step), initial=0.0) < 1e-16:
            break
    r[1:-1] = interior
    r[0], r[-1] = -1.0, 1.0
    # exact symmetry r_i = -r_{p-i}
    r = 0.5 * (r - r[::-1])
    return r


def weights(p):
    """LGL quadrature weights w_i = 2 / (p(p+1) P_p(r_i)^2)."""
    r = nodes(p)
    pn, _ = legendre(p, r)
    return 2.0 / (p * (p + 1) * pn ** 2)


def diff_matrix(p):
    """Nodal differentiation matrix D_ij = l_j'(r_i) on the LGL nodes."""
    r = nodes(p)
    pn, _ = legendre(p, r)
    D = np.zeros((p + 1, p + 1))
    for i in range(p + 1):
        for j in range(p + 1):
            if i != j:
                D[i, j] = pn[i] / (pn[j] * (r[i] - r[j]))
    D[0, 0] = -p * (p + 1) / 4.0
    D[p, p] = p * (p + 1) / 4.0
    return D


def endpoint_weight(p):
    """w_0 = w_p = 2 / (p (p+1)); the LGL lift factor is 1/w_0."""
    return 2.0 / (p * (p + 1))


def min_node_spacing(p):
    """Smallest distance between neighbouring LGL nodes on [-1, 1]
    (the dx of the paper's Courant number, Sec. 5 footnote, on the
    reference element)."""
    r = nodes(p)
    return float(np.min(np.diff(r)))


def factorial(n):
    return float(math.factorial(n))
