"""Pins for the oracle's LGL tables (closed forms, a library root finder,
polynomial exactness)."""
import math
import os

import numpy as np
import pytest

from oracle import lgl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lgl_closed_forms.txt")


def _golden():
    rows = {}
    env = {"sqrt": math.sqrt}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            p, x, w = (s.strip() for s in line.split("|"))
            rows.setdefault(int(p), []).append((eval(x, env), eval(w, env)))
    return rows


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_closed_forms(p):
    g = sorted(_golden()[p])
    np.testing.assert_allclose(lgl.nodes(p), [x for x, _ in g], rtol=0, atol=1e-15)
    np.testing.assert_allclose(lgl.weights(p), [w for _, w in g], rtol=1e-14, atol=0)


@pytest.mark.parametrize("p", range(1, 13))
def test_nodes_are_roots_of_dP(p):
    from numpy.polynomial import legendre as L
    r = lgl.nodes(p)
    assert r[0] == -1.0 and r[-1] == 1.0
    if p > 1:
        c = np.zeros(p + 1)
        c[p] = 1.0
        roots = np.sort(np.real(L.legroots(L.legder(c))))
        np.testing.assert_allclose(r[1:-1], roots, atol=1e-13)
    np.testing.assert_array_equal(r, -r[::-1])


@pytest.mark.parametrize("p", range(1, 13))
def test_quadrature_exactness(p):
    r, w = lgl.nodes(p), lgl.weights(p)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * p):            # LGL is exact up to degree 2p-1
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, r ** k) - exact) < 1e-13
    assert abs(w[0] - lgl.endpoint_weight(p)) < 1e-15


@pytest.mark.parametrize("p", range(1, 13))
def test_differentiation_exact_on_polynomials(p):
    r, D = lgl.nodes(p), lgl.diff_matrix(p)
    for k in range(p + 1):
        dk = k * r ** (k - 1) if k > 0 else np.zeros_like(r)
        np.testing.assert_allclose(D @ r ** k, dk, atol=1e-12 * max(1, p * p))
    # SBP: W D + (W D)^T = diag(-1, 0, ..., 0, 1)
    W = np.diag(lgl.weights(p))
    B = W @ D + (W @ D).T
    E = np.zeros_like(B)
    E[0, 0], E[-1, -1] = -1.0, 1.0
    np.testing.assert_allclose(B, E, atol=1e-13)
