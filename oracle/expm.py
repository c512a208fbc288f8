"""Dense matrix exponential, FP64, by scaling and squaring.

exp(H) = (exp(H / 2^s))^(2^s) with s the smallest non-negative integer for
which ||H / 2^s||_1 <= 1/2, and exp(X) of the scaled matrix summed as the
Taylor polynomial of degree 18 (Horner form).  For ||X||_1 <= 1/2 the
truncation error is below 0.5^19/19! < 1e-22 relative to ||exp(X)||.  This is
the plain method of Moler & Van Loan ("Nineteen dubious ways", method 3 with
squaring); the paper's Krylov solvers (Sec. 2.3, refs. Sidje; Al-Mohy &
Higham; Niesen & Wright; KIOPS) each use a dense exponential of this kind on
the small projected matrix.

Test infrastructure only (see ``oracle/__init__``).
"""

import math
import numpy as np

TAYLOR_DEGREE = 18


def scaling_exponent(H):
    nrm = float(np.max(np.sum(np.abs(H), axis=0))) if H.size else 0.0
    if nrm <= 0.5:
        return 0
    return int(math.ceil(math.log2(nrm / 0.5)))


def expm(H):
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    s = scaling_exponent(H)
    X = H / (2.0 ** s)
    E = np.eye(n)
    for k in range(TAYLOR_DEGREE, 0, -1):
        E = np.eye(n) + (X @ E) / k
    for _ in range(s):
        E = E @ E
    return E


def phi_scalar(i, z):
    """Scalar phi_i(z) from the paper's integral definition
    phi_i(z) = int_0^1 e^{(1-t) z} t^{i-1}/(i-1)! dt (Sec. 2.3), evaluated
    through phi_{i+1}(z) = (phi_i(z) - 1/i!)/z for |z| > 1 and by its power
    series sum_k z^k/(k+i)! otherwise (the recurrence is cancellation-prone
    near 0)."""
    z = complex(z)
    if abs(z) > 1.0:
        val = np.exp(z)
        for k in range(i):
            val = (val - 1.0 / math.factorial(k)) / z
        return val
    val = 0.0
    term_fact = 1.0 / math.factorial(i)
    zk = 1.0 + 0j
    for k in range(40):
        val += zk / math.factorial(k + i)
        zk *= z
    del term_fact
    return val
