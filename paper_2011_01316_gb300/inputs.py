"""Seeded synthetic inputs: initial states and exact solutions.

This module holds no part of the DG method or the time integrator.  Its
functions map node coordinates (computed by whoever calls them) to states in
the canonical layout ``q[field, element, node]``.  They serve both the CUDA
library's tests and benchmarks and the CPU oracle's tests; neither side's
arithmetic lives here.

Workloads (shapes of the paper's test problems):

* ``burgers_sine``: u0(x) = 0.5 + sin(x) on [0, 2 pi] (1D inviscid Burgers,
  smooth until t = 1, the method-of-characteristics solution is
  ``burgers_characteristics``).
* ``isentropic_vortex``: the translating vortex of Sec. 5.2 (after Zhou & Wei)
  with strength lambda, decay alpha, free stream (u_inf, v_inf),
  rho_inf = T_inf = p_inf = 1, c_p = gamma/(gamma-1), rho = T^(1/(gamma-1)),
  p = rho T; periodic images by the minimum-image convention.
* ``density_wave``: rho = 1 + a sin(sum_d (x_d - u_d t)), constant velocity
  and pressure (an exact, periodic Euler solution).
* ``fourier_modes``: 1 + sum_k a_k sin(k x + phi_k) with seeded a_k, phi_k.
* ``random_euler_state`` / ``random_field``: seeded positive states for
  operator parity tests.
"""

import math
import numpy as np


def conservative(rho, vel, p, gamma):
    """(rho, rho u_1.., rho E) from primitives, rho E = p/(gamma-1) + rho|u|^2/2."""
    vel = [np.broadcast_to(np.asarray(u, dtype=np.float64), np.shape(rho)) for u in vel]
    ke = 0.5 * rho * sum(u * u for u in vel)
    return np.stack([rho] + [rho * u for u in vel] + [p / (gamma - 1.0) + ke])


def burgers_sine(x):
    """u0 = 0.5 + sin(x); x has shape [1, Ne, Np] (or any); returns [1, Ne, Np]."""
    x = np.asarray(x, dtype=np.float64)
    return (0.5 + np.sin(x[0]))[None]


def burgers_characteristics(x, t, u0=lambda s: 0.5 + np.sin(s), du0=lambda s: np.cos(s)):
    """Exact smooth Burgers solution u = u0(x - u t) by Newton on
    g(u) = u - u0(x - u t) (unique while 1 + t u0' > 0, i.e. t < 1 for 0.5 + sin)."""
    x = np.asarray(x, dtype=np.float64)
    u = u0(x)
    for _ in range(100):
        g = u - u0(x - u * t)
        dg = 1.0 + t * du0(x - u * t)
        du = g / dg
        u = u - du
        if np.max(np.abs(du)) < 1e-15:
            break
    return u


def _wrap(d, L):
    """Minimum-image displacement on a periodic interval of length L."""
    return d - L * np.round(d / L)


def isentropic_vortex(X, t=0.0, strength=5.0, alpha=1.0, u_inf=(1.0, 1.0), center=(5.0, 5.0),
                      lo=(0.0, 0.0), hi=(10.0, 10.0), gamma=1.4):
    """Conservative state [4, ...] of the translating isentropic vortex at time t.
    X = [x, y] coordinate arrays."""
    x, y = np.asarray(X[0], np.float64), np.asarray(X[1], np.float64)
    Lx, Ly = hi[0] - lo[0], hi[1] - lo[1]
    xt = _wrap(x - center[0] - u_inf[0] * t, Lx)
    yt = _wrap(y - center[1] - u_inf[1] * t, Ly)
    r2 = xt * xt + yt * yt
    cp = gamma / (gamma - 1.0)
    k = strength / (2.0 * math.pi)
    g = np.exp(alpha * (1.0 - r2) / 2.0)
    u = u_inf[0] - k * yt * g
    v = u_inf[1] + k * xt * g
    T = 1.0 - (1.0 / (2.0 * alpha * cp)) * k * k * g * g
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    return conservative(rho, [u, v], p, gamma)


def density_wave(X, t=0.0, amp=0.2, vel=None, pressure=1.0, gamma=1.4):
    """rho = 1 + amp sin(sum_d (x_d - vel_d t)), velocity vel, pressure const."""
    dim = len(X)
    vel = (1.0,) * dim if vel is None else tuple(vel)
    phase = sum(np.asarray(X[d], np.float64) - vel[d] * t for d in range(dim))
    rho = 1.0 + amp * np.sin(phase)
    return conservative(rho, list(vel), pressure * np.ones_like(rho), gamma)


def fourier_modes(x, rng, nmodes=4, amp_max=0.3, mean=1.0):
    """mean + sum_{k=1}^{nmodes} a_k sin(k x + phi_k), a_k ~ U[0, amp_max],
    phi_k ~ U[0, 2 pi); returns (values, (a, phi))."""
    a = rng.uniform(0.0, amp_max, nmodes)
    phi = rng.uniform(0.0, 2.0 * math.pi, nmodes)
    x = np.asarray(x, np.float64)
    val = mean + sum(a[k] * np.sin((k + 1) * x + phi[k]) for k in range(nmodes))
    return val, (a, phi)


def random_field(shape, rng, lo=-1.0, hi=1.0):
    return rng.uniform(lo, hi, size=shape)


def random_euler_state(dim, n_elem, n_node, rng, gamma=1.4, amp=0.2):
    """Seeded positive Euler state [dim+2, n_elem, n_node]: rho, p in
    [1-amp, 1+amp], velocity components in [-amp, amp] about (0.5, 0.3, 0.2)."""
    shp = (n_elem, n_node)
    rho = rng.uniform(1.0 - amp, 1.0 + amp, shp)
    p = rng.uniform(1.0 - amp, 1.0 + amp, shp)
    base = (0.5, 0.3, 0.2)
    vel = [base[d] + rng.uniform(-amp, amp, shp) for d in range(dim)]
    return conservative(rho, vel, p, gamma)
