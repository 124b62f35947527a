"""IMQ radial-basis cardinal functions on perimeter arcs (a10), Eq. 19-22.

  phi_j(t) = ((t - t_j)^2 + c^2)^(-1/2)          Eq. 19
  K_lk     = phi_k(t_l)                          Eq. 20 (symmetric, positive definite)
  H_j(t)   = sum_l (K^-1)_lj phi_l(t)            Eq. 22

Reading of Eq. 19: theta measures length along the interface (arclength
s = r theta, in the units of Omega), so c has the units of length; with the
paper's c^2 = 1.5 on its radius-9, 44-knot circles, c is about one knot
spacing and K is well conditioned (kappa ~ 50), as Sec. 2.2 states.  Since
phi_l(s) = r^-1 ((u - u_l)^2 + c^2/r^2)^(-1/2) for the local angle u, and the
cardinal functions of Eq. 22 do not change when the basis is scaled, the
functions below take the local unwrapped angles u and c^2 / r^2 (angle_c2).
K is inverted through its Cholesky factor.

Pins (tests): the Kronecker property Eq. 14, exact reproduction of any
function in the span of {phi_l}, and agreement with a 50-digit solve.
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def angle_c2(c2, r):
    """c^2 of Eq. 19 (squared length) as a squared angle on a circle of radius r."""
    return float(c2) / (float(r) * float(r))


def imq(t, tj, c2):
    t = np.asarray(t, np.float64)
    d = t[..., None] - np.asarray(tj, np.float64)
    return 1.0 / np.sqrt(d * d + c2)


def kernel_matrix(u, c2):
    return imq(u, u, c2)


def inverse(u, c2):
    """K^-1 through the Cholesky factor of K."""
    K = kernel_matrix(u, c2)
    L = np.linalg.cholesky(K)
    eye = np.eye(u.size)
    return sla.cho_solve((L, True), eye)


def cardinal(t, u, c2, Kinv=None):
    """H_j(t) for every stencil knot j (last axis)."""
    if Kinv is None:
        Kinv = inverse(u, c2)
    return imq(t, u, c2) @ Kinv


def condition(u, c2):
    s = np.linalg.svd(kernel_matrix(u, c2), compute_uv=False)
    return float(s[0] / s[-1])
