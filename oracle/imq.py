"""IMQ radial-basis cardinal functions on perimeter arcs (a10), Eq. 19-22.

  phi_j(t) = ((t - t_j)^2 + c^2)^(-1/2)          Eq. 19
  K_lk     = phi_k(t_l)                          Eq. 20 (symmetric, positive definite)
  H_j(t)   = sum_l (K^-1)_lj phi_l(t)            Eq. 22

Reading of Eq. 19: theta is the knots' local unwrapped angle in radians (not
scaled by the radius), with c^2 = 1.5 as in the paper's experiments (Sec. 4).
Read as arclength instead (c in length units, about one knot spacing on the
paper's radius-9 circles), K would be well conditioned (kappa ~ 46 against
~7e11), but the interpolant of the Eq. 46 solution on the perimeter arcs would
be off by 0.07, far above the RMS error of 3.7e-5 that Table 1 reports; in
radians it is off by 6e-5 (oracle/imq_reading.py).  K is inverted through its
Cholesky factor.

Pins (tests): the Kronecker property Eq. 14, exact reproduction of any
function in the span of {phi_l}, and agreement with a 50-digit solve.
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


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
