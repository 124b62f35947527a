"""Floating rows by Chebyshev(r) x Fourier(theta) collocation on the disk (a6-a9).

Follows Sec. 2.2 and Sec. 3.3 of the paper:
  * Eq. 18   Fourier cardinal H_j(t) = (1/n) sum_{k=-n/2}^{n/2-1} cos k(t - t_j);
  * Eq. 32   L G_j + c G_j = 0 in the disk, G_j = -H_j on the circle;
  * Eq. 35   L B + c B + f = 0 in the disk, B = 0 on the circle;
  * Eq. 33   C_ij = G_j(x_i), r_i = B(x_i) for a knot x_i assigned to the disk;
  * Eq. 40-41 one collocation matrix A for all 1 + #Xi right-hand sides,
             factored once by Householder QR and solved as R w = Q^T rhs.

The collocation is the polar construction the paper cites ([29, p.29]):
N_c = 2 n_r + 1 Chebyshev points x_k = cos(k pi / N_c) on [-1, 1]; the
unknowns sit at the n_r positive interior radii times n_theta equispaced
angles t_j = 2 pi j / n_theta; a point at negative x is the point at radius
|x| and angle t + pi.  Physical radius R scales d/dr by 1/R.  With sigma = I
the operator in polar form is

  (1/2)(u_rr + u_r/r + u_tt/r^2) + b_x (cos t u_r - sin t u_t / r)
                                 + b_y (sin t u_r + cos t u_t / r) + c u.

Readings where the paper is silent: off-grid knots are evaluated by tensor
interpolation (Lagrange in r over all N_c + 1 points, boundary values
included, then the Fourier cardinal in theta); when n_theta > n the boundary
data -H_j is sampled at the grid angles.

The differentiation matrices are built from their definitions (Lagrange
basis derivatives from the product form; Fourier ones by summing the series
of Eq. 18), not from the closed forms.

Pins (tests): the Fourier matrices against the textbook closed forms; for
L = Laplacian/2 the rows against the Poisson-kernel closed form of a
band-limited boundary datum; B for f = 1 against the mean exit time
(R^2 - |x-c|^2)/2; the manufactured solution of the variable-coefficient
workload.  Test infrastructure only.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from .problem import Operator

TWO_PI = 2.0 * math.pi


# --------------------------------------------------------------------------
# Fourier cardinal functions (Eq. 18) and their derivatives
# --------------------------------------------------------------------------

def fourier_cardinal(t, tj, n):
    """H_j(t) of Eq. 18 by the sum over k = -n/2 .. n/2-1 (n even)."""
    t = np.asarray(t, np.float64)
    x = t[..., None] - np.asarray(tj, np.float64)
    ks = np.arange(-n // 2, n // 2)
    return np.cos(x[..., None] * ks).sum(-1) / n


def fourier_diff(n):
    """D1[i, j] = H_j'(t_i), D2[i, j] = H_j''(t_i) on t_i = 2 pi i / n, from the series."""
    t = TWO_PI * np.arange(n) / n
    x = t[:, None] - t[None, :]
    ks = np.arange(-n // 2, n // 2)
    d1 = -(np.sin(x[..., None] * ks) * ks).sum(-1) / n
    d2 = -(np.cos(x[..., None] * ks) * (ks * ks)).sum(-1) / n
    return d1, d2


# --------------------------------------------------------------------------
# Chebyshev points and Lagrange basis (definition by the product form)
# --------------------------------------------------------------------------

def cheb_points(nc):
    return np.cos(math.pi * np.arange(nc + 1) / nc)


def lagrange_weights(x):
    """w_j = 1 / prod_{k != j} (x_j - x_k)."""
    n = x.size
    w = np.empty(n)
    for j in range(n):
        d = x[j] - np.delete(x, j)
        w[j] = 1.0 / np.prod(d)
    return w


def lagrange_diff(x):
    """D[i, j] = l_j'(x_i) for the Lagrange basis on the points x."""
    n = x.size
    w = lagrange_weights(x)
    D = np.empty((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (w[j] / w[i]) / (x[i] - x[j])
            else:
                D[i, i] = np.sum(1.0 / (x[i] - np.delete(x, i)))
    return D


def lagrange_eval(x, xq):
    """l_j(xq) = prod_{k != j} (xq - x_k) / (x_j - x_k) for every j."""
    n = x.size
    out = np.empty(n)
    for j in range(n):
        others = np.delete(x, j)
        out[j] = np.prod((xq - others) / (x[j] - others))
    return out


# --------------------------------------------------------------------------
# a6: the collocation operator of one disk
# --------------------------------------------------------------------------

class DiskShape:
    """Grid tables shared by every disk with the same (n_r, n_theta)."""

    def __init__(self, n_r, n_t):
        self.n_r = n_r
        self.n_t = n_t
        self.nc = 2 * n_r + 1
        self.x = cheb_points(self.nc)
        self.D = lagrange_diff(self.x)
        self.D2 = self.D @ self.D
        self.F1, self.F2 = fourier_diff(n_t)
        self.t = TWO_PI * np.arange(n_t) / n_t
        self.n = n_r * n_t


def node_xy(shape: DiskShape, cx, cy, R):
    rho = shape.x[1:shape.n_r + 1]
    X = cx + (R * rho)[:, None] * np.cos(shape.t)[None, :]
    Y = cy + (R * rho)[:, None] * np.sin(shape.t)[None, :]
    return X.ravel(), Y.ravel()


def disk_operator(shape: DiskShape, op: Operator, cx, cy, R):
    """A_II (n x n) and A_IB (n x n_theta) of the polar collocation of L + c."""
    nr, nt, nc = shape.n_r, shape.n_t, shape.nc
    n = shape.n
    A = np.zeros((n, n))
    AB = np.zeros((n, nt))
    half = nt // 2
    X, Y = node_xy(shape, cx, cy, R)
    bx, by = op.b(X, Y)
    cval = op.c(X, Y)
    for k in range(1, nr + 1):
        rho = shape.x[k]
        for j in range(nt):
            p = (k - 1) * nt + j
            ct, st = math.cos(shape.t[j]), math.sin(shape.t[j])
            alpha = 0.5 / (R * R)
            beta = 0.5 / (R * R * rho) + (bx[p] * ct + by[p] * st) / R
            gamma = 0.5 / (R * R * rho * rho)
            delta = (-bx[p] * st + by[p] * ct) / (R * rho)
            for l in range(nc + 1):
                wl = alpha * shape.D2[k, l] + beta * shape.D[k, l]
                if l == 0:
                    AB[p, j] += wl
                elif l <= nr:
                    A[p, (l - 1) * nt + j] += wl
                elif l < nc:
                    A[p, (nc - l - 1) * nt + (j + half) % nt] += wl
                else:
                    AB[p, (j + half) % nt] += wl
            A[p, (k - 1) * nt:(k - 1) * nt + nt] += gamma * shape.F2[j] + delta * shape.F1[j]
            A[p, p] += cval[p]
    return A, AB


def boundary_data(shape: DiskShape, n_knots):
    """Hmat[j'', j] = H_j(t_j'') for the disk's knots t_j = 2 pi j / n_knots."""
    tk = TWO_PI * np.arange(n_knots) / n_knots
    return fourier_cardinal(shape.t, tk, n_knots)


# --------------------------------------------------------------------------
# a7-a8: factor once (Householder QR, Eq. 41) and solve all right-hand sides
# --------------------------------------------------------------------------

def disk_solve(shape: DiskShape, op: Operator, cx, cy, R, n_knots):
    """Interior solutions W (n x (n_knots+1)) and boundary rings for every column.

    Columns 0..n_knots-1 are G_j (Eq. 32), column n_knots is B (Eq. 35).
    Returns (W, beta) with beta (n_theta x (n_knots+1)) the boundary values.
    """
    A, AB = disk_operator(shape, op, cx, cy, R)
    Hmat = boundary_data(shape, n_knots)
    X, Y = node_xy(shape, cx, cy, R)
    beta = np.concatenate([-Hmat, np.zeros((shape.n_t, 1))], 1)
    rhs = -AB @ beta
    rhs[:, n_knots] -= op.f(X, Y)
    Q, Rm = np.linalg.qr(A)
    W = sla.solve_triangular(Rm, Q.T @ rhs)
    return W, beta


# --------------------------------------------------------------------------
# a9: evaluate at a knot
# --------------------------------------------------------------------------

def eval_weights(shape: DiskShape, rho, phi):
    """Radial Lagrange values l_l(rho), l = 0..N_c, and angular H_j'(phi)."""
    lr = lagrange_eval(shape.x, rho)
    st = fourier_cardinal(phi, shape.t, shape.n_t)
    return lr, st


def disk_eval(shape: DiskShape, W, beta, cx, cy, R, xq, yq):
    """Values of every column's solution at (xq, yq) inside the disk."""
    nr, nt, nc = shape.n_r, shape.n_t, shape.nc
    half = nt // 2
    dx = xq - cx
    dy = yq - cy
    rho = math.sqrt(dx * dx + dy * dy) / R
    phi = math.atan2(dy, dx)
    lr, st = eval_weights(shape, rho, phi)
    ncol = W.shape[1]
    V = np.zeros((nt, ncol))          # V[j'] = sum_l l_l(rho) U_l(j')
    Wg = W.reshape(nr, nt, ncol)
    shift = (np.arange(nt) + half) % nt
    V += lr[0] * beta
    for l in range(1, nr + 1):
        V += lr[l] * Wg[l - 1]
    for l in range(nr + 1, nc):
        V += lr[l] * Wg[nc - l - 1][shift]
    V += lr[nc] * beta[shift]
    return st @ V


def floating_rows(cov, op: Operator, m: int, shapes: dict | None = None):
    """C entries and b for every row assigned to floating disk m.

    Returns {i: (cols, vals, b_i)} with the stencil columns of Xi_m in order.
    """
    nr, nt, nk = int(cov.n_r[m]), int(cov.n_theta[m]), int(cov.n_knots[m])
    if shapes is None:
        shapes = {}
    key = (nr, nt)
    if key not in shapes:
        shapes[key] = DiskShape(nr, nt)
    shape = shapes[key]
    cx, cy, R = float(cov.cx[m]), float(cov.cy[m]), float(cov.r[m])
    W, beta = disk_solve(shape, op, cx, cy, R, nk)
    cols = np.arange(cov.knot_ptr[m], cov.knot_ptr[m + 1])
    out = {}
    for i in cov.sub_rows(m):
        v = disk_eval(shape, W, beta, cx, cy, R, float(cov.kx[i]), float(cov.ky[i]))
        out[int(i)] = (cols, v[:nk].copy(), float(v[nk]))
    return out


def poisson_kernel_row(n, rho, phi, tj):
    """Closed form of G_j at (rho, phi) for L = Laplacian/2 and data -H_j (band-limited)."""
    ks = np.arange(1, n // 2)
    x = phi - tj
    s = 1.0 + 2.0 * np.sum(rho ** ks * np.cos(ks * x)) + rho ** (n // 2) * math.cos(n // 2 * x)
    return -s / n
