"""Adjoint gradient of a misfit J(u) with respect to the RBF weights of c and f and g's coefficients (a14).

The paper has no gradient; this restates the standard discrete adjoint of the
assembled system.  With C(theta) u = r(theta) and lambda solving
C^T lambda = dJ/du,

    dJ/dtheta = lambda^T (dr/dtheta - (dC/dtheta) u).

Row by row:
  * Dirichlet rows: r_i = g(x_i), so d/da_k = psi^g_k(x_i).
  * Floating rows (Eq. 33, 35): the disk's local solution with interface data
    u_hat = sum_j H_j u_j is V = B - sum_j G_j u_j, solving A V = -A_IB beta - f.
    A depends on c's weights (through c at the nodes) and the right-hand side on
    f's, so sum_i lambda_i dV(x_i)/dw_q = -z^T diag(psi_q * active) V and
    sum_i lambda_i dV(x_i)/dv_q = -z^T psi^f_q with A^T z = sum_i lambda_i E_i
    (one transposed disk solve per disk).
  * Perimeter rows (Eq. 29-30): the paths do not depend on c, only the weight
    Y_tau = prod_k (1 + c(X_k) h) and Z_tau do (pathwise derivative under common
    random numbers):  d/dw_q of E[(1_dOmega g + 1_Gamma u_hat) Y + Z] is
    E[(1_dOmega g + 1_Gamma u_hat) dY_q + dZ_q]; d/da_k is E[1_dOmega psi^g_k Y]; f's
    weights enter Z_tau = sum_k f(X_k) Y_k h only: d/dv_q is E[sum_k psi^f_q(X_k) Y_k h].
  * c = min(0, sum_p w_p psi_p): the derivative carries the indicator of sum < 0.

Pins (tests): central finite differences of J with the same Philox streams.
Test infrastructure only.
"""
from __future__ import annotations

import math

import numpy as np

from . import imq
from . import krylov
from . import spectral
from .cover import unwrap


def eval_vector(shape, rho, phi):
    """E_I (n) and E_B (n_theta) with value = E_I . W + E_B . beta (see spectral.disk_eval)."""
    nr, nt, nc = shape.n_r, shape.n_t, shape.nc
    half = nt // 2
    lr, st = spectral.eval_weights(shape, rho, phi)
    EI = np.zeros((nr, nt))
    EB = np.zeros(nt)
    shift = (np.arange(nt) + half) % nt
    EB += lr[0] * st
    for l in range(1, nr + 1):
        EI[l - 1] += lr[l] * st
    for l in range(nr + 1, nc):
        EI[nc - l - 1][shift] += lr[l] * st
    EB[shift] += lr[nc] * st
    return EI.ravel(), EB


def gradient(cfg, system, u, dJdu):
    """(dJ/dw, dJ/da, lambda, dJ/dv): RBF weights of c, boundary Fourier coefficients of g, the
    adjoint solution, RBF weights of f."""
    cov = system.cov
    op = system.op
    C = system.csr()
    lam = krylov.solve_transpose(C, dJdu)
    n_w = op.rbf_w.size
    n_g = op.g_coef.size
    n_f = op.frbf_w.size if op.f_kind == "rbf" else 0
    gw = np.zeros(n_w)
    ga = np.zeros(n_g)
    gf = np.zeros(n_f)
    # Dirichlet rows
    dirich = np.nonzero(cov.row_sub < 0)[0]
    if n_g and op.g_kind == "boundary_fourier" and dirich.size:
        e = op.nearest_edge(cov.kx[dirich], cov.ky[dirich])
        s = cov.domain.arclength(cov.kx[dirich], cov.ky[dirich], e)
        ga += lam[dirich] @ op.g_fourier_basis(s)
    # floating rows
    shapes = {}
    by_disk = {}
    for i in system.fl_rows:
        by_disk.setdefault(int(cov.row_sub[i]), []).append(i)
    for m, rows in by_disk.items():
        nr, nt, nk = int(cov.n_r[m]), int(cov.n_theta[m]), int(cov.n_knots[m])
        key = (nr, nt)
        if key not in shapes:
            shapes[key] = spectral.DiskShape(nr, nt)
        shape = shapes[key]
        cx, cy, R = float(cov.cx[m]), float(cov.cy[m]), float(cov.r[m])
        A, AB = spectral.disk_operator(shape, op, cx, cy, R)
        Hmat = spectral.boundary_data(shape, nk)
        uX = u[cov.knot_ptr[m]:cov.knot_ptr[m + 1]]
        beta = Hmat @ uX
        X, Y = spectral.node_xy(shape, cx, cy, R)
        V = np.linalg.solve(A, -AB @ beta - op.f(X, Y))
        e = np.zeros(shape.n)
        for i in rows:
            dx = cov.kx[i] - cx
            dy = cov.ky[i] - cy
            rho = math.sqrt(dx * dx + dy * dy) / R
            phi = math.atan2(dy, dx)
            EI, _EB = eval_vector(shape, rho, phi)
            e += lam[i] * EI
        z = np.linalg.solve(A.T, e)
        if n_w and op.c_kind == "rbf":
            psi = op.rbf_psi(X, Y)
            active = (psi @ op.rbf_w < 0.0).astype(np.float64)
            gw -= (z * V * active) @ psi
        if n_f:
            gf -= z @ op.frbf_psi(X, Y)
    # perimeter rows
    c2 = float(cfg.get("imq_c2", 1.5))
    for i, row in system.mc_rows.items():
        m = int(cov.row_sub[i])
        rec = row.records
        P = rec.side.size
        gam = rec.side == 0
        bnd = rec.side == 1
        uX = u[row.cols]
        if cov.floating[m]:
            n = row.cols.size
            tk = 2.0 * math.pi * np.arange(n) / n
            H = spectral.fourier_cardinal(rec.etheta, tk, n)
        else:
            ut = np.array([unwrap(t, float(cov.theta_s[m])) for t in rec.etheta])
            H = imq.imq(ut, row.u_stencil, c2) @ row.Kinv if row.cols.size else np.zeros((P, 0))
        uhat = np.where(gam, H @ uX if row.cols.size else 0.0, 0.0)
        gv = np.zeros(P)
        if np.any(bnd):
            gv[bnd] = op.g(rec.ex[bnd], rec.ey[bnd], rec.edge[bnd].astype(np.int64))
        payoff = np.where(bnd, gv, 0.0) + uhat
        if n_w and rec.dY is not None:
            gw += lam[i] * (payoff @ rec.dY + rec.dZ.sum(0)) / P
        if n_f and rec.dZf is not None:
            gf += lam[i] * rec.dZf.sum(0) / P
        if n_g and op.g_kind == "boundary_fourier" and np.any(bnd):
            s = cov.domain.arclength(rec.ex[bnd], rec.ey[bnd], rec.edge[bnd].astype(np.int64))
            ga += lam[i] * (rec.Y[bnd] @ op.g_fourier_basis(s)) / P
    return gw, ga, lam, gf
