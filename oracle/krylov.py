"""Global solve C u = r (a13).

The paper solves with right-preconditioned GMRES (Eq. 45).  The oracle solves
directly: a dense LU for small systems, SuperLU (scipy) otherwise; both are
library primitives whose residual the tests check.  A plain restarted GMRES
(Saad and Schultz) with modified Gram-Schmidt is also given, as the textbook
iteration, for the tests of the Krylov stopping rule, with an optional right
preconditioner: the one-level restricted additive Schwarz operator of
Eq. 42-44 (ras_subsets, ras_operator).
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def solve(C, b, dense_limit: int = 5000):
    C = sp.csr_matrix(C)
    if C.shape[0] <= dense_limit:
        return sla.solve(C.toarray(), b)
    return spla.spsolve(C.tocsc(), b)


def solve_transpose(C, rhs, dense_limit: int = 5000):
    C = sp.csr_matrix(C)
    if C.shape[0] <= dense_limit:
        return sla.solve(C.toarray().T, rhs)
    return spla.spsolve(C.T.tocsc(), rhs)


def ras_subsets(knot_ptr, row_sub):
    """The overlapping subsets w_p of Sec. 4 (Eq. 42).  The paper partitions the graph of C
    without overlap (METIS) and then adds the neighbouring entries; here the nonoverlapping part
    of subset p is the set of rows the row assignment of Sec. 3.2 gives to subdomain p, and the
    neighbours of those rows in the graph of C are their columns other than themselves: the knots
    of circle p (Eq. 29).  w_p lists the owned rows, then p's knots."""
    knot_ptr = np.asarray(knot_ptr)
    row_sub = np.asarray(row_sub)
    W = []
    for p in range(knot_ptr.size - 1):
        own = np.nonzero(row_sub == p)[0]
        knots = np.arange(knot_ptr[p], knot_ptr[p + 1])
        if own.size + knots.size:
            W.append(np.concatenate([own, knots]).astype(np.int64))
    return W


def ras_operator(C, W):
    """M_RAS^-1 = sum_p R_p^T D_p C_p^-1 R_p (Eq. 44) with C_p = R_p C R_p^T (Eq. 42) and the
    partition of unity (D_p)_ii = 1 / #{q : x_i in w_q} (Eq. 43).  Returns (apply, mult)."""
    C = sp.csr_matrix(C)
    n = C.shape[0]
    mult = np.zeros(n)
    for w in W:
        mult[w] += 1.0
    if np.any(mult == 0):
        raise ValueError("the subsets do not cover every row")
    blocks = [(w, np.linalg.inv(C[w][:, w].toarray()), 1.0 / mult[w]) for w in W]

    def apply(v):
        y = np.zeros(n)
        for w, Cinv, d in blocks:
            y[w] += d * (Cinv @ v[w])
        return y

    return apply, mult


def gmres(C, b, restart: int = 50, rtol: float = 1e-13, max_iters: int = 10000, M=None):
    """Restarted GMRES(m) with modified Gram-Schmidt and Givens rotations; with M (a callable
    v -> M^-1 v) it solves C M^-1 (M u) = b, the right-preconditioned form of Eq. 45."""
    C = sp.csr_matrix(C)
    Minv = M if M is not None else (lambda v: v)
    n = b.size
    x = np.zeros(n)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, 0.0
    it = 0
    while it < max_iters:
        r = b - C @ x
        beta = np.linalg.norm(r)
        if beta / bn <= rtol:
            return x, it, beta / bn
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        V[0] = r / beta
        g = np.zeros(restart + 1)
        g[0] = beta
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        k_used = 0
        for k in range(restart):
            w = C @ Minv(V[k])
            for j in range(k + 1):
                H[j, k] = w @ V[j]
                w = w - H[j, k] * V[j]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0:
                V[k + 1] = w / H[k + 1, k]
            for j in range(k):
                t = cs[j] * H[j, k] + sn[j] * H[j + 1, k]
                H[j + 1, k] = -sn[j] * H[j, k] + cs[j] * H[j + 1, k]
                H[j, k] = t
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k] = H[k, k] / den
            sn[k] = H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            it += 1
            k_used = k + 1
            if abs(g[k + 1]) / bn <= rtol or it >= max_iters:
                break
        y = sla.solve_triangular(H[:k_used, :k_used], g[:k_used])
        x = x + Minv(V[:k_used].T @ y)
    r = b - C @ x
    return x, it, np.linalg.norm(r) / bn
