"""Global solve C u = r (a13).

The paper solves with right-preconditioned GMRES (Eq. 45).  The oracle solves
directly: a dense LU for small systems, SuperLU (scipy) otherwise; both are
library primitives whose residual the tests check.  A plain restarted GMRES
(Saad and Schultz) with modified Gram-Schmidt is also given, as the textbook
iteration, for the tests of the Krylov stopping rule.
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


def gmres(C, b, restart: int = 50, rtol: float = 1e-13, max_iters: int = 10000):
    """Restarted GMRES(m) with modified Gram-Schmidt and Givens rotations."""
    C = sp.csr_matrix(C)
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
            w = C @ V[k]
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
        x = x + V[:k_used].T @ y
    r = b - C @ x
    return x, it, np.linalg.norm(r) / bn
