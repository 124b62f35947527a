"""The interfacial system C u = r of Eq. 28-30 assembled by the oracle (a1-a12).

Row kinds:
  * Dirichlet rows (knots on dOmega, a reading of "deleting the knots on the
    boundary" in Sec. 3.1): C_ii = 1, r_i = g(x_i);
  * floating rows (Eq. 33): pseudospectral, see ``spectral``;
  * perimeter rows (Eq. 29-30): Monte Carlo, see ``mc``.
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from . import cover as cover_mod
from . import mc as mc_mod
from . import spectral
from .problem import Operator


class System:
    def __init__(self, cov, op, vals, b, se, se_b, mc_rows, fl_rows):
        self.cov = cov
        self.op = op
        self.vals = vals
        self.b = b
        self.se = se
        self.se_b = se_b
        self.mc_rows = mc_rows
        self.fl_rows = fl_rows

    def csr(self):
        import scipy.sparse as sp
        N = self.cov.N
        return sp.csr_matrix((self.vals, self.cov.col, self.cov.rowptr), shape=(N, N))


def _put_row(cov, vals, i, cols, v):
    a, b = int(cov.rowptr[i]), int(cov.rowptr[i + 1])
    rc = cov.col[a:b]
    pos = np.searchsorted(rc, cols)
    vals[a + pos] = v


def assemble(cfg: dict, cov=None, rows=None, floating_method: str = "ps", threads: int = 1,
             with_grad: bool = False) -> System:
    """Assemble C and r (all rows, or only ``rows`` when given).

    Every row sums the contributions of the subdomains in Pi_i (one subdomain, Sec. 3.2, or all
    that hold the knot, Eq. 38-39): C_ii = #Pi_i, C_ij = the sum of the subdomains' entries of
    their stencils (disjoint), r_i = the sum of their r's.  The standard error of r_i is the
    root sum of squares of the subdomains' (their paths are independent).
    """
    if cov is None:
        cov = cover_mod.full_cover(cfg)
    op = Operator(cfg["op"], cov.domain)
    N = cov.N
    rows = np.arange(N) if rows is None else np.asarray(rows)
    averaged = cov.row_mode == "averaged"
    vals = np.zeros(cov.col.size)
    se = np.zeros(cov.col.size)
    se_b = np.zeros(N)
    b = np.zeros(N)
    # the diagonal: 1 for a Dirichlet row and for one subdomain (Eq. 29), #Pi_i (Eq. 38)
    for i in rows:
        _put_row(cov, vals, i, np.array([i]), np.array([float(max(1, cov.pi(i).size))]))
    dirich = [int(i) for i in rows if cov.row_sub[i] < 0]
    if dirich:
        d = np.array(dirich)
        b[d] = op.g(cov.kx[d], cov.ky[d])
    fl_rows = {}
    mcl = []
    disks = {}
    for i in rows:
        for m in cov.pi(i):
            m = int(m)
            if cov.floating[m] and floating_method == "ps":
                disks.setdefault(m, []).append(int(i))
            else:
                mcl.append((int(i), m) if averaged else int(i))
    shapes = {}
    se_b2 = np.zeros(N)
    for m, want in disks.items():
        res = spectral.floating_rows(cov, op, m, shapes)
        for i in want:
            cols, v, bi = res[i]
            _put_row(cov, vals, i, cols, v)
            b[i] += bi
            fl_rows[(i, m) if averaged else i] = res[i]
    mc_rows = mc_mod.mc_rows(cov, op, mcl, cfg["mc"], float(cfg.get("imq_c2", 1.5)),
                             threads=threads, with_grad=with_grad) if mcl else {}
    for key, row in mc_rows.items():
        i = key[0] if averaged else key
        _put_row(cov, vals, i, row.cols, row.vals)
        _put_row(cov, se, i, row.cols, row.se)
        b[i] += row.b
        se_b2[i] += row.se_b * row.se_b
    se_b[:] = np.sqrt(se_b2)
    return System(cov, op, vals, b, se, se_b, mc_rows, fl_rows)
