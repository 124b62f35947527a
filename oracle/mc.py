"""Monte Carlo perimeter rows (a11 path simulation in plain C, a12 finalize here).

Eq. 29-30 of the paper:
  C_ii = 1,  C_ij = -E[1{X_tau in Gamma_m} H_j(X_tau) Y_tau]  (j in Xi_m),
  r_i  = E[1{X_tau in dOmega} g(X_tau) Y_tau + Z_tau],
with H_j the IMQ cardinal functions of the arc (Eq. 22) for a perimeter
circle, or the Fourier cardinals (Eq. 18) when a floating circle is
integrated by Monte Carlo.  Because H_j = sum_l (K^-1)_lj phi_l (Eq. 22), the
paths estimate the basis moments M_l = E[1_Gamma Y_tau phi_l(u_tau)] and
C_ij = -sum_l (K^-1)_lj M_l (the same estimator, reassociated).  The standard
errors are the sample standard deviations of the per-path values divided by
sqrt(paths).

Pins (tests): the generator against an independent Philox4x32-10
implementation; exit statistics of Brownian motion from a disk (mean exit
time (R^2 - |x|^2)/2, harmonic measure = Poisson kernel); the boundary shift
against optional stopping of a harmonic function on circles cut by one and by
two edges of the square (exits on their edges); the batch-means standard error
against its chi-square law on normal samples; the adaptive path counts by
hand; constant data give unit rows up to the interpolation error.  Test
infrastructure only.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import imq
from .cover import unwrap
from .problem import Operator
from .spectral import fourier_cardinal

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mc_paths.c")
_LIB = os.path.join(_HERE, "_mc_paths.so")
_lib = None

B_KIND = {"zero": 0, "sinx_cosy": 1}
C_KIND = {"zero": 0, "quadratic": 1, "rbf": 2}
F_KIND = {"zero": 0, "one": 1, "manufactured": 2, "eq46": 3, "rbf": 4}


def build(force: bool = False) -> str:
    """Compile the path simulator with gcc (IEEE arithmetic, no contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                               "-fno-fast-math", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("dom_kind", ctypes.c_int), ("dom", ctypes.c_double * 4),
                ("b_kind", ctypes.c_int), ("c_kind", ctypes.c_int), ("f_kind", ctypes.c_int),
                ("n_rbf", ctypes.c_int), ("rbf_x", ctypes.c_void_p), ("rbf_y", ctypes.c_void_p),
                ("rbf_w", ctypes.c_void_p), ("rbf_sigma", ctypes.c_double),
                ("n_frbf", ctypes.c_int), ("frbf_x", ctypes.c_void_p), ("frbf_y", ctypes.c_void_p),
                ("frbf_w", ctypes.c_void_p), ("frbf_sigma", ctypes.c_double)]


class _Walk(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_double), ("cy", ctypes.c_double), ("r", ctypes.c_double),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("knot", ctypes.c_uint32),
                ("sub", ctypes.c_uint32), ("seed", ctypes.c_uint64), ("h", ctypes.c_double), ("n_paths", ctypes.c_int),
                ("max_steps", ctypes.c_int), ("shift", ctypes.c_double), ("cv_degree", ctypes.c_int)]


# c0 = -zeta(1/2) / sqrt(2 pi): the Gobet-Menozzi boundary shift in units of |sigma^T n| sqrt(h)
# (the double nearest to it; a test recomputes it from the zeta function)
GM_C0 = 0.5825971579390108


def boundary_shift(mc: dict) -> float:
    """Shift of the boundaries for the stopped Euler scheme: c0 sqrt(h) with sigma = I, or 0."""
    return GM_C0 * math.sqrt(float(mc["h"])) if mc.get("boundary_shift", False) else 0.0


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.oracle_walk_knot.restype = ctypes.c_int
        _lib.oracle_philox4x32_10.restype = None
        _lib.oracle_normals.restype = None
    return _lib


def philox(ctr, key):
    """Philox4x32-10 block for a 4-word counter and 2-word key (generator tests)."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def normals(seed, knot, step, path, sub=0):
    xi = (ctypes.c_double * 2)()
    lib().oracle_normals(ctypes.c_uint64(seed), ctypes.c_uint32(knot), ctypes.c_uint32(sub),
                         ctypes.c_uint32(step), ctypes.c_uint32(path), xi)
    return xi[0], xi[1]


class PathRecords:
    """Per-path exit records of one knot."""

    def __init__(self, n, n_rbf=0, n_cv=0, n_frbf=0):
        self.side = np.zeros(n, np.int8)
        self.edge = np.zeros(n, np.int8)
        self.ex = np.zeros(n)
        self.ey = np.zeros(n)
        self.etheta = np.zeros(n)
        self.Y = np.zeros(n)
        self.Z = np.zeros(n)
        self.steps = np.zeros(n, np.int32)
        self.dY = np.zeros((n, n_rbf)) if n_rbf else None
        self.dZ = np.zeros((n, n_rbf)) if n_rbf else None
        self.Q = np.zeros((n, n_cv)) if n_cv else None        # control-variate features
        self.dZf = np.zeros((n, n_frbf)) if n_frbf else None  # dZ_tau / d(weights of f)
        self.capped = 0


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def max_steps_for(r, h):
    """Path cap 50 r^2 / h (about 100 mean exit times of the disk)."""
    return int(min(2**31 - 1, math.ceil(50.0 * r * r / h)))


def n_cv_features(degree):
    """Control-variate features for monomials of total degree 1..degree: degree (degree + 3) / 2."""
    d = int(degree)
    return d * (d + 3) // 2


def walk(op: Operator, cx, cy, r, x0, y0, knot, seed, h, n_paths, with_grad=False,
         max_steps=None, shift=0.0, sub=0, cv_degree=0) -> PathRecords:
    dom = op.domain
    nr = op.rbf_w.size if with_grad else 0
    nf = op.frbf_w.size if (with_grad and op.f_kind == "rbf") else 0
    rec = PathRecords(n_paths, nr, n_cv_features(cv_degree), nf)
    keep = [op.rbf_x, op.rbf_y, op.rbf_w, op.frbf_x, op.frbf_y, op.frbf_w]
    prob = _Problem(0 if dom.kind == "square" else 1, (ctypes.c_double * 4)(*dom.p),
                    B_KIND[op.b_kind], C_KIND[op.c_kind], F_KIND[op.f_kind],
                    int(op.rbf_w.size), _ptr(keep[0]), _ptr(keep[1]), _ptr(keep[2]),
                    op.rbf_sigma, int(op.frbf_w.size), _ptr(keep[3]), _ptr(keep[4]), _ptr(keep[5]),
                    op.frbf_sigma)
    ms = max_steps_for(r, h) if max_steps is None else int(max_steps)
    w = _Walk(cx, cy, r, x0, y0, int(knot), int(sub), int(seed), h, int(n_paths), ms, float(shift),
              int(cv_degree))
    got = lib().oracle_walk_knot(ctypes.byref(prob), ctypes.byref(w), _ptr(rec.side),
                                 _ptr(rec.edge), _ptr(rec.ex), _ptr(rec.ey), _ptr(rec.etheta),
                                 _ptr(rec.Y), _ptr(rec.Z), _ptr(rec.steps), _ptr(rec.dY),
                                 _ptr(rec.dZ), _ptr(rec.Q), _ptr(rec.dZf))
    if got == -2:
        raise ValueError("control-variate degree above 4")
    if got < 0:
        raise ValueError("too many RBF terms for the path derivative buffer")
    rec.capped = got
    return rec


class McRow:
    """Monte Carlo estimates of one row: stencil columns, C entries, b, SE, raw moments."""

    def __init__(self, cols, vals, b, se, se_b, moments, steps, records, Kinv, u_stencil):
        self.cols = cols
        self.vals = vals
        self.b = b
        self.se = se
        self.se_b = se_b
        self.moments = moments
        self.steps = steps
        self.records = records
        self.Kinv = Kinv
        self.u_stencil = u_stencil


def batch_mean_se(per_path, bsamp, batches=32):
    """Standard errors by batch means (path p in batch p mod 32), largest over the row's entries."""
    P = bsamp.size
    bid = np.arange(P) % batches
    nb = np.bincount(bid, minlength=batches).astype(np.float64)
    out = []
    for v in list(per_path.T) + [bsamp]:
        sums = np.bincount(bid, weights=v, minlength=batches)
        mean = sums.sum() / P
        bm = np.where(nb > 0, sums / np.maximum(nb, 1), 0.0)
        f = nb / P
        out.append(np.sqrt(batches / (batches - 1) * np.sum(f * f * (bm - mean) ** 2)))
    return max(out)


def control_variate_coef(Q, payoffs):
    """Regression coefficients of the per-path payoffs on the control-variate features:
    beta = Cov(Q)^-1 Cov(Q, P) (covariances normalised by the path count), one column per
    payoff.  Any beta leaves the estimator's mean unchanged (E[Q] = 0); this one minimises the
    variance over the sample (Milstein and Tretyakov's regression method, with beta from the
    same paths: a bias of order 1/paths)."""
    n = Q.shape[0]
    qm = Q.mean(0)
    covq = Q.T @ Q / n - np.outer(qm, qm)
    covqp = Q.T @ payoffs / n - np.outer(qm, payoffs.mean(0))
    return np.linalg.solve(covq, covqp)


def adaptive_paths(P0, Pmax, se, target):
    """Path count of the adaptive rule: a row whose largest standard error se is at most the
    target keeps its P0 pilot paths; otherwise ceil(P0 (se/target)^2) rounded up to a
    multiple of 32, capped at Pmax."""
    if not se > target:
        return P0
    want = math.ceil(P0 * (se / target) ** 2)
    want = ((want + 31) // 32) * 32
    return min(want, Pmax)


def mc_row(cov, op: Operator, i: int, m: int, mc: dict, c2: float, basis: str = "imq",
           with_grad=False, Kinv=None) -> McRow:
    """a11 + a12 for knot i integrated in subdomain m (c2: c^2 of Eq. 19, angles in radians).

    With mc["paths_max"] > mc["paths"] and mc["se_target"] > 0 the pilot of
    mc["paths"] paths is followed, when the row's largest batch-means standard
    error exceeds the target, by a run of adaptive_paths(...) paths on the same
    streams (path ids 0.. continue the pilot's).
    """
    P0 = int(mc["paths"])
    row = _mc_row_paths(cov, op, i, m, mc, c2, basis, with_grad, Kinv, P0)
    Pmax = int(mc.get("paths_max", 0))
    tgt = float(mc.get("se_target", 0.0))
    if Pmax > P0 and tgt > 0.0:
        need = adaptive_paths(P0, Pmax, batch_mean_se(row.per_path, row.bsamp), tgt)
        if need > P0:
            row = _mc_row_paths(cov, op, i, m, mc, c2, basis, with_grad, row.Kinv, need)
    return row


def _sub_index(cov, i, m):
    """Position of m in Pi_i (the Philox counter word that keeps the paths of a row's
    subdomains independent when the row averages several, Eq. 38-39); 0 otherwise."""
    if getattr(cov, "pi_ptr", None) is None:
        return 0
    hit = np.nonzero(cov.pi(i) == m)[0]
    return int(hit[0]) if hit.size else 0


def _mc_row_paths(cov, op: Operator, i: int, m: int, mc: dict, c2: float, basis, with_grad, Kinv, P) -> McRow:
    cx, cy, r = float(cov.cx[m]), float(cov.cy[m]), float(cov.r[m])
    cvd = int(mc.get("cv_degree", 0))
    rec = walk(op, cx, cy, r, float(cov.kx[i]), float(cov.ky[i]), i, int(mc["seed"]),
               float(mc["h"]), P, with_grad=with_grad, max_steps=mc.get("max_steps") or None,
               shift=boundary_shift(mc), sub=_sub_index(cov, i, m), cv_degree=cvd)
    if rec.capped:
        raise RuntimeError(f"EPATH_CAP: {rec.capped} paths of knot {i} hit the step cap")
    a, b = int(cov.knot_ptr[m]), int(cov.knot_ptr[m + 1])
    cols = np.arange(a, b)
    us = cov.ku[a:b]
    gam = rec.side == 0
    bnd = rec.side == 1
    gvals = np.zeros(P)
    if np.any(bnd):
        gvals[bnd] = op.g(rec.ex[bnd], rec.ey[bnd], rec.edge[bnd].astype(np.int64))
    bsamp = np.where(bnd, gvals * rec.Y, 0.0) + rec.Z
    if basis == "imq":
        if Kinv is None and us.size:
            Kinv = imq.inverse(us, c2)
        ut = np.array([unwrap(t, float(cov.theta_s[m])) for t in rec.etheta])
        phi = imq.imq(ut, us, c2) if us.size else np.zeros((P, 0))
        phi = np.where(gam[:, None], phi, 0.0)
        moments = (phi * rec.Y[:, None]).sum(0) / P
        vals = -(Kinv.T @ moments) if us.size else np.zeros(0)
        per_path = -(phi @ Kinv) * rec.Y[:, None] if us.size else np.zeros((P, 0))
    else:
        n = b - a
        tk = 2.0 * math.pi * np.arange(n) / n
        H = fourier_cardinal(rec.etheta, tk, n)
        H = np.where(gam[:, None], H, 0.0)
        moments = (H * rec.Y[:, None]).sum(0) / P
        vals = -moments
        per_path = -H * rec.Y[:, None]
    row_beta = None
    if cvd:
        # regression control variate on every payoff (the basis moments and r's payoff): the
        # corrected per-path payoff is P - Q beta, whose mean is mean(P) - beta^T mean(Q)
        mpp = (phi if basis == "imq" else H) * rec.Y[:, None]
        beta = control_variate_coef(rec.Q, np.concatenate([mpp, bsamp[:, None]], 1))
        mcorr = mpp - rec.Q @ beta[:, :-1]
        moments = mcorr.sum(0) / P
        bsamp = bsamp - rec.Q @ beta[:, -1]
        if basis == "imq":
            if us.size:
                vals = -(Kinv.T @ moments)
                per_path = -(mcorr @ Kinv)
        else:
            vals = -moments
            per_path = -mcorr
        row_beta = beta
    bval = bsamp.sum() / P
    se = per_path.std(0, ddof=1) / math.sqrt(P) if P > 1 else np.zeros(b - a)
    se_b = float(bsamp.std(ddof=1) / math.sqrt(P)) if P > 1 else 0.0
    row = McRow(cols, vals, float(bval), se, se_b, moments, int(rec.steps.sum()), rec, Kinv, us)
    row.per_path = per_path
    row.bsamp = bsamp
    row.paths = P
    row.cv_beta = row_beta
    return row


def mc_rows(cov, op: Operator, rows, mc: dict, c2: float, threads: int = 1, basis=None,
            with_grad=False):
    """Monte Carlo rows for a list of knots i (integrated in their subdomain row_sub[i], keyed
    by i) or of pairs (i, m) (knot i integrated in subdomain m, keyed by (i, m))."""
    Kcache = {}

    def pair(item):
        if isinstance(item, tuple):
            return int(item[0]), int(item[1]), item
        return int(item), int(cov.row_sub[item]), int(item)

    def kinv(m):
        if m not in Kcache:
            a, b = int(cov.knot_ptr[m]), int(cov.knot_ptr[m + 1])
            Kcache[m] = imq.inverse(cov.ku[a:b], c2) if b > a else np.zeros((0, 0))
        return Kcache[m]

    def one(item):
        i, m, key = pair(item)
        bas = basis or ("fourier" if cov.floating[m] else "imq")
        Kinv = kinv(m) if bas == "imq" else None
        return key, mc_row(cov, op, i, m, mc, c2, bas, with_grad, Kinv)

    lib()
    if threads <= 1:
        return dict(one(item) for item in rows)
    # build the IMQ inverses first so the worker threads only read the cache
    for item in rows:
        i, m, _ = pair(item)
        if not cov.floating[m] and (basis or "imq") == "imq":
            kinv(m)
    with ThreadPoolExecutor(threads) as ex:
        return dict(ex.map(one, rows))
