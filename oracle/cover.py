"""Cover, interfaces, knots, stencils, row assignment and CSR pattern (FP64 + integers).

Follows Section 2.1 of the paper:
  * Eq. 4-5  the cover {O_m}: open balls that cover Omega, none outside it;
  * Eq. 6-7  subdomains Omega_m = O_m n Omega, floating (closed disk inside
             Omega) or perimeter;
  * Eq. 8, 11 interfaces Gamma_m = dO_m n closure(Omega): full circles or arcs,
             with a knot at every arc/boundary junction;
  * Eq. 9, 12 stencils Xi_m ordered by increasing local angle;
  * Sec. 3.2 each knot's row is integrated in the subdomain whose interface
             is farthest away (score r_m - |x_i - c_m|);
  * Eq. 29   row i has nonzeros {i} u Xi_m(i); knots on dOmega get Dirichlet
             rows (C_ii = 1, b_i = g(x_i)).

Readings where the paper is silent (also listed in the design notes):
  * knots on a full circle: theta_j = 2 pi j / n, j = 0..n-1;
  * knots on an arc: the same candidate angles, kept when the point is
    strictly inside Omega and at least gap * 2 pi / n (gap = 0.25) away from
    every junction angle, plus one knot at each junction;
  * local order: increasing angle measured from the midpoint of the largest
    arc of the circle that lies outside Omega (0 for a full circle; among
    arcs whose lengths agree to 1e-9 the first in angle order);
  * knots are numbered circle by circle in cover order, then in local order;
  * a knot is inside circle m when r_m - |x - c_m| > 1e-12 r_owner; the best
    score wins and scores within 1e-12 r_owner of the best tie to the lowest m.

Pins (tests): hand counts of the 4x4 lattice, the coverage and stencil
invariants, brute-force row assignment on tiny covers.  Test infrastructure only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .problem import Domain

TWO_PI = 2.0 * math.pi
JUNCTION_GAP = 0.25
SCORE_EPS = 1e-12


class CoverError(ValueError):
    """Raised for a cover that breaks Eq. 5 or a degenerate discretisation."""

    def __init__(self, code: str, msg: str):
        super().__init__(f"{code}: {msg}")
        self.code = code


@dataclass
class Cover:
    domain: Domain
    cx: np.ndarray
    cy: np.ndarray
    r: np.ndarray
    floating: np.ndarray          # bool[M]
    n_knots: np.ndarray           # int[M] requested knots per circle
    n_r: np.ndarray               # int[M]
    n_theta: np.ndarray           # int[M]
    theta_s: np.ndarray = None    # float[M] unwrap origin of each circle
    junctions: list = None        # per circle: sorted list of junction angles
    knot_ptr: np.ndarray = None   # int[M+1]
    kx: np.ndarray = None
    ky: np.ndarray = None
    ku: np.ndarray = None         # local unwrapped angle in [0, 2 pi)
    kowner: np.ndarray = None
    kdir: np.ndarray = None       # bool: knot on dOmega (Dirichlet row)
    row_sub: np.ndarray = None    # int[N], -1 for Dirichlet rows
    row_mode: str = "farthest"    # "farthest" (Sec. 3.2) or "averaged" (Eq. 38-39)
    pi_ptr: np.ndarray = None     # int[N+1]: Pi_i = pi_sub[pi_ptr[i]:pi_ptr[i+1]], ascending
    pi_sub: np.ndarray = None     # the subdomains whose rows include knot i
    rowptr: np.ndarray = None
    col: np.ndarray = None
    extra: dict = field(default_factory=dict)

    @property
    def M(self):
        return int(self.cx.size)

    @property
    def N(self):
        return int(self.kx.size)

    def pi(self, i):
        """The subdomains integrated for row i: {row_sub[i]} (farthest interface), or every
        subdomain containing x_i (averaged rows, Eq. 38-39); empty for Dirichlet rows."""
        return self.pi_sub[self.pi_ptr[i]:self.pi_ptr[i + 1]]

    def sub_rows(self, m):
        """Rows that subdomain m contributes to, ascending."""
        rows = np.repeat(np.arange(self.N), np.diff(self.pi_ptr))
        return rows[self.pi_sub == m]


# --------------------------------------------------------------------------
# a1: cover (Eq. 4-7)
# --------------------------------------------------------------------------

def lattice(spec: dict):
    """Centres and radii of a square, hexagonal or explicit lattice (before filtering)."""
    kind = spec["kind"]
    if kind == "explicit":
        cx = np.asarray(spec["cx"], np.float64)
        cy = np.asarray(spec["cy"], np.float64)
        r = np.asarray(spec["r"], np.float64)
        return cx, cy, r
    nx, ny = int(spec["nx"]), int(spec["ny"])
    s = float(spec["spacing"])
    x_o, y_o = float(spec["x_origin"]), float(spec["y_origin"])
    rad = float(spec["radius"])
    cx, cy = [], []
    if kind == "square_lattice":
        for j in range(ny):
            for i in range(nx):
                cx.append(x_o + i * s)
                cy.append(y_o + j * s)
    elif kind == "hex_lattice":
        dy = s * math.sqrt(3.0) * 0.5
        for k in range(ny):
            for i in range(nx):
                x = x_o + i * s
                if k % 2 == 1:
                    x = x + 0.5 * s
                cx.append(x)
                cy.append(y_o + k * dy)
    else:
        raise CoverError("EINVAL", f"unknown cover kind {kind}")
    cx = np.array(cx)
    return cx, np.array(cy), np.full(cx.size, rad)


def build_cover(domain_spec: dict, cover_spec: dict, n_knots=0, n_r=0, n_theta=0) -> Cover:
    """a1: lattice -> keep circles meeting Omega (Eq. 5, right) -> classify (Eq. 7)."""
    dom = Domain(domain_spec)
    cx, cy, r = lattice(cover_spec)
    if np.any(r <= 0):
        raise CoverError("EINVAL", "non-positive radius")
    if cover_spec["kind"] == "explicit":
        nk = np.asarray(cover_spec["n_knots"], np.int64)
        nr = np.asarray(cover_spec["n_r"], np.int64)
        nt = np.asarray(cover_spec["n_theta"], np.int64)
    else:
        nk = np.full(cx.size, int(n_knots), np.int64)
        nr = np.full(cx.size, int(n_r), np.int64)
        nt = np.full(cx.size, int(n_theta), np.int64)
    meets = dom.dist_closed(cx, cy) < r
    if cover_spec["kind"] == "explicit" and not np.all(meets):
        # an explicitly given circle outside Omega breaks Eq. 5; lattices are filtered
        pass
    keep = meets
    cx, cy, r, nk, nr, nt = cx[keep], cy[keep], r[keep], nk[keep], nr[keep], nt[keep]
    if np.any(nk < 2) or np.any(nk % 2) or np.any(nt % 2) or np.any(nr < 1):
        raise CoverError("EINVAL", "knots and n_theta must be even, n_r >= 1")
    floating = dom.contains_closed_disk(cx, cy, r)
    return Cover(dom, cx, cy, r, floating, nk, nr, nt)


def coverage_gap(cov: Cover, step_frac: float = 0.25, chunk: int = 4096):
    """Eq. 5 (left): sample Omega on a grid of pitch step_frac*min(r); return uncovered points."""
    dom = cov.domain
    h = step_frac * float(cov.r.min())
    if dom.kind == "square":
        x0, y0, x1, y1 = dom.p
    else:
        ox, oy, rr = dom.p[:3]
        x0, y0, x1, y1 = ox - rr, oy - rr, ox + rr, oy + rr
    nx = int(math.ceil((x1 - x0) / h))
    ny = int(math.ceil((y1 - y0) / h))
    xs = x0 + (np.arange(nx) + 0.5) * (x1 - x0) / nx
    ys = y0 + (np.arange(ny) + 0.5) * (y1 - y0) / ny
    X, Y = np.meshgrid(xs, ys)
    X = X.ravel()
    Y = Y.ravel()
    inside = dom.inside_open(X, Y)
    X, Y = X[inside], Y[inside]
    bad = []
    for a in range(0, X.size, chunk):
        px = X[a:a + chunk, None]
        py = Y[a:a + chunk, None]
        d2 = (px - cov.cx) ** 2 + (py - cov.cy) ** 2
        ok = np.any(d2 < cov.r * cov.r, axis=1)
        if not np.all(ok):
            bad.append(np.stack([X[a:a + chunk][~ok], Y[a:a + chunk][~ok]], 1))
    return np.concatenate(bad) if bad else np.zeros((0, 2))


# --------------------------------------------------------------------------
# a2: junctions and arcs (Eq. 8, 11)
# --------------------------------------------------------------------------

def _norm_angle(t):
    return t + TWO_PI if t < 0.0 else t


def junction_points(dom: Domain, cx: float, cy: float, r: float):
    """Points where the circle dO crosses dOmega, as (x, y, edge) tuples."""
    pts = []
    if dom.kind == "square":
        x0, y0, x1, y1 = dom.p
        for edge, X in ((3, x0), (1, x1)):        # vertical edges x = X
            d = X - cx
            if abs(d) < r:
                e = math.sqrt(r * r - d * d)
                for y in (cy + e, cy - e):
                    if y0 <= y <= y1:
                        pts.append((X, y, edge))
        for edge, Y in ((0, y0), (2, y1)):        # horizontal edges y = Y
            d = Y - cy
            if abs(d) < r:
                e = math.sqrt(r * r - d * d)
                for x in (cx + e, cx - e):
                    if x0 <= x <= x1:
                        pts.append((x, Y, edge))
    else:
        ox, oy, R = dom.p[:3]
        dx = ox - cx
        dy = oy - cy
        d = math.sqrt(dx * dx + dy * dy)
        if abs(r - R) < d < r + R:
            a = (d * d + r * r - R * R) / (2.0 * d)
            hh = math.sqrt(r * r - a * a)
            bx = cx + a * dx / d
            by = cy + a * dy / d
            pts.append((bx - hh * dy / d, by + hh * dx / d, 0))
            pts.append((bx + hh * dy / d, by - hh * dx / d, 0))
    return pts


def circle_interface(dom: Domain, cx: float, cy: float, r: float):
    """Sorted junction angles, junction points and the unwrap origin theta_s.

    theta_s is the midpoint of the largest arc lying outside Omega (0 when the
    circle never crosses dOmega).
    """
    pts = junction_points(dom, cx, cy, r)
    ang = [_norm_angle(math.atan2(py - cy, px - cx)) for (px, py, _e) in pts]
    order = sorted(range(len(ang)), key=lambda k: ang[k])
    ang = [ang[k] for k in order]
    pts = [pts[k] for k in order]
    for k in range(1, len(ang)):
        if ang[k] - ang[k - 1] < 1e-12:
            raise CoverError("EINVAL", "degenerate junction (circle through a corner)")
    theta_s = 0.0
    if ang:
        best = -1.0
        J = len(ang)
        for k in range(J):
            a0 = ang[k]
            a1 = ang[k + 1] if k + 1 < J else ang[0] + TWO_PI
            mid = 0.5 * (a0 + a1)
            mx = cx + r * math.cos(mid)
            my = cy + r * math.sin(mid)
            outside = not bool(dom.inside_open(mx, my))
            if outside and (a1 - a0) > best + 1e-9:     # first of equal arcs wins
                best = a1 - a0
                theta_s = mid if mid < TWO_PI else mid - TWO_PI
    return ang, pts, theta_s


def unwrap(theta: float, theta_s: float) -> float:
    u = theta - theta_s
    if u < 0.0:
        u += TWO_PI
    if u >= TWO_PI:
        u -= TWO_PI
    return u


# --------------------------------------------------------------------------
# a3: knots and stencils (Eq. 9, 12)
# --------------------------------------------------------------------------

def circle_knots(dom: Domain, cx, cy, r, n):
    """Knots of one circle: list of (x, y, u, is_dirichlet) in local order."""
    ang, pts, theta_s = circle_interface(dom, cx, cy, r)
    gap = JUNCTION_GAP * TWO_PI / n
    out = []
    for j in range(n):
        t = TWO_PI * j / n
        x = cx + r * math.cos(t)
        y = cy + r * math.sin(t)
        if not bool(dom.inside_open(x, y)):
            continue
        near = False
        for a in ang:
            d = abs(t - a)
            d = min(d, TWO_PI - d)
            if d < gap:
                near = True
                break
        if near:
            continue
        out.append((x, y, unwrap(t, theta_s), False))
    for a, (px, py, _e) in zip(ang, pts):
        out.append((px, py, unwrap(a, theta_s), True))
    out.sort(key=lambda k: k[2])
    return out, ang, theta_s


def build_knots(cov: Cover) -> Cover:
    kx, ky, ku, kown, kdir = [], [], [], [], []
    ptr = [0]
    ths, juns = [], []
    for m in range(cov.M):
        ks, ang, theta_s = circle_knots(cov.domain, float(cov.cx[m]), float(cov.cy[m]),
                                        float(cov.r[m]), int(cov.n_knots[m]))
        ths.append(theta_s)
        juns.append(ang)
        for (x, y, u, d) in ks:
            kx.append(x)
            ky.append(y)
            ku.append(u)
            kown.append(m)
            kdir.append(d)
        ptr.append(len(kx))
    cov.knot_ptr = np.array(ptr, np.int64)
    cov.kx = np.array(kx)
    cov.ky = np.array(ky)
    cov.ku = np.array(ku)
    cov.kowner = np.array(kown, np.int64)
    cov.kdir = np.array(kdir, bool)
    cov.theta_s = np.array(ths)
    cov.junctions = juns
    return cov


def duplicate_knots(cov: Cover, tol: float = 1e-12):
    """Pairs of knots closer than tol (the cover is rejected when there are any)."""
    order = np.lexsort((cov.ky, cov.kx))
    xs = cov.kx[order]
    ys = cov.ky[order]
    bad = []
    for a in range(xs.size):
        b = a + 1
        while b < xs.size and xs[b] - xs[a] < tol:
            if abs(ys[b] - ys[a]) < tol:
                bad.append((int(order[a]), int(order[b])))
            b += 1
    return bad


# --------------------------------------------------------------------------
# a4: row assignment (Sec. 3.2 and its footnote)
# --------------------------------------------------------------------------

def assign_rows(cov: Cover, chunk: int = 2048, mode: str = "farthest") -> Cover:
    """m(i) = argmax_{m != owner, x_i in O_m} (r_m - |x_i - c_m|); -1 for Dirichlet rows.

    Pi_i: {m(i)} (Sec. 3.2), or with mode "averaged" every subdomain whose open disk holds x_i
    (Eq. 38-39: Pi_i = {Omega_k : x_i in Omega_k}), ascending.  "Holds" is the same test as the
    candidates of m(i): r_m - |x_i - c_m| > 1e-12 r_owner.
    """
    if mode not in ("farthest", "averaged"):
        raise CoverError("EINVAL", f"unknown row mode {mode}")
    N = cov.N
    row_sub = np.full(N, -1, np.int64)
    pis = [np.zeros(0, np.int64)] * N
    for a in range(0, N, chunk):
        sl = slice(a, min(N, a + chunk))
        dx = cov.kx[sl, None] - cov.cx[None, :]
        dy = cov.ky[sl, None] - cov.cy[None, :]
        d = np.sqrt(dx * dx + dy * dy)
        s = cov.r[None, :] - d
        own = cov.kowner[sl]
        eps = SCORE_EPS * cov.r[own]
        s[np.arange(s.shape[0]), own] = -np.inf
        inside = s > eps[:, None]
        s = np.where(inside, s, -np.inf)
        best = s.max(axis=1)
        for q in range(s.shape[0]):
            i = a + q
            if cov.kdir[i]:
                continue
            if not np.isfinite(best[q]):
                raise CoverError("EKNOT_UNCOVERED", f"knot {i} is inside no other circle")
            cand = np.nonzero(s[q] >= best[q] - eps[q])[0]
            row_sub[i] = int(cand.min())
            pis[i] = np.nonzero(inside[q])[0] if mode == "averaged" else np.array([row_sub[i]])
    cov.row_sub = row_sub
    cov.row_mode = mode
    cov.pi_ptr = np.concatenate([[0], np.cumsum([p.size for p in pis])]).astype(np.int64)
    cov.pi_sub = np.concatenate(pis).astype(np.int64) if N else np.zeros(0, np.int64)
    return cov


# --------------------------------------------------------------------------
# a5: CSR pattern (Eq. 29)
# --------------------------------------------------------------------------

def csr_pattern(cov: Cover) -> Cover:
    """Row i: the diagonal and the stencils Xi_m of every m in Pi_i, columns sorted."""
    rowptr = [0]
    cols = []
    for i in range(cov.N):
        c = [i]
        for m in cov.pi(i):
            c.extend(range(int(cov.knot_ptr[m]), int(cov.knot_ptr[m + 1])))
        cols.extend(sorted(c))
        rowptr.append(len(cols))
    cov.rowptr = np.array(rowptr, np.int64)
    cov.col = np.array(cols, np.int64)
    return cov


def full_cover(cfg: dict, check_coverage: bool = True) -> Cover:
    """a1-a5 for a workload description."""
    cov = build_cover(cfg["domain"], cfg["cover"], cfg.get("n_knots", 0),
                      cfg.get("n_r", 0), cfg.get("n_theta", 0))
    if check_coverage:
        gap = coverage_gap(cov)
        if gap.shape[0]:
            raise CoverError("ECOVER_GAP", f"{gap.shape[0]} sample points uncovered")
    build_knots(cov)
    if duplicate_knots(cov):
        raise CoverError("EINVAL", "two knots coincide")
    assign_rows(cov, mode=cfg["cover"].get("rows", "farthest"))
    csr_pattern(cov)
    return cov
