"""Pins of the oracle's problem data and cover/knot/row/CSR steps (a1-a5).

Checks against facts fixed by the paper and by hand, never against the oracle
itself: hand counts of the 4x4 lattice, coverage (Eq. 5), junction knots on
dOmega (Sec. 2.1), stencil order (Eq. 12), a brute-force row assignment
(Sec. 3.2) and the CSR structure of Eq. 29.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import cover, problem


def _fd_residual(op, x, y, h=1e-4):
    u = problem.Operator.u_star
    uxx = (u(x + h, y) - 2 * u(x, y) + u(x - h, y)) / h ** 2
    uyy = (u(x, y + h) - 2 * u(x, y) + u(x, y - h)) / h ** 2
    ux = (u(x + h, y) - u(x - h, y)) / (2 * h)
    uy = (u(x, y + h) - u(x, y - h)) / (2 * h)
    bx, by = op.b(x, y)
    return 0.5 * (uxx + uyy) + bx * ux + by * uy + op.c(x, y) * u(x, y) + op.f(x, y)


def test_manufactured_source_solves_eq1():
    cfg = workloads.varcoef()
    op = problem.Operator(cfg["op"], problem.Domain(cfg["domain"]))
    rng = np.random.default_rng(3)
    x, y = rng.uniform(0, 2, 50), rng.uniform(0, 2, 50)
    assert np.abs(_fd_residual(op, x, y)).max() < 1e-5


def test_exp_sin_is_harmonic():
    x, y, h = 0.3, 0.7, 1e-4
    u = lambda a, b: math.exp(a) * math.sin(b)
    lap = (u(x + h, y) + u(x - h, y) + u(x, y + h) + u(x, y - h) - 4 * u(x, y)) / h ** 2
    assert abs(lap) < 1e-6


def test_eq46_solution_pins():
    """u46 of the Poisson test (Eq. 46): its value at the origin (s = 1, w = 0), the odd symmetry
    of its tanh part, and its gradient and Laplacian against central differences."""
    u46 = problem.Operator.u46
    assert abs(u46(0.0, 0.0)[0] - (3.0 + math.sin(1.0) / 3.0)) < 1e-15
    rng = np.random.default_rng(46)
    x, y = rng.uniform(-50, 50, 64), rng.uniform(-50, 50, 64)
    u, ux, uy, lap = u46(x, y)
    um = u46(-x, -y)[0]
    # sin(s) is even in (x, y), tanh(w) odd: u(x) + u(-x) = 6 + 2 sin(s) / 3
    s = np.sqrt(1.0 + x * x / 100.0 + y * y / 50.0)
    assert np.abs(u + um - 6.0 - 2.0 * np.sin(s) / 3.0).max() < 1e-14
    h = 1e-3
    f = lambda a, b: u46(a, b)[0]
    fx = (f(x + h, y) - f(x - h, y)) / (2 * h)
    fy = (f(x, y + h) - f(x, y - h)) / (2 * h)
    flap = (f(x + h, y) + f(x - h, y) + f(x, y + h) + f(x, y - h) - 4 * f(x, y)) / h ** 2
    assert np.abs(fx - ux).max() < 1e-8
    assert np.abs(fy - uy).max() < 1e-8
    assert np.abs(flap - lap).max() < 1e-6
    assert np.abs(lap).max() > 1e-2                  # the check above is not vacuous


@pytest.mark.parametrize("b,c", [("zero", "zero"), ("sinx_cosy", "quadratic")])
def test_eq46_source_solves_eq1(b, c):
    """f = -(L u46 + c u46): (1/2) Lap u + b.grad u + c u + f = 0 by central differences; with
    b = c = 0 this is the paper's Lap u = F with f = -F/2."""
    dom = problem.Domain({"kind": "square", "p": [-50.0, -50.0, 50.0, 50.0]})
    op = problem.Operator({"b": b, "c": c, "f": "eq46", "g": "eq46"}, dom)
    rng = np.random.default_rng(47)
    x, y = rng.uniform(-50, 50, 64), rng.uniform(-50, 50, 64)
    h = 1e-3
    u = lambda a, bb: problem.Operator.u46(a, bb)[0]
    uxx = (u(x + h, y) - 2 * u(x, y) + u(x - h, y)) / h ** 2
    uyy = (u(x, y + h) - 2 * u(x, y) + u(x, y - h)) / h ** 2
    ux = (u(x + h, y) - u(x - h, y)) / (2 * h)
    uy = (u(x, y + h) - u(x, y - h)) / (2 * h)
    bx, by = op.b(x, y)
    res = 0.5 * (uxx + uyy) + bx * ux + by * uy + op.c(x, y) * u(x, y) + op.f(x, y)
    assert np.abs(res).max() < 1e-6 * max(1.0, np.abs(op.c(x, y)).max())
    assert np.allclose(op.g(x, y), u(x, y), rtol=0, atol=0)


@pytest.fixture(scope="module")
def tiny_cover():
    return cover.full_cover(workloads.tiny())


def test_tiny_hand_counts(tiny_cover):
    c = tiny_cover
    assert c.M == 16
    fl = np.nonzero(c.floating)[0]
    assert sorted((round(c.cx[m], 3), round(c.cy[m], 3)) for m in fl) == \
        [(0.375, 0.375), (0.375, 0.625), (0.625, 0.375), (0.625, 0.625)]
    per = np.diff(c.knot_ptr)
    # corner circles: 7 interior candidates + 2 junctions; edge circles 11 + 2;
    # floating circles 16 (worked out by hand from the candidate angles 22.5 j deg)
    for m in range(16):
        xs, ys = c.cx[m], c.cy[m]
        corner = (xs in (0.125, 0.875)) and (ys in (0.125, 0.875))
        edge = ((xs in (0.125, 0.875)) or (ys in (0.125, 0.875))) and not corner
        want = 9 if corner else (13 if edge else 16)
        assert per[m] == want, (m, xs, ys, per[m])
    assert c.N == 4 * 9 + 8 * 13 + 4 * 16
    assert c.kdir.sum() == 24


def test_coverage_and_gap_detection(tiny_cover):
    assert cover.coverage_gap(tiny_cover).shape[0] == 0
    # drop one floating circle: its centre region is then uncovered
    cfg = workloads.tiny()
    bad = cover.build_cover(cfg["domain"], cfg["cover"], 16, 16, 16)
    keep = np.ones(bad.M, bool)
    keep[5] = False
    for f in ("cx", "cy", "r", "floating", "n_knots", "n_r", "n_theta"):
        setattr(bad, f, getattr(bad, f)[keep])
    assert cover.coverage_gap(bad).shape[0] > 0


def test_lattice_coverage_radius():
    # square lattice: the farthest point from every centre is s/sqrt(2) < r
    cfg = workloads.tiny()
    s, r = cfg["cover"]["spacing"], cfg["cover"]["radius"]
    assert s / math.sqrt(2) < r
    # hexagonal lattice: s/sqrt(3) < r
    cfg = workloads.varcoef()
    s, r = cfg["cover"]["spacing"], cfg["cover"]["radius"]
    assert s / math.sqrt(3) < r


def test_junction_knots_on_boundary_and_circle(tiny_cover):
    c = tiny_cover
    d = np.nonzero(c.kdir)[0]
    x0, y0, x1, y1 = c.domain.p
    on_edge = np.minimum.reduce([np.abs(c.kx[d] - x0), np.abs(c.kx[d] - x1),
                                 np.abs(c.ky[d] - y0), np.abs(c.ky[d] - y1)])
    assert np.all(on_edge == 0.0)
    own = c.kowner[d]
    rad = np.hypot(c.kx[d] - c.cx[own], c.ky[d] - c.cy[own])
    assert np.allclose(rad, c.r[own], rtol=0, atol=1e-15)


def test_stencils_ordered_by_local_angle(tiny_cover):
    c = tiny_cover
    for m in range(c.M):
        u = c.ku[c.knot_ptr[m]:c.knot_ptr[m + 1]]
        assert np.all(np.diff(u) > 0)
        if c.floating[m]:
            n = int(c.n_knots[m])
            assert np.allclose(u, 2 * math.pi * np.arange(n) / n, atol=0)


def test_interior_knots_strictly_inside_domain(tiny_cover):
    c = tiny_cover
    nd = ~c.kdir
    assert np.all(c.domain.inside_open(c.kx[nd], c.ky[nd]))


def _brute_force_rows(c):
    out = []
    for i in range(c.N):
        if c.kdir[i]:
            out.append(-1)
            continue
        best, arg = None, None
        eps = 1e-12 * c.r[c.kowner[i]]
        scores = []
        for m in range(c.M):
            if m == c.kowner[i]:
                continue
            s = c.r[m] - math.sqrt((c.kx[i] - c.cx[m]) ** 2 + (c.ky[i] - c.cy[m]) ** 2)
            if s > eps:
                scores.append((s, m))
        best = max(s for s, _ in scores)
        arg = min(m for s, m in scores if s >= best - eps)
        out.append(arg)
    return np.array(out)


def test_row_assignment_brute_force(tiny_cover):
    assert np.array_equal(_brute_force_rows(tiny_cover), tiny_cover.row_sub)


def test_csr_structure(tiny_cover):
    c = tiny_cover
    for i in range(c.N):
        cols = c.col[c.rowptr[i]:c.rowptr[i + 1]]
        assert np.all(np.diff(cols) > 0)
        assert i in cols
        m = c.row_sub[i]
        if m < 0:
            assert cols.size == 1
        else:
            want = set(range(c.knot_ptr[m], c.knot_ptr[m + 1])) | {i}
            assert set(cols.tolist()) == want


def test_averaged_rows_brute_force():
    """Eq. 38-39: Pi_i = every subdomain (other than the knot's own circle) whose open disk holds
    x_i, by brute force over all circles; row i of C holds the diagonal and the union of their
    stencils; the farthest-interface choice of Sec. 3.2 is one of them."""
    cfg = workloads.tiny()
    cfg["cover"]["rows"] = "averaged"
    c = cover.full_cover(cfg)
    multi = 0
    for i in range(c.N):
        got = c.pi(i).tolist()
        if c.kdir[i]:
            assert got == [] and c.row_sub[i] == -1
            continue
        own = c.kowner[i]
        want = [m for m in range(c.M) if m != own and
                c.r[m] - math.hypot(c.kx[i] - c.cx[m], c.ky[i] - c.cy[m]) > 1e-12 * c.r[own]]
        assert got == want, i
        assert c.row_sub[i] in got
        multi += len(got) > 1
        cols = c.col[c.rowptr[i]:c.rowptr[i + 1]]
        stencil = {i} | {k for m in got for k in range(c.knot_ptr[m], c.knot_ptr[m + 1])}
        assert cols.tolist() == sorted(stencil)
    assert multi > c.N // 4            # the lattice overlaps: many knots lie in two or more disks


def test_hex_workload_cover_is_valid():
    cfg = workloads.varcoef()
    c = cover.full_cover(cfg)
    assert 900 <= c.M <= 1100
    # Eq. 5 right: every circle meets Omega
    assert np.all(c.domain.dist_closed(c.cx, c.cy) < c.r)
    # every non-Dirichlet row is integrated inside a circle that contains its knot
    nd = np.nonzero(c.row_sub >= 0)[0]
    m = c.row_sub[nd]
    assert np.all(np.hypot(c.kx[nd] - c.cx[m], c.ky[nd] - c.cy[m]) < c.r[m])
    assert np.all(m != c.kowner[nd])


def test_corner_degenerate_rejected():
    dom = problem.Domain({"kind": "square", "p": [0, 0, 1, 1]})
    # a circle through the corner (0, 0): junctions coincide
    with pytest.raises(cover.CoverError):
        cover.circle_interface(dom, 0.3, 0.4, 0.5)
