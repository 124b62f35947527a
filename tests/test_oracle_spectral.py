"""Pins of the oracle's pseudospectral floating rows (a6-a9) and IMQ cardinals (a10).

Checks against closed forms and textbook matrices: the Fourier and Chebyshev
differentiation matrices (Trefethen, Spectral Methods in MATLAB, ch. 3 and 6),
the Kronecker property (Eq. 14) and the closed form of Eq. 18, the Poisson
kernel for band-limited data, the mean exit time (R^2-|x|^2)/2, the
manufactured solution of the variable-coefficient workload, and a 50-digit
solve of the IMQ system (Eq. 19-22).
"""
import math

import numpy as np
import pytest

import workloads
from oracle import imq, problem, spectral


def test_fourier_diff_matches_textbook():
    for n in (8, 16, 32):
        h = 2 * math.pi / n
        F1, F2 = spectral.fourier_diff(n)
        i = np.arange(n)
        k = i[:, None] - i[None, :]
        off = k != 0
        T1 = np.zeros((n, n))
        T1[off] = 0.5 * (-1.0) ** k[off] / np.tan(k[off] * h / 2)
        T2 = np.full((n, n), -math.pi ** 2 / (3 * h * h) - 1.0 / 6)
        T2[off] = -0.5 * (-1.0) ** k[off] / np.sin(k[off] * h / 2) ** 2
        assert np.abs(F1 - T1).max() < 1e-12 * n
        assert np.abs(F2 - T2).max() < 1e-12 * n * n


def test_chebyshev_diff_matches_textbook():
    for N in (9, 33):
        x = spectral.cheb_points(N)
        D = spectral.lagrange_diff(x)
        c = np.ones(N + 1)
        c[0] = c[-1] = 2.0
        T = np.zeros((N + 1, N + 1))
        for i in range(N + 1):
            for j in range(N + 1):
                if i != j:
                    T[i, j] = c[i] / c[j] * (-1.0) ** (i + j) / (x[i] - x[j])
        T[0, 0] = (2 * N * N + 1) / 6.0
        T[N, N] = -(2 * N * N + 1) / 6.0
        for i in range(1, N):
            T[i, i] = -x[i] / (2 * (1 - x[i] ** 2))
        assert np.abs(D - T).max() < 1e-11 * N * N


def test_fourier_cardinal_kronecker_and_closed_form():
    n = 16
    tj = 2 * math.pi * np.arange(n) / n
    H = spectral.fourier_cardinal(tj, tj, n)
    assert np.abs(H - np.eye(n)).max() < 1e-14
    t = np.linspace(0.01, 6.2, 97)
    Ht = spectral.fourier_cardinal(t, tj, n)
    assert np.abs(Ht.sum(1) - 1.0).max() < 1e-14
    x = t[:, None] - tj[None, :]
    closed = np.sin(n * x / 2) / np.tan(x / 2) / n
    assert np.abs(Ht - closed).max() < 1e-12


def _one_disk(nr, nt, nk, R, cx, cy, ops):
    sh = spectral.DiskShape(nr, nt)
    dom = problem.Domain({"kind": "square", "p": [-5, -5, 5, 5]})
    op = problem.Operator(ops, dom)
    W, beta = spectral.disk_solve(sh, op, cx, cy, R, nk)
    return sh, op, W, beta


@pytest.mark.parametrize("nr,nt,nk", [(16, 16, 16), (8, 32, 16), (22, 44, 44)])
def test_poisson_kernel_rows(nr, nt, nk):
    R, cx, cy = 0.37, 0.2, -0.1
    sh, op, W, beta = _one_disk(nr, nt, nk, R, cx, cy,
                                {"b": "zero", "c": "zero", "f": "one", "g": "zero"})
    rng = np.random.default_rng(nr)
    for _ in range(12):
        rho, phi = rng.uniform(0, 0.97), rng.uniform(0, 2 * math.pi)
        v = spectral.disk_eval(sh, W, beta, cx, cy, R, cx + R * rho * math.cos(phi),
                               cy + R * rho * math.sin(phi))
        want = [spectral.poisson_kernel_row(nk, rho, phi, 2 * math.pi * j / nk) for j in range(nk)]
        assert np.abs(v[:nk] - want).max() < 1e-12
        # mean exit time of Brownian motion (generator Laplacian/2) from the disk
        assert abs(v[nk] - 0.5 * (R * R - (R * rho) ** 2)) < 1e-12 * max(1.0, R * R)
        # constants are reproduced: rows of C sum to 0 when c = 0
        assert abs(1.0 + v[:nk].sum()) < 1e-11     # n entries, kappa(A) ~ 1e4


def test_manufactured_variable_coefficients():
    cfg = workloads.varcoef()
    R, cx, cy, nk = 0.05, 0.93, 1.21, 32
    sh = spectral.DiskShape(32, 32)
    op = problem.Operator(cfg["op"], problem.Domain(cfg["domain"]))
    W, beta = spectral.disk_solve(sh, op, cx, cy, R, nk)
    tk = 2 * math.pi * np.arange(nk) / nk
    uk = op.u_star(cx + R * np.cos(tk), cy + R * np.sin(tk))
    rng = np.random.default_rng(5)
    for _ in range(8):
        rho, phi = rng.uniform(0, 0.95), rng.uniform(0, 2 * math.pi)
        x, y = cx + R * rho * math.cos(phi), cy + R * rho * math.sin(phi)
        v = spectral.disk_eval(sh, W, beta, cx, cy, R, x, y)
        # u(x_i) = -sum_j C_ij u_j + r_i for the exact solution (up to discretisation error)
        assert abs(-(v[:nk] @ uk) + v[nk] - op.u_star(x, y)) < 1e-10


def test_eq46_disk_reproduces_the_exact_solution():
    """Sec. 4's floating disk: radius 9, 44 knots, 22 x 44 nodes, Poisson data of Eq. 46.  The
    paper reports a maximum interior error of order 1e-12 for this solver; the row identity
    u(x_i) = -sum_j C_ij u_j + r_i holds to the knot interpolation error."""
    cfg = workloads.poisson46()
    R, cx, cy, nk = 9.0, -5.0, 15.0, 44
    sh = spectral.DiskShape(22, 44)
    op = problem.Operator(cfg["op"], problem.Domain(cfg["domain"]))
    W, beta = spectral.disk_solve(sh, op, cx, cy, R, nk)
    tk = 2 * math.pi * np.arange(nk) / nk
    uk = op.u46(cx + R * np.cos(tk), cy + R * np.sin(tk))[0]
    rng = np.random.default_rng(9)
    worst = 0.0
    for _ in range(8):
        rho, phi = rng.uniform(0, 0.95), rng.uniform(0, 2 * math.pi)
        x, y = cx + R * rho * math.cos(phi), cy + R * rho * math.sin(phi)
        v = spectral.disk_eval(sh, W, beta, cx, cy, R, x, y)
        worst = max(worst, abs(-(v[:nk] @ uk) + v[nk] - op.u46(x, y)[0]))
        # the source term matters: without r_i the identity fails by far more
        assert abs(-(v[:nk] @ uk) - op.u46(x, y)[0]) > 1e-5 or rho < 0.2
    assert worst < 1e-9, worst


def test_imq_kronecker_and_span():
    u = np.sort(np.random.default_rng(1).uniform(0, 3.0, 9))
    c2 = 1.5
    Kinv = imq.inverse(u, c2)
    tol = 10.0 * imq.condition(u, c2) * np.finfo(float).eps     # backward-stable solve
    H = imq.cardinal(u, u, c2, Kinv)
    assert np.abs(H - np.eye(u.size)).max() < tol
    # any f in span{phi_l} is reproduced: f = phi(t) . a, interpolate f(u_j)
    a = np.random.default_rng(2).standard_normal(u.size)
    t = np.linspace(u[0], u[-1], 33)
    f_at_knots = imq.imq(u, u, c2) @ a
    interp = imq.cardinal(t, u, c2, Kinv) @ f_at_knots
    assert np.abs(interp - imq.imq(t, u, c2) @ a).max() < tol * np.abs(a).sum()


def test_imq_against_50_digits():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    u = 2 * math.pi * np.arange(8) / 16
    c2 = 1.5
    K = mp.matrix(u.size, u.size)
    for a in range(u.size):
        for b in range(u.size):
            K[a, b] = 1 / mp.sqrt((mp.mpf(u[a]) - mp.mpf(u[b])) ** 2 + mp.mpf(c2))
    t = 0.77
    p = mp.matrix([1 / mp.sqrt((mp.mpf(t) - mp.mpf(x)) ** 2 + mp.mpf(c2)) for x in u])
    Hm = np.array([float(v) for v in mp.lu_solve(K, p)])
    assert np.abs(imq.cardinal(np.array([t]), u, c2)[0] - Hm).max() < 1e-12


def test_imq_reading_reaches_table1_accuracy():
    """Eq. 19 read with theta in radians (c^2 = 1.5): the IMQ interpolant of the exact solution of
    Eq. 46 along every perimeter arc of the [-50, 50]^2 cover is within 1e-4 of it, below the
    RMS error of 3.72e-5 x a few that Table 1 reports.  Read as arclength (c in length units)
    the interpolant would be off by more than 1e-2: that reading cannot reach Table 1."""
    import workloads
    from oracle import cover, imq_reading
    cfg = workloads.poisson46(paths=8)
    cov = cover.full_cover(cfg)
    rad = imq_reading.interpolation_error(cov, "radians", 1.5)
    arc = imq_reading.interpolation_error(cov, "arclength", 1.5)
    assert rad[0] < 1e-4, rad
    assert arc[0] > 1e-2, arc
