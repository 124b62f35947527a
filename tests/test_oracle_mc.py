"""Pins of the oracle's Monte Carlo rows (a11-a12), Krylov solve (a13) and adjoint (a14).

* The Philox4x32-10 generator against an independent library implementation
  (Triton's, run by its CPU interpreter in a child process).
* Normal draws: moments and (uniform) marginals.
* Brownian exit from a disk (generator Laplacian/2): E[tau] = (R^2 - rho^2)/2
  and the harmonic measure of a band-limited datum = the Poisson kernel,
  within 4 standard errors plus the Euler-Maruyama exit bias bound.
* g = 1, f = c = 0: every perimeter row satisfies 1 + sum_j C_ij = r_i up to
  the IMQ interpolation error of the constant.
* The direct solve's residual; GMRES against the direct solve.
* The RAS preconditioner (Eq. 42-45): partition of unity, M^-1 = I when C = I,
  M^-1 = C^-1 when one subset holds every knot, and right-preconditioned GMRES
  against the direct solve in fewer iterations than plain GMRES.
* The adjoint gradient (weights of c and f, coefficients of g) against central finite
  differences (common random numbers).
"""
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import adjoint, cover, imq, krylov, mc, problem, system

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_philox_against_library_implementation():
    pytest.importorskip("triton")
    cases = [((0, 0, 0, 0), (0, 0)), ((7, 3, 0, 0), (0, 12)), ((123456, 42, 0, 0), (99, 31337)),
             ((0xffffffff, 0xffffffff, 0, 0), (0xffffffff, 0xffffffff))]
    prog = textwrap.dedent("""
        import os, sys, json
        os.environ["TRITON_INTERPRET"] = "1"
        import torch, triton, triton.language as tl
        @triton.jit
        def k(out, seed, c0, c1):
            z = c1 * 0
            a, b, c, d = tl.philox(seed, c0, c1, z, z, n_rounds=10)
            tl.store(out + 0, a); tl.store(out + 1, b); tl.store(out + 2, c); tl.store(out + 3, d)
        def s32(v):
            return v - (1 << 32) if v >= (1 << 31) else v
        res = []
        for (ctr, key) in json.loads(sys.argv[1]):
            out = torch.zeros(4, dtype=torch.int32)
            seed = (key[1] << 32) | key[0]
            k[(1,)](out, seed, s32(ctr[0]), s32(ctr[1]))
            res.append([v & 0xffffffff for v in out.tolist()])
        print(json.dumps(res))
    """)
    import json
    try:
        outp = subprocess.run([sys.executable, "-c", prog, json.dumps(cases)], capture_output=True,
                              text=True, timeout=600, env={**os.environ, "TRITON_INTERPRET": "1"})
    except subprocess.TimeoutExpired:
        pytest.skip("library Philox did not finish")
    if outp.returncode != 0:
        pytest.skip("library Philox unavailable: " + outp.stderr[-300:])
    ref = json.loads(outp.stdout.strip().splitlines()[-1])
    for (ctr, key), want in zip(cases, ref):
        assert mc.philox(ctr, key) == want


def test_philox_avalanche_and_uniformity():
    base = mc.philox((5, 9, 0, 0), (0, 1))
    flips = []
    for bit in range(32):
        o = mc.philox((5 ^ (1 << bit), 9, 0, 0), (0, 1))
        flips.append(sum(bin(a ^ b).count("1") for a, b in zip(base, o)))
    assert 40 < np.mean(flips) < 88            # ~64 of 128 bits change
    xs = np.array([mc.normals(0, 3, s, p) for s in range(200) for p in range(100)])
    assert abs(xs.mean()) < 0.02
    assert abs(xs.var() - 1.0) < 0.02
    assert abs(np.mean(xs[:, 0] * xs[:, 1])) < 0.02


def _disk_cover(R=0.3, n=16, ops=None):
    cfg = workloads.floating_only_disk(R, n, 16, 16)
    if ops:
        cfg["op"] = ops
    cov = cover.build_cover(cfg["domain"], cfg["cover"])
    cover.build_knots(cov)
    return cfg, cov


def test_mean_exit_time_from_disk():
    cfg, cov = _disk_cover()
    op = problem.Operator({"b": "zero", "c": "zero", "f": "one", "g": "zero"}, cov.domain)
    R = cov.r[0]
    for rho in (0.0, 0.5, 0.8):
        h = 1e-5
        x0 = cov.cx[0] + R * rho
        rec = mc.walk(op, cov.cx[0], cov.cy[0], R, x0, cov.cy[0], 7, 0, h, 4000)
        est, se = rec.Z.mean(), rec.Z.std(ddof=1) / math.sqrt(rec.Z.size)
        exact = 0.5 * (R * R - (R * rho) ** 2)
        # Euler-Maruyama overshoots the exit by O(sqrt h) in space: bias <= 2 R sqrt(h)
        assert abs(est - exact) < 4 * se + 2 * R * math.sqrt(h)
        assert np.all(rec.side == 0)


def test_boundary_shift_removes_the_exit_bias():
    """Gobet-Menozzi: stopping at the disk shrunk by c0 sqrt(h) (c0 = -zeta(1/2)/sqrt(2 pi)) takes
    the mean exit time's O(sqrt h) overshoot down to O(h).  At sqrt(h) = R/10 the plain scheme
    overshoots by ~10 % of (R^2 - rho^2)/2; the shifted one is within 4 SE + 2 h."""
    cfg, cov = _disk_cover()
    op = problem.Operator({"b": "zero", "c": "zero", "f": "one", "g": "zero"}, cov.domain)
    R = cov.r[0]
    h = (0.1 * R) ** 2
    shift = mc.boundary_shift({"h": h, "boundary_shift": True})
    from scipy.special import zeta
    assert abs(mc.GM_C0 - (-zeta(0.5)) / math.sqrt(2.0 * math.pi)) <= 2e-16
    assert abs(shift - mc.GM_C0 * 0.1 * R) < 1e-15
    for rho in (0.0, 0.5):
        x0 = cov.cx[0] + R * rho
        exact = 0.5 * (R * R - (R * rho) ** 2)
        plain = mc.walk(op, cov.cx[0], cov.cy[0], R, x0, cov.cy[0], 7, 3, h, 40000)
        shifted = mc.walk(op, cov.cx[0], cov.cy[0], R, x0, cov.cy[0], 7, 3, h, 40000, shift=shift)
        bias_p = plain.Z.mean() - exact
        bias_s = shifted.Z.mean() - exact
        se = shifted.Z.std(ddof=1) / math.sqrt(shifted.Z.size)
        assert bias_p > 0.05 * exact, (rho, bias_p)
        assert abs(bias_s) < 4 * se + 2 * h, (rho, bias_s, se)
        # exit points lie on the circle itself (projection onto the true boundary)
        d = np.hypot(shifted.ex - cov.cx[0], shifted.ey - cov.cy[0])
        assert np.abs(d - R).max() < 1e-12


def test_boundary_shift_on_the_square_edges():
    """Gobet-Menozzi projection onto the domain's edges (the paths of a perimeter circle that
    leave through dOmega): with L = Laplacian/2, f = c = 0 and the harmonic u = e^x sin y,
    optional stopping gives E[u(X_tau)] = u(x0) for the exact exit law.  On a circle cut by one
    edge and on a corner circle cut by two, at sqrt(h) = r/10, the shifted scheme scored at its
    projected exit points is within 4 SE + h of u(x0), while the plain scheme shows its
    O(sqrt h) bias (> 5 SE).  Every exit through dOmega lies exactly on the edge it records,
    inside the closed square, and every interface exit lies on the circle."""
    dom = problem.Domain({"kind": "square", "p": [0.0, 0.0, 1.0, 1.0]})
    op = problem.Operator({"b": "zero", "c": "zero", "f": "zero", "g": "exp_sin"}, dom)
    edge_value = {0: ("y", 0.0), 1: ("x", 1.0), 2: ("y", 1.0), 3: ("x", 0.0)}
    # (circle, start): one cut by the bottom edge, one cut by the left and bottom edges
    for (cx, cy, r), (x0, y0), want_edges in (((0.5, 0.1, 0.3), (0.45, 0.12), {0}),
                                              ((0.1, 0.1, 0.3), (0.12, 0.15), {0, 3})):
        h = (0.1 * r) ** 2
        shift = mc.boundary_shift({"h": h, "boundary_shift": True})
        u0 = math.exp(x0) * math.sin(y0)
        plain = mc.walk(op, cx, cy, r, x0, y0, 7, 3, h, 100000)
        shifted = mc.walk(op, cx, cy, r, x0, y0, 7, 3, h, 100000, shift=shift)
        us = np.exp(shifted.ex) * np.sin(shifted.ey)
        up = np.exp(plain.ex) * np.sin(plain.ey)
        se = us.std(ddof=1) / math.sqrt(us.size)
        assert abs(us.mean() - u0) < 4 * se + h, (cx, cy, us.mean(), u0, se)
        assert up.mean() - u0 > 5 * se, (cx, cy, up.mean(), u0, se)
        side1 = shifted.side == 1
        assert 0.2 < side1.mean() < 0.8
        assert set(np.unique(shifted.edge[side1]).tolist()) == want_edges
        for e, (axis, v) in edge_value.items():
            sel = side1 & (shifted.edge == e)
            coord = shifted.ey if axis == "y" else shifted.ex
            assert np.all(coord[sel] == v), e
        assert np.all((shifted.ex[side1] >= 0.0) & (shifted.ex[side1] <= 1.0))
        assert np.all((shifted.ey[side1] >= 0.0) & (shifted.ey[side1] <= 1.0))
        side0 = shifted.side == 0
        d = np.hypot(shifted.ex[side0] - cx, shifted.ey[side0] - cy)
        assert np.abs(d - r).max() < 1e-12


def test_batch_mean_standard_error():
    """The batch-means standard error (path p in batch p mod 32) on i.i.d. N(mu, s^2) samples:
    with equal batches, 31 (SE / (s / sqrt(P)))^2 is chi-square with 31 degrees of freedom.
    Every replicate lies inside its 1e-6 quantiles, and the mean of (SE / (s / sqrt(P)))^2
    over 4000 replicates is 1 within 5 of its standard deviations (a wrong degrees-of-freedom
    factor, 32/31, is 6 of them).  The estimator reports the largest SE over the row's
    columns and its right-hand side."""
    from scipy.stats import chi2
    rng = np.random.default_rng(11)
    P, s = 32 * 40, 2.5
    lo, hi = chi2.ppf(1e-6, 31) / 31, chi2.ppf(1 - 1e-6, 31) / 31
    ratios = []
    for _ in range(4000):
        x = 3.0 + s * rng.standard_normal(P)
        se = mc.batch_mean_se(np.zeros((P, 0)), x)
        ratios.append((se / (s / math.sqrt(P))) ** 2)
    ratios = np.array(ratios)
    assert np.all((ratios > lo) & (ratios < hi)), (ratios.min(), ratios.max())
    sd = math.sqrt(2.0 / 31.0) / math.sqrt(ratios.size)
    assert abs(ratios.mean() - 1.0) < 5 * sd, ratios.mean()
    # the largest over the columns and the right-hand side
    a = rng.standard_normal(P)
    cols = np.stack([0.01 * a, 10.0 * a], 1)
    assert mc.batch_mean_se(cols, 0.1 * a) == pytest.approx(mc.batch_mean_se(np.zeros((P, 0)), 10.0 * a), rel=1e-12)
    # a constant sample has zero standard error; batch membership is p mod 32
    assert mc.batch_mean_se(np.zeros((P, 1)), np.full(P, 4.0)) == 0.0
    y = np.where(np.arange(P) % 32 == 5, 1.0, 0.0)
    bm = np.zeros(32)
    bm[5] = 1.0
    want = math.sqrt(np.sum((bm - bm.mean()) ** 2) / 31.0 / 32.0)
    assert mc.batch_mean_se(np.zeros((P, 0)), y) == pytest.approx(want, rel=1e-12)


def test_adaptive_path_counts_by_hand():
    """The adaptive rule: a row whose largest standard error se exceeds the target reruns with
    ceil(P0 (se/target)^2) paths rounded up to a multiple of 32 and capped at paths_max; a row at
    or below the target keeps its pilot."""
    assert mc.adaptive_paths(1000, 100000, 2.0e-3, 2.0e-3) == 1000
    assert mc.adaptive_paths(1000, 100000, 1.0e-3, 2.0e-3) == 1000
    assert mc.adaptive_paths(1000, 100000, 4.0e-3, 2.0e-3) == 4000        # 1000 * 4
    assert mc.adaptive_paths(1000, 100000, 3.0e-3, 2.0e-3) == 2272        # 2250 -> 71 * 32
    assert mc.adaptive_paths(1000, 100000, 2.002e-3, 2.0e-3) == 1024      # 1002.001 -> 1003 -> 32 * 32
    assert mc.adaptive_paths(1000, 100000, 1.0, 2.0e-3) == 100000         # capped
    assert mc.adaptive_paths(1000, 5000, 1.0, 2.0e-3) == 5000
    assert mc.adaptive_paths(1000, 5010, 1.0, 2.0e-3) == 5010             # the cap itself, not rounded past it
    assert mc.adaptive_paths(64, 1000, 5.0, 1.0) == 1000                  # 64 * 25 = 1600 -> cap


def test_feynman_kac_eq46_on_a_disk():
    """Feynman-Kac (Eq. 25-27) for the Poisson test of Eq. 46 on a radius-9 disk at h = 0.015
    with the boundary shift: E[u46(X_tau) + Z_tau] = u46(x0) within 4 SE + the O(h) bias.  This
    ties the path simulator's source term to the exact solution; E[Z_tau] is far larger than
    the tolerance, so a dropped or sign-flipped source fails."""
    dom = problem.Domain({"kind": "square", "p": [-50.0, -50.0, 50.0, 50.0]})
    op = problem.Operator({"b": "zero", "c": "zero", "f": "eq46", "g": "eq46"}, dom)
    cx, cy, R, h = 12.0, -7.0, 9.0, 0.015
    shift = mc.boundary_shift({"h": h, "boundary_shift": True})
    for (x0, y0) in ((cx, cy), (cx + 4.0, cy - 3.0)):
        rec = mc.walk(op, cx, cy, R, x0, y0, 5, 2, h, 6000, shift=shift)
        score = op.u46(rec.ex, rec.ey)[0] + rec.Z
        est, se = score.mean(), score.std(ddof=1) / math.sqrt(score.size)
        tol = 4 * se + 20 * h * 1e-2
        assert abs(est - op.u46(x0, y0)[0]) < tol, (x0, y0, est, se)
        assert abs(rec.Z.mean()) > 5 * tol


def test_control_variate_on_a_disk():
    """Pathwise variance reduction (the regression control variate of Milstein and Tretyakov) on
    the Eq. 46 Feynman-Kac test of a radius-9 disk: the features
    Q = sum_k Y_k sqrt(h) grad psi(X_k) . xi_k of the monomials of degree 1..4 in the centred,
    scaled coordinates have mean zero (each within 5 SE), the corrected estimate of
    E[u46(X_tau) + Z_tau] stays within 4 SE + 2e-4 of u46(x0), and its standard error is more than
    ten times smaller than the plain one (the local solution is smooth, so low-degree
    polynomials carry most of its gradient)."""
    dom = problem.Domain({"kind": "square", "p": [-50.0, -50.0, 50.0, 50.0]})
    op = problem.Operator({"b": "zero", "c": "zero", "f": "eq46", "g": "eq46"}, dom)
    cx, cy, R, h = 12.0, -7.0, 9.0, 0.015
    shift = mc.boundary_shift({"h": h, "boundary_shift": True})
    assert mc.n_cv_features(4) == 14 and mc.n_cv_features(2) == 5
    for (x0, y0) in ((cx, cy), (cx + 4.0, cy - 3.0)):
        rec = mc.walk(op, cx, cy, R, x0, y0, 5, 2, h, 4000, shift=shift, cv_degree=4)
        plain = mc.walk(op, cx, cy, R, x0, y0, 5, 2, h, 4000, shift=shift)
        # the same paths with and without the features
        assert np.array_equal(rec.ex, plain.ex) and np.array_equal(rec.Z, plain.Z)
        score = op.u46(rec.ex, rec.ey)[0] + rec.Z
        n = score.size
        zq = np.abs(rec.Q.mean(0)) / (rec.Q.std(0, ddof=1) / math.sqrt(n))
        assert zq.max() < 5.0, zq
        beta = mc.control_variate_coef(rec.Q, score[:, None])
        corr = score - rec.Q @ beta[:, 0]
        se_p = score.std(ddof=1) / math.sqrt(n)
        se_c = corr.std(ddof=1) / math.sqrt(n)
        assert abs(corr.mean() - op.u46(x0, y0)[0]) < 4 * se_c + 2e-4, (x0, y0, corr.mean(), se_c)
        assert se_c < se_p / 10, (se_c, se_p)


def test_control_variate_rows():
    """Monte Carlo rows with the control variate (cv_degree 3) against the plain rows on the same
    streams: every C entry and r within 4 plain standard errors, and the standard errors of the
    corrected rows mostly smaller."""
    cfg = workloads.tiny(paths=800)
    cov = cover.full_cover(cfg)
    rows = [i for i in range(cov.N) if cov.row_sub[i] >= 0 and not cov.floating[cov.row_sub[i]]][:10]
    plain = system.assemble(cfg, cov, rows=rows, threads=4)
    cfg_cv = dict(cfg, mc=dict(cfg["mc"], cv_degree=3))
    cvs = system.assemble(cfg_cv, cov, rows=rows, threads=4)
    ratios = []
    for i in rows:
        p, c = plain.mc_rows[i], cvs.mc_rows[i]
        assert np.all(np.abs(c.vals - p.vals) <= 4 * p.se + 1e-12), i
        assert abs(c.b - p.b) <= 4 * p.se_b + 1e-12, i
        ok = p.se > 0
        ratios += list(c.se[ok] / p.se[ok])
    assert np.median(ratios) < 0.9, np.median(ratios)


def test_harmonic_measure_is_poisson_kernel():
    from oracle import spectral
    cfg, cov = _disk_cover()
    op = problem.Operator({"b": "zero", "c": "zero", "f": "zero", "g": "zero"}, cov.domain)
    R, n = cov.r[0], 16
    rho, phi = 0.45, 1.1
    x0, y0 = cov.cx[0] + R * rho * math.cos(phi), cov.cy[0] + R * rho * math.sin(phi)
    h = 1e-5
    rec = mc.walk(op, cov.cx[0], cov.cy[0], R, x0, y0, 11, 0, h, 6000)
    tk = 2 * math.pi * np.arange(n) / n
    H = spectral.fourier_cardinal(rec.etheta, tk, n)
    est = -H.mean(0)
    se = H.std(0, ddof=1) / math.sqrt(H.shape[0])
    want = np.array([spectral.poisson_kernel_row(n, rho, phi, t) for t in tk])
    assert np.all(np.abs(est - want) < 4 * se + 4 * math.sqrt(h))


def test_constant_data_rows():
    cfg = workloads.tiny(paths=200)
    cfg["op"] = {"b": "zero", "c": "zero", "f": "zero", "g": "one"}
    cov = cover.full_cover(cfg)
    rows = [i for i in range(cov.N) if cov.row_sub[i] >= 0 and not cov.floating[cov.row_sub[i]]][:12]
    S = system.assemble(cfg, cov, rows=rows)
    for i in rows:
        row = S.mc_rows[i]
        m = cov.row_sub[i]
        # worst interpolation error of the constant 1 over the sampled exit angles
        t = np.linspace(row.u_stencil[0], row.u_stencil[-1], 200)
        err1 = np.abs(imq.cardinal(t, row.u_stencil, cfg["imq_c2"], row.Kinv).sum(1) - 1).max()
        lhs = 1.0 + row.vals.sum()
        assert abs(lhs - row.b) <= err1 + 1e-12, (i, m, lhs, row.b)


def test_averaged_rows_special_cases():
    """Eq. 38-39 on the 4x4 lattice.  (a) Rows whose every subdomain is floating: each
    subdomain's row reproduces the harmonic e^x sin y from its knot values, so the averaged row
    does too, (C u*)_i = r_i, with C_ii = #Pi_i.  (b) Constant data on Monte Carlo pairs: each
    subdomain's part satisfies 1 + sum_j C^m_ij = r^m_i up to the IMQ interpolation error of 1.
    (c) A row's subdomains use independent streams: only the first shares the paths of the
    single-subdomain row."""
    cfg = workloads.tiny(paths=200)
    cfg["cover"]["rows"] = "averaged"
    cov = cover.full_cover(cfg)
    fl = [i for i in range(cov.N) if cov.pi(i).size >= 2 and all(cov.floating[m] for m in cov.pi(i))]
    assert fl
    S = system.assemble(cfg, cov, rows=fl)
    C = S.csr()
    ustar = np.exp(cov.kx) * np.sin(cov.ky)
    res = C @ ustar - S.b
    for i in fl:
        assert C[i, i] == cov.pi(i).size
        assert abs(res[i]) < 1e-9, (i, res[i])
    # a dropped subdomain or a diagonal of 1 would break the identity by O(1)
    assert np.abs(ustar[fl]).max() > 0.1
    # (b) constant data
    cfg1 = workloads.tiny(paths=200)
    cfg1["cover"]["rows"] = "averaged"
    cfg1["op"] = {"b": "zero", "c": "zero", "f": "zero", "g": "one"}
    cov1 = cover.full_cover(cfg1)
    pairs = [(i, int(m)) for i in range(cov1.N) for m in cov1.pi(i)
             if cov1.pi(i).size >= 2 and not cov1.floating[m]][:8]
    assert pairs
    rows = mc.mc_rows(cov1, problem.Operator(cfg1["op"], cov1.domain), pairs, cfg1["mc"], 1.5)
    for (i, m), row in rows.items():
        t = np.linspace(row.u_stencil[0], row.u_stencil[-1], 200)
        err1 = np.abs(imq.cardinal(t, row.u_stencil, cfg["imq_c2"], row.Kinv).sum(1) - 1).max()
        assert abs(1.0 + row.vals.sum() - row.b) <= err1 + 1e-12, (i, m)
    # (c) streams: the k-th subdomain of a row draws with Philox counter word 3 = k
    assert mc.normals(0, 5, 3, 7) == mc.normals(0, 5, 3, 7, sub=0)
    assert mc.normals(0, 5, 3, 7) != mc.normals(0, 5, 3, 7, sub=1)


def test_direct_and_gmres_solves():
    cfg = workloads.tiny(paths=100)
    S = system.assemble(cfg)
    C = S.csr()
    u = krylov.solve(C, S.b)
    assert np.linalg.norm(C @ u - S.b) <= 1e-13 * np.linalg.norm(S.b)
    ug, it, rel = krylov.gmres(C, S.b, restart=30, rtol=1e-13)
    assert rel <= 1e-13
    assert np.abs(ug - u).max() < 1e-11


def test_ras_preconditioner_special_cases():
    cfg = workloads.tiny(paths=100)
    cov = cover.full_cover(cfg)
    S = system.assemble(cfg, cov)
    C = S.csr()
    n = C.shape[0]
    W = krylov.ras_subsets(cov.knot_ptr, cov.row_sub)
    # every knot lies in its own circle's subset and, unless it is a Dirichlet row, in its owner's:
    # the partition of unity of Eq. 43 weighs it by 1/2 or 1
    apply, mult = krylov.ras_operator(C, W)
    want = 1.0 + (np.asarray(cov.row_sub) >= 0)
    assert np.array_equal(mult, want)
    rng = np.random.default_rng(5)
    v = rng.standard_normal(n)
    # C = I: every C_p is the identity, so M^-1 v = sum_p R_p^T D_p R_p v = v
    apply_i, _ = krylov.ras_operator(sp.identity(n, format="csr"), W)
    assert np.abs(apply_i(v) - v).max() <= 1e-15
    # a single subset holding every knot: M^-1 = C^-1
    apply_1, _ = krylov.ras_operator(C, [np.arange(n)])
    assert np.abs(apply_1(v) - np.linalg.solve(C.toarray(), v)).max() <= 1e-12 * np.abs(v).max() * 1e3


def test_ras_gmres_against_direct_solve():
    cfg = workloads.tiny(paths=100)
    cov = cover.full_cover(cfg)
    S = system.assemble(cfg, cov)
    C = S.csr()
    u = krylov.solve(C, S.b)
    apply, _ = krylov.ras_operator(C, krylov.ras_subsets(cov.knot_ptr, cov.row_sub))
    up, it_p, rel_p = krylov.gmres(C, S.b, restart=30, rtol=1e-13, M=apply)
    _, it_0, _ = krylov.gmres(C, S.b, restart=30, rtol=1e-13)
    assert rel_p <= 1e-13
    assert np.abs(up - u).max() < 1e-11
    assert it_p < it_0, (it_p, it_0)


def _J(cfg, u_obs, cov):
    S = system.assemble(cfg, cov, with_grad=True)
    u = krylov.solve(S.csr(), S.b)
    return float(np.sum((u - u_obs) ** 2)), S, u


def _fd(param, idx, eps, u_obs, cov):
    cp = workloads.grad(paths=60)
    cm = workloads.grad(paths=60)
    for c, sgn in ((cp, 1.0), (cm, -1.0)):
        if param == "w":
            c["op"]["rbf"]["w"] = c["op"]["rbf"]["w"].copy()
            c["op"]["rbf"]["w"][idx] += sgn * eps
        elif param == "v":
            c["op"]["frbf"]["w"] = c["op"]["frbf"]["w"].copy()
            c["op"]["frbf"]["w"][idx] += sgn * eps
        else:
            c["op"]["g_coef"] = c["op"]["g_coef"].copy()
            c["op"]["g_coef"][idx] += sgn * eps
    return (_J(cp, u_obs, cov)[0] - _J(cm, u_obs, cov)[0]) / (2 * eps)


def test_adjoint_against_central_differences():
    """Central differences with common random numbers.

    With step 1e-4 the truncation error is O(eps^2) and the check is tight
    (1e-6 relative).  With step 1e-6 the quotient is limited by the rounding
    of J itself (about kappa(A) u |J| ~ 4e-12 from the disk solves, divided
    by eps), so it is checked at 2e-5 relative.
    """
    cfg = workloads.grad(paths=60)
    cov = cover.full_cover(cfg)
    rng = np.random.default_rng(9)
    u_obs = np.exp(cov.kx) * np.sin(cov.ky) + 0.01 * rng.standard_normal(cov.N)
    J0, S, u = _J(cfg, u_obs, cov)
    gw, ga, _lam, gv = adjoint.gradient(cfg, S, u, 2.0 * (u - u_obs))
    assert gv.size == 16
    for param, idx, g in (("w", 0, gw), ("w", 17, gw), ("w", 40, gw), ("a", 0, ga), ("a", 5, ga),
                          ("a", 20, ga), ("v", 0, gv), ("v", 7, gv), ("v", 15, gv)):
        fd4 = _fd(param, idx, 1e-4, u_obs, cov)
        assert abs(fd4 - g[idx]) <= 1e-6 * max(1e-2, abs(fd4)), (param, idx, fd4, g[idx])
        fd6 = _fd(param, idx, 1e-6, u_obs, cov)
        assert abs(fd6 - g[idx]) <= 2e-5 * max(1e-2, abs(fd6)), (param, idx, fd6, g[idx])


def _table1():
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_poisson46.txt")
    out = {}
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_poisson46_statistics_against_table1():
    """The oracle's C for the Poisson test of Eq. 46 against the [-50,50]^2 column of Table 1.
    The circle layout is ours (the paper's figure of it is missing; radius 9 on a pitch-10
    lattice), so the statistics are compared loosely: 100 subdomains exactly, rho(C - I) within
    0.03 (an M-matrix-like C with spectral radius just below one), kappa_2(C) within a factor
    of 2, and the solution within the Monte Carlo error of 64 paths per knot (the paper's RMS
    comes from 5000 paths with variance reduction)."""
    t1 = _table1()
    cfg = workloads.poisson46(paths=64)
    cov = cover.full_cover(cfg)
    S = system.assemble(cfg, cov, threads=8)
    C = S.csr().toarray()
    assert cov.M == t1["subdomains"]
    assert abs(cov.N - t1["N"]) < 0.1 * t1["N"]
    rho = np.abs(np.linalg.eigvals(C - np.eye(cov.N))).max()
    sv = np.linalg.svd(C, compute_uv=False)
    assert abs(rho - t1["rho_C_minus_I"]) < 0.03 and rho < 1.0, rho
    assert 0.5 * t1["kappa2_C"] < sv[0] / sv[-1] < 2.0 * t1["kappa2_C"], sv[0] / sv[-1]
    u = np.linalg.solve(C, S.b)
    rms = np.sqrt(np.mean((u - problem.Operator.u46(cov.kx, cov.ky)[0]) ** 2))
    assert rms < 0.05, rms
