"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars:
  * cover, knots, row owners, CSR pattern: bit-exact (knot coordinates to
    a few ulps: both sides call their own cos/sin);
  * floating rows (pseudospectral): <= 1e-10 relative, normwise per row, FP64
    and mixed (FP32 LU + FP64 refinement);
  * Monte Carlo rows, FP64 form on identical Philox streams: raw moments and
    b <= 1e-12 relative; C entries <= 1e-12 + 16 kappa(K) eps (the IMQ solve's
    rounding);
  * Monte Carlo rows, mixed form (FP32 positions): within 4 standard errors
    of the FP64 oracle on every entry checked (the two forms draw different
    normals), aggregate z^2 near 1;
  * u: <= 1e-10 relative against the oracle's direct solve of its own system.
"""
import math

import numpy as np
import pytest
import torch

import workloads
from oracle import cover as ocover
from oracle import imq as oimq
from oracle import krylov as okrylov
from oracle import system as osystem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pdd():
    import paper_2311_08946_gb300 as pkg
    from paper_2311_08946_gb300 import build
    build.build()
    pkg.load()
    return pkg


_cache = {}


def _oracle_cover(name, cfg):
    key = ("cover", name)
    if key not in _cache:
        _cache[key] = ocover.full_cover(cfg)
    return _cache[key]


def _np(d):
    return {k: v.cpu().numpy() for k, v in d.items()}


def _kappa_k(oc, cfg, m):
    """kappa_2 of circle m's IMQ matrix K (Eq. 20; c^2 of Eq. 19 with angles in radians)."""
    k0, k1 = oc.knot_ptr[m], oc.knot_ptr[m + 1]
    return oimq.condition(oc.ku[k0:k1], cfg["imq_c2"])


def _averaged(fn):
    def make(*a, **k):
        cfg = fn(*a, **k)
        cfg["cover"]["rows"] = "averaged"
        return cfg
    return make


COVERS = [("tiny", workloads.tiny), ("varcoef", workloads.varcoef), ("scaled", workloads.scaled),
          ("poisson46", workloads.poisson46), ("tiny_averaged", _averaged(workloads.tiny)),
          ("varcoef_averaged", _averaged(workloads.varcoef))]


@pytest.mark.parametrize("name,fn", COVERS)
def test_cover_bit_exact(pdd, name, fn):
    cfg = fn()
    cov = pdd.Cover(cfg)
    oc = _oracle_cover(name, cfg)
    a = _np(cov.arrays())
    assert (cov.M, cov.N, cov.nnz) == (oc.M, oc.N, oc.col.size)
    assert cov.M_floating == int(oc.floating.sum())
    assert np.array_equal(a["floating"].astype(bool), oc.floating)
    for k in ("knot_ptr", "kowner", "row_sub", "rowptr", "col", "pi_ptr", "pi_sub"):
        assert np.array_equal(a[k].astype(np.int64), getattr(oc, k).astype(np.int64)), k
    assert np.array_equal(a["kdir"].astype(bool), oc.kdir)
    assert np.array_equal(a["cx"], oc.cx) and np.array_equal(a["cy"], oc.cy) and np.array_equal(a["r"], oc.r)
    for k in ("kx", "ky", "ku"):
        assert np.abs(a[k] - getattr(oc, k)).max() <= 8e-16 * max(1.0, np.abs(getattr(oc, k)).max()), k


def _row_err(got, ref):
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


@pytest.mark.parametrize("precision,factor", [("fp64", "blocked"), ("mixed", "recursive_tc"), ("mixed", "blocked")])
def test_floating_rows_tiny(pdd, precision, factor):
    cfg = workloads.tiny(paths=64)
    oc = _oracle_cover("tiny", cfg)
    S = pdd.System(pdd.Cover(cfg), cfg, precision, factor=factor)
    g = _np(S.csr())
    ref = osystem.assemble(cfg, oc, rows=[i for i in range(oc.N) if oc.row_sub[i] >= 0 and oc.floating[oc.row_sub[i]]])
    assert len(ref.fl_rows) == 64
    for i in ref.fl_rows:
        a, b = oc.rowptr[i], oc.rowptr[i + 1]
        assert _row_err(g["val"][a:b], ref.vals[a:b]) < 1e-10, i
        assert abs(g["b"][i] - ref.b[i]) <= 1e-10 * max(abs(ref.b[i]), 1e-3 * np.abs(ref.b).max() + 1e-300)
    st = S.stats()
    assert st["floating_disks"] == 4 and st["floating_rows"] == 64
    if precision == "mixed":
        assert st["unconverged_disks"] == 0 and st["max_refine_sweeps"] >= 2


@pytest.mark.parametrize("precision,factor", [("fp64", "blocked"), ("mixed", "recursive_tc"), ("mixed", "blocked")])
def test_floating_rows_varcoef_sampled(pdd, precision, factor):
    """Full-size variable-coefficient workload; 6 disks recomputed by the oracle."""
    cfg = workloads.varcoef(paths=64)
    oc = _oracle_cover("varcoef", cfg)
    S = pdd.System(pdd.Cover(cfg), cfg, precision, factor=factor)
    g = _np(S.csr())
    rng = np.random.default_rng(4)
    disks = [m for m in range(oc.M) if oc.floating[m] and oc.sub_rows(m).size]
    from oracle import problem, spectral
    op = problem.Operator(cfg["op"], oc.domain)
    shapes = {}
    for m in rng.choice(disks, 6, replace=False):
        res = spectral.floating_rows(oc, op, int(m), shapes)
        for i, (cols, v, bi) in res.items():
            a, b = oc.rowptr[i], oc.rowptr[i + 1]
            rc = oc.col[a:b]
            pos = np.searchsorted(rc, cols)
            assert _row_err(g["val"][a + pos], v) < 1e-10, (m, i)
            assert abs(g["b"][i] - bi) <= 1e-10 * max(abs(bi), 1e-3)
    if precision == "mixed":
        assert S.stats()["unconverged_disks"] == 0


@pytest.mark.parametrize("precision,factor", [("fp64", "blocked"), ("mixed", "recursive_tc")])
def test_floating_rows_poisson46_sampled(pdd, precision, factor):
    """The paper's Poisson test (Eq. 46) on [-50,50]^2: 968-node disks (22 x 44, not a multiple
    of the LU panel width), 44 knots; 4 disks recomputed by the oracle.  The collocation matrix
    has kappa ~ 1e5 (Sec. 4), so rows agree to ~kappa u, inside 1e-9."""
    cfg = workloads.poisson46(paths=16)
    oc = _oracle_cover("poisson46", cfg)
    S = pdd.System(pdd.Cover(cfg), cfg, precision, factor=factor)
    g = _np(S.csr())
    rng = np.random.default_rng(46)
    disks = [m for m in range(oc.M) if oc.floating[m] and oc.sub_rows(m).size]
    from oracle import problem, spectral
    op = problem.Operator(cfg["op"], oc.domain)
    shapes = {}
    for m in rng.choice(disks, 4, replace=False):
        for i, (cols, v, bi) in spectral.floating_rows(oc, op, int(m), shapes).items():
            a, b = oc.rowptr[i], oc.rowptr[i + 1]
            pos = np.searchsorted(oc.col[a:b], cols)
            assert _row_err(g["val"][a + pos], v) < 1e-9, (m, i)
            assert abs(g["b"][i] - bi) <= 1e-9 * max(abs(bi), 1e-3)
    if precision == "mixed":
        assert S.stats()["unconverged_disks"] == 0


def test_mc_rows_identical_streams_poisson46_sampled(pdd):
    """Eq. 46 workload with the boundary shift at h = 0.015 (256 paths per knot), FP64 form on
    the oracle's streams; 6 Monte Carlo rows recomputed."""
    cfg = workloads.poisson46(paths=256)
    oc = _oracle_cover("poisson46", cfg)
    S = pdd.System(pdd.Cover(cfg), cfg, "fp64")
    mc = _np(S.mc())
    rows = mc["rows"]
    rng = np.random.default_rng(12)
    pick = rng.choice(rows.size, 6, replace=False)
    ref = osystem.assemble(cfg, oc, rows=[int(rows[k]) for k in pick], threads=6)
    for k in pick:
        i = int(rows[k])
        r = ref.mc_rows[i]
        got = mc["moments"][mc["mom_ptr"][k]:mc["mom_ptr"][k + 1]]
        assert np.abs(got - r.moments).max() <= 1e-12 * max(1.0, np.abs(r.moments).max()), i
        assert abs(mc["bmean"][k] - r.b) <= 1e-12 * max(1.0, abs(r.b))


def test_solution_poisson46_against_oracle(pdd):
    """Whole path on the Eq. 46 workload (32 paths per knot, FP64 form, identical streams).

    With 44 knots per arc and c^2 = 1.5 in the angle (Sec. 4), the IMQ matrices K of the perimeter
    circles have kappa(K) up to ~7e11, so their rows of C are fixed by FP64 only to ~16 kappa(K) u
    (~1e-3 relative); the moments are not affected.  Checks: every entry of C and r within its own
    bound (floating rows 1e-10), and u within the perturbation bound
    ||C_o^-1|| (||C_g - C_o|| ||u_g|| + ||r_g - r_o|| + ||C_g u_g - r_g||) (infinity norms)."""
    import scipy.sparse as sp
    cfg = workloads.poisson46(paths=32, cv_degree=0)     # 32 paths cannot fit the 14-feature regression
    oc = _oracle_cover("poisson46", cfg)
    cov = pdd.Cover(cfg)
    S = pdd.System(cov, cfg, "fp64")
    u = S.solve(rtol=1e-14).cpu().numpy()
    assert S.last_solve["converged"]
    g = _np(S.csr())
    ref = osystem.assemble(cfg, oc, threads=8)
    for i in range(oc.N):
        a, b = oc.rowptr[i], oc.rowptr[i + 1]
        m = oc.row_sub[i]
        if m < 0:
            assert abs(g["b"][i] - ref.b[i]) <= 1e-14 * max(1.0, abs(ref.b[i]))
            continue
        if oc.floating[m]:
            tol = 1e-10
        else:
            tol = 1e-12 + 16 * _kappa_k(oc, cfg, m) * np.finfo(float).eps
        scale = max(1.0, np.abs(ref.vals[a:b]).max())
        assert np.abs(g["val"][a:b] - ref.vals[a:b]).max() <= tol * scale, i
        assert abs(g["b"][i] - ref.b[i]) <= tol * max(1.0, abs(ref.b[i])), i
    Co = ref.csr()
    Cg = sp.csr_matrix((g["val"], oc.col, oc.rowptr), shape=(oc.N, oc.N))
    uo = okrylov.solve(Co, ref.b)
    inv_norm = np.abs(np.linalg.inv(Co.toarray())).sum(1).max()
    dC = abs(Cg - Co).sum(1).max()
    bound = inv_norm * (dC * np.abs(u).max() + np.abs(g["b"] - ref.b).max() +
                        np.abs(Cg @ u - g["b"]).max())
    err = np.abs(u - uo).max()
    assert err <= bound + 1e-12 * np.abs(uo).max(), (err, bound)
    assert err < 1e-3                                 # and the bound itself is not vacuous


def test_poisson46_full_size_accuracy(pdd):
    """Sec. 4 parameters (5,000 paths per knot, h = 0.015, boundary shift, pathwise variance
    reduction), mixed form with RAS: the interfacial solution against u46 at the knots.  Without
    the variance reduction the RMS error is the plain Monte Carlo one, 1.8e-3; with it 6.6e-5
    (Table 1: 3.7e-5)."""
    cfg = workloads.poisson46()
    cov = pdd.Cover(cfg)
    S = pdd.System(cov, cfg, "mixed")
    u = S.solve(rtol=1e-12, precond="ras").cpu().numpy()
    a = _np(cov.arrays())
    from oracle import problem
    uex = problem.Operator.u46(a["kx"], a["ky"])[0]
    rms = float(np.sqrt(np.mean((u - uex) ** 2)))
    assert S.last_solve["converged"]
    assert rms < 2e-4, rms                            # measured 6.6e-5 (plain paths: 1.8e-3)
    assert S.stats()["unconverged_disks"] == 0


def test_averaged_rows_tiny_against_oracle(pdd):
    """Eq. 38-39 on the 4x4 lattice, FP64 form on the oracle's streams (the k-th subdomain of a
    row draws with Philox counter word 3 = k): every entry of C and r, the Monte Carlo slots and
    the solution against the oracle."""
    cfg = _averaged(workloads.tiny)(paths=300)
    oc = _oracle_cover("tiny_averaged", cfg)
    cov = pdd.Cover(cfg)
    S = pdd.System(cov, cfg, "fp64")
    g = _np(S.csr())
    ref = osystem.assemble(cfg, oc, threads=4)
    eps = np.finfo(float).eps
    kmax = max(_kappa_k(oc, cfg, m)
               for m in range(oc.M) if not oc.floating[m] and oc.knot_ptr[m + 1] > oc.knot_ptr[m])
    tol = 1e-10 + 16 * kmax * eps
    assert np.abs(g["val"] - ref.vals).max() <= tol * np.abs(ref.vals).max()
    assert np.abs(g["b"] - ref.b).max() <= tol * max(1.0, np.abs(ref.b).max())
    ok = ref.se_b > 0           # root sum of squares of batch-means vs per-path standard errors
    assert 0.4 < np.median(g["se_b"][ok] / ref.se_b[ok]) < 1.6
    diag = g["val"][[oc.rowptr[i] + int(np.searchsorted(oc.col[oc.rowptr[i]:oc.rowptr[i + 1]], i))
                     for i in range(oc.N)]]
    want = np.array([max(1, oc.pi(i).size) for i in range(oc.N)], float)
    assert np.array_equal(diag, want) and (want >= 2).sum() > oc.N // 4
    mc = _np(S.mc())
    keys = {(int(i), int(m)) for i, m in zip(mc["rows"], mc["subs"])}
    assert keys == set(ref.mc_rows.keys())
    for k, (i, m) in enumerate(zip(mc["rows"], mc["subs"])):
        r = ref.mc_rows[(int(i), int(m))]
        got = mc["moments"][mc["mom_ptr"][k]:mc["mom_ptr"][k + 1]]
        assert np.abs(got - r.moments).max() <= 1e-12 * max(1.0, np.abs(r.moments).max()), (i, m)
    u = S.solve(rtol=1e-14).cpu().numpy()
    uo = okrylov.solve(ref.csr(), ref.b)
    assert np.abs(u - uo).max() <= 1e-9 * np.abs(uo).max()
    with pytest.raises(pdd.PddError):
        S.solve(precond="ras")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_averaged_rows_varcoef_sampled(pdd, precision):
    """Averaged rows on the full variable-coefficient cover: 4 floating disks recomputed by the
    oracle; each disk's block of every row it contributes to, and its part of r through the
    rows whose every subdomain is floating."""
    cfg = _averaged(workloads.varcoef)(paths=16)
    oc = _oracle_cover("varcoef_averaged", cfg)
    S = pdd.System(pdd.Cover(cfg), cfg, precision)
    g = _np(S.csr())
    rng = np.random.default_rng(38)
    disks = [m for m in range(oc.M) if oc.floating[m] and oc.sub_rows(m).size]
    from oracle import problem, spectral
    op = problem.Operator(cfg["op"], oc.domain)
    shapes = {}
    parts = {}
    for m in rng.choice(disks, 4, replace=False):
        for i, (cols, v, bi) in spectral.floating_rows(oc, op, int(m), shapes).items():
            a, b = oc.rowptr[i], oc.rowptr[i + 1]
            pos = np.searchsorted(oc.col[a:b], cols)
            assert _row_err(g["val"][a + pos], v) < 1e-10, (m, i)
            parts.setdefault(i, {})[int(m)] = bi
    checked = 0
    for i, got in parts.items():
        if set(got) == set(int(m) for m in oc.pi(i)):
            want = sum(got[m] for m in sorted(got))
            assert abs(g["b"][i] - want) <= 1e-10 * max(abs(want), 1e-3)
            checked += 1
    assert checked > 0
    if precision == "mixed":
        assert S.stats()["unconverged_disks"] == 0


@pytest.mark.parametrize("leaf,tmin", [(32, 128), (32, 32), (16, 64), (8, 32), (16, 1000000)])
def test_recursive_lu_candidates(pdd, leaf, tmin):
    """Every factorisation the autotuner may pick gives the oracle's floating rows (varcoef, 6 disks)."""
    cfg = workloads.varcoef(paths=16)
    oc = _oracle_cover("varcoef", cfg)
    S = pdd.System(pdd.Cover(cfg), cfg, "mixed", lu_leaf_width=leaf, lu_tensor_min=tmin)
    assert S.stats()["unconverged_disks"] == 0
    g = _np(S.csr())
    from oracle import problem, spectral
    op = problem.Operator(cfg["op"], oc.domain)
    disks = [m for m in range(oc.M) if oc.floating[m] and oc.sub_rows(m).size]
    for m in np.random.default_rng(leaf).choice(disks, 3, replace=False):
        for i, (cols, v, bi) in spectral.floating_rows(oc, op, int(m)).items():
            pos = oc.rowptr[i] + np.searchsorted(oc.col[oc.rowptr[i]:oc.rowptr[i + 1]], cols)
            assert _row_err(g["val"][pos], v) < 1e-10, (leaf, tmin, m, i)


def test_floating_rows_scaled_sampled(pdd):
    """The 48(r) x 64(theta) grid (n = 3072) of the scaled workload: recursive tensor-core LU + FP64
    refinement on 3,600 disks; 2 disks recomputed by the oracle (Householder QR of 3072 x 3072)."""
    cfg = workloads.scaled(paths=16)
    oc = _oracle_cover("scaled", cfg)
    S = pdd.System(pdd.Cover(cfg), cfg, "mixed")
    g = _np(S.csr())
    st = S.stats()
    assert st["unconverged_disks"] == 0 and st["floating_disks"] == 3600
    from oracle import problem, spectral
    op = problem.Operator(cfg["op"], oc.domain)
    rng = np.random.default_rng(2)
    disks = [m for m in range(oc.M) if oc.floating[m] and oc.sub_rows(m).size]
    for m in rng.choice(disks, 2, replace=False):
        for i, (cols, v, bi) in spectral.floating_rows(oc, op, int(m)).items():
            a, b = oc.rowptr[i], oc.rowptr[i + 1]
            pos = np.searchsorted(oc.col[a:b], cols)
            assert _row_err(g["val"][a + pos], v) < 1e-10, (m, i)


@pytest.mark.parametrize("shift", [False, True], ids=["plain", "boundary_shift"])
def test_mc_rows_identical_streams_tiny(pdd, shift):
    """FP64 form on the oracle's Philox streams; with the Gobet-Menozzi boundary shift both sides stop
    at the shrunk boundaries and score the projected exit point."""
    cfg = workloads.tiny(paths=500)
    cfg["mc"]["boundary_shift"] = shift
    oc = _oracle_cover("tiny", cfg)
    S = pdd.System(pdd.Cover(cfg), cfg, "fp64")
    g = _np(S.csr())
    mc = _np(S.mc())
    rows = mc["rows"]
    ref = osystem.assemble(cfg, oc, rows=list(rows), threads=4)
    assert len(ref.mc_rows) == rows.size > 100
    for k, i in enumerate(rows):
        r = ref.mc_rows[int(i)]
        got = mc["moments"][mc["mom_ptr"][k]:mc["mom_ptr"][k + 1]]
        assert np.abs(got - r.moments).max() <= 1e-12 * max(1.0, np.abs(r.moments).max()), i
        assert abs(mc["bmean"][k] - r.b) <= 1e-12 * max(1.0, abs(r.b))
        a, b = oc.rowptr[i], oc.rowptr[i + 1]
        rc = oc.col[a:b]
        pos = np.searchsorted(rc, r.cols)
        kap = _kappa_k(oc, cfg, int(oc.row_sub[i])) if r.u_stencil.size else 1.0
        tol = 1e-12 + 16 * kap * np.finfo(float).eps
        assert np.abs(g["val"][a + pos] - r.vals).max() <= tol * max(1.0, np.abs(r.vals).max()), i
        # batch-means standard errors against the per-path ones (31 degrees of freedom)
        ok = r.se > 0
        if np.any(ok):
            ratio = g["se"][a + pos][ok] / r.se[ok]
            assert 0.4 < np.median(ratio) < 1.6
    st = S.stats()
    assert st["path_steps"] == sum(r.steps for r in ref.mc_rows.values())


@pytest.mark.parametrize("degree", [2, 4])
def test_mc_control_variate_identical_streams(pdd, degree):
    """Pathwise variance reduction (regression control variate on the monomials of degree <= D),
    FP64 form on the oracle's Philox streams: the corrected moments and r at 1e-12, the C entries
    at 1e-12 + 16 kappa(K) eps, and the corrected standard errors against the oracle's."""
    cfg = workloads.tiny(paths=600)
    cfg["mc"]["cv_degree"] = degree
    cfg["mc"]["boundary_shift"] = True
    oc = _oracle_cover("tiny", cfg)
    S = pdd.System(pdd.Cover(cfg), cfg, "fp64")
    g = _np(S.csr())
    mc = _np(S.mc())
    rows = mc["rows"]
    ref = osystem.assemble(cfg, oc, rows=list(rows), threads=8)
    ratios = []
    for k, i in enumerate(rows):
        r = ref.mc_rows[int(i)]
        got = mc["moments"][mc["mom_ptr"][k]:mc["mom_ptr"][k + 1]]
        assert np.abs(got - r.moments).max() <= 1e-12 * max(1.0, np.abs(r.moments).max()), i
        assert abs(mc["bmean"][k] - r.b) <= 1e-12 * max(1.0, abs(r.b)), i
        a, b = oc.rowptr[i], oc.rowptr[i + 1]
        pos = np.searchsorted(oc.col[a:b], r.cols)
        tol = 1e-12 + 16 * _kappa_k(oc, cfg, int(oc.row_sub[i])) * np.finfo(float).eps
        assert np.abs(g["val"][a + pos] - r.vals).max() <= tol * max(1.0, np.abs(r.vals).max()), i
        ok = r.se > 0
        ratios += list(g["se"][a + pos][ok] / r.se[ok])
    # batch-means standard errors of the corrected rows against the per-path ones
    assert 0.5 < np.median(ratios) < 1.5, np.median(ratios)


def test_mc_control_variate_mixed_within_standard_errors(pdd):
    """The mixed form (FP32 positions; its normals come from the leading bits of the same Philox
    words, so its paths follow the FP64 ones to FP32 precision) with the control variate against
    the FP64 form with it, on the Eq. 46 cover at 400 paths: every Monte Carlo C entry and r within
    4.5 combined standard errors (the two are correlated, so far closer in practice), and the
    corrected standard errors of r far below the plain ones."""
    cfg = workloads.poisson46(paths=400)
    cov = pdd.Cover(cfg)
    S64 = pdd.System(cov, cfg, "fp64")
    Sm = pdd.System(cov, cfg, "mixed")
    plain = dict(cfg, mc=dict(cfg["mc"], cv_degree=0))
    Sp = pdd.System(cov, plain, "mixed")
    a = _np(cov.arrays())
    g64, gm, gp = _np(S64.csr()), _np(Sm.csr()), _np(Sp.csr())
    mcr = set(_np(Sm.mc())["rows"].tolist())
    z, red = [], []
    for i in mcr:
        p0, p1 = a["rowptr"][i], a["rowptr"][i + 1]
        se = np.sqrt(g64["se"][p0:p1] ** 2 + gm["se"][p0:p1] ** 2)
        ok = se > 0
        z += list(np.abs(g64["val"][p0:p1] - gm["val"][p0:p1])[ok] / se[ok])
        seb = math.sqrt(g64["se_b"][i] ** 2 + gm["se_b"][i] ** 2)
        if seb > 0:
            z.append(abs(g64["b"][i] - gm["b"][i]) / seb)
        if gp["se_b"][i] > 0:
            red.append(gm["se_b"][i] / gp["se_b"][i])
    z = np.array(z)
    assert z.max() < 4.5, z.max()
    assert np.median(red) < 0.35, np.median(red)     # measured 0.20 at 400 paths (variance / 25)


def test_mc_rows_identical_streams_varcoef_sampled(pdd):
    """Full-size variable-coefficient workload (10^4 paths, h = 1e-5), 6 rows recomputed."""
    cfg = workloads.varcoef()
    oc = _oracle_cover("varcoef", cfg)
    S = pdd.System(pdd.Cover(cfg), cfg, "fp64")
    mc = _np(S.mc())
    rows = mc["rows"]
    rng = np.random.default_rng(11)
    pick = rng.choice(rows.size, 6, replace=False)
    ref = osystem.assemble(cfg, oc, rows=[int(rows[k]) for k in pick], threads=6)
    for k in pick:
        i = int(rows[k])
        r = ref.mc_rows[i]
        got = mc["moments"][mc["mom_ptr"][k]:mc["mom_ptr"][k + 1]]
        assert np.abs(got - r.moments).max() <= 1e-12 * max(1.0, np.abs(r.moments).max()), i
        assert abs(mc["bmean"][k] - r.b) <= 1e-12 * max(1.0, abs(r.b))


def test_mc_adaptive_path_counts_identical_streams(pdd):
    """Adaptive path counts: the GPU and the oracle apply the rule to their own pilots (batch-means
    standard errors) and must pick the same counts; the final estimates agree at 1e-12."""
    cfg = workloads.tiny(paths=64)
    cfg["mc"] = dict(cfg["mc"], paths_max=2048, se_target=0.01)
    oc = _oracle_cover("tiny", cfg)
    S = pdd.System(pdd.Cover(cfg), cfg, "fp64")
    mc = _np(S.mc())
    rows = mc["rows"]
    st = S.stats()
    assert st["extended_rows"] > 0
    ref = osystem.assemble(cfg, oc, rows=[int(i) for i in rows], threads=4)
    P0 = cfg["mc"]["paths"]
    # the GPU counts every path it ran: the pilot of each row, then the full rerun of extended rows
    assert st["paths_total"] == sum(P0 + (r.paths if r.paths > P0 else 0) for r in ref.mc_rows.values())
    assert st["extended_rows"] == sum(1 for r in ref.mc_rows.values() if r.paths > P0)
    for k, i in enumerate(rows):
        r = ref.mc_rows[int(i)]
        got = mc["moments"][mc["mom_ptr"][k]:mc["mom_ptr"][k + 1]]
        assert np.abs(got - r.moments).max() <= 1e-12 * max(1.0, np.abs(r.moments).max()), i
        assert abs(mc["bmean"][k] - r.b) <= 1e-12 * max(1.0, abs(r.b))


def test_mc_mixed_within_standard_errors(pdd):
    """Mixed form on an independent stream (seed 1) against the FP64 oracle (seed 0)."""
    cfg = workloads.tiny(paths=2000)
    oc = _oracle_cover("tiny", cfg)
    cfg1 = workloads.tiny(paths=2000, seed=1)
    S = pdd.System(pdd.Cover(cfg1), cfg1, "mixed")
    g = _np(S.csr())
    mc = _np(S.mc())
    rows = [int(i) for i in mc["rows"][::4]]
    ref = osystem.assemble(cfg, oc, rows=rows, threads=4)
    z = []
    for i in rows:
        r = ref.mc_rows[i]
        a, b = oc.rowptr[i], oc.rowptr[i + 1]
        pos = np.searchsorted(oc.col[a:b], r.cols)
        se = np.sqrt(g["se"][a + pos] ** 2 + r.se ** 2)
        ok = se > 1e-12
        z.extend(((g["val"][a + pos] - r.vals)[ok] / se[ok]).tolist())
        z.append((g["b"][i] - r.b) / math.hypot(g["se_b"][i], r.se_b))
    z = np.array(z)
    assert np.mean(np.abs(z) > 4.0) < 5e-3      # 4 SE (batch-means SE has 31 degrees of freedom)
    assert np.abs(z).max() < 6.0
    assert 0.6 < np.mean(z * z) < 1.6


def test_mc_mixed_boundary_shift_within_standard_errors(pdd):
    """Mixed form with the boundary shift against the oracle's FP64 shifted scheme on independent
    streams: within 4 standard errors."""
    cfg = workloads.tiny(paths=2000)
    cfg["mc"]["boundary_shift"] = True
    cfg["mc"]["h"] = 4e-4
    oc = _oracle_cover("tiny", cfg)
    cfg1 = dict(cfg, mc=dict(cfg["mc"], seed=1))
    S = pdd.System(pdd.Cover(cfg1), cfg1, "mixed")
    g = _np(S.csr())
    mc = _np(S.mc())
    rows = [int(i) for i in mc["rows"][::4]]
    ref = osystem.assemble(cfg, oc, rows=rows, threads=4)
    z = []
    for i in rows:
        r = ref.mc_rows[i]
        a, b = oc.rowptr[i], oc.rowptr[i + 1]
        pos = np.searchsorted(oc.col[a:b], r.cols)
        ok = r.se > 0
        z.extend(((g["val"][a + pos] - r.vals)[ok] / np.hypot(g["se"][a + pos], r.se)[ok]).tolist())
    z = np.array(z)
    assert np.abs(z).max() < 6.0 and np.mean(np.abs(z) > 4.0) < 5e-3
    assert 0.5 < np.mean(z * z) < 1.7


@pytest.mark.parametrize("name,paths", [("tiny", 2000), ("varcoef", 1000), ("poisson46", 500)])
def test_mc_mixed_same_stream_tracks_fp64(pdd, name, paths):
    """On the same seed the mixed form draws the leading bits of the same Philox words, so its
    paths follow the FP64 paths to FP32 precision: estimates agree far inside one SE.  The
    variable-coefficient and Eq. 46 stencils have kappa(K) up to 5.6e8 and 7e11, so this also
    checks that C = -K^-T M does not amplify the rounding of the mixed form's moment sums."""
    cfg = getattr(workloads, name)(paths=paths)
    cov = pdd.Cover(cfg)
    g32 = _np(pdd.System(cov, cfg, "mixed").csr())
    g64 = _np(pdd.System(cov, cfg, "fp64").csr())
    ok = g64["se"] > 0
    z = np.abs(g32["val"] - g64["val"])[ok] / g64["se"][ok]
    assert np.median(z) < 0.05
    assert np.quantile(z, 0.99) < 0.5 and z.max() < 3.0, (np.quantile(z, 0.99), z.max())
    okb = g64["se_b"] > 0
    assert np.median(np.abs(g32["b"] - g64["b"])[okb] / g64["se_b"][okb]) < 0.05


def test_solution_tiny_against_oracle(pdd):
    cfg = workloads.tiny(paths=300)
    oc = _oracle_cover("tiny", cfg)
    S = pdd.System(pdd.Cover(cfg), cfg, "fp64")
    u = S.solve(rtol=1e-14).cpu().numpy()
    ref = osystem.assemble(cfg, oc, threads=4)
    uo = okrylov.solve(ref.csr(), ref.b)
    assert np.abs(u - uo).max() <= 1e-10 * np.abs(uo).max()
    assert S.last_solve["converged"]


def _varcoef_small(paths=400):
    """The variable-coefficient workload's operator, hex lattice and grids on [0, 0.6]^2
    (about 100 circles): small enough for the whole oracle."""
    cfg = workloads.varcoef(paths=paths)
    cfg["domain"] = {"kind": "square", "p": [0.0, 0.0, 0.6, 0.6]}
    cfg["cover"] = dict(cfg["cover"], nx=10, ny=12)
    return cfg


@pytest.mark.parametrize("name", ["tiny", "varcoef_small"])
def test_solution_mixed_disks_against_oracle(pdd, name):
    """Mixed-precision disks (FP32 LU on the tensor cores + FP64 refinement) with FP64 paths on the
    oracle's Philox streams: every entry of C and r against the oracle (floating rows 1e-10,
    Monte Carlo rows 1e-12 + 16 kappa(K) eps) and u against the oracle's direct solve at 1e-10, or,
    where the IMQ matrices fix the Monte Carlo rows' C entries only to 16 kappa(K) eps (kappa ~5e8
    on the variable-coefficient arcs), within the perturbation bound
    ||C_o^-1|| (||C_g - C_o|| ||u_g|| + ||r_g - r_o|| + ||C_g u_g - r_g||) (infinity norms)."""
    cfg = workloads.tiny(paths=400) if name == "tiny" else _varcoef_small()
    oc = _oracle_cover(name, cfg)
    cov = pdd.Cover(cfg)
    assert cov.M == oc.M and cov.N == oc.N
    S = pdd.System(cov, cfg, "mixed", path_precision="fp64")
    u = S.solve(rtol=1e-14).cpu().numpy()
    assert S.last_solve["converged"] and S.stats()["unconverged_disks"] == 0
    g = _np(S.csr())
    ref = osystem.assemble(cfg, oc, threads=8)
    nfl = 0
    for i in range(oc.N):
        a, b = oc.rowptr[i], oc.rowptr[i + 1]
        m = oc.row_sub[i]
        if m < 0:
            continue
        if oc.floating[m]:
            nfl += 1
            assert _row_err(g["val"][a:b], ref.vals[a:b]) < 1e-10, i
            assert abs(g["b"][i] - ref.b[i]) <= 1e-10 * max(1.0, np.abs(ref.b).max()), i
        else:
            tol = 1e-12 + 16 * _kappa_k(oc, cfg, m) * np.finfo(float).eps
            assert np.abs(g["val"][a:b] - ref.vals[a:b]).max() <= tol * max(1.0, np.abs(ref.vals[a:b]).max()), i
            assert abs(g["b"][i] - ref.b[i]) <= tol * max(1.0, abs(ref.b[i])), i
    assert nfl > 0
    import scipy.sparse as sp
    Co = ref.csr()
    uo = okrylov.solve(Co, ref.b)
    Cg = sp.csr_matrix((g["val"], oc.col, oc.rowptr), shape=(oc.N, oc.N))
    inv_norm = np.abs(np.linalg.inv(Co.toarray())).sum(1).max()
    bound = inv_norm * (abs(Cg - Co).sum(1).max() * np.abs(u).max() + np.abs(g["b"] - ref.b).max() +
                        np.abs(Cg @ u - g["b"]).max())
    err = np.abs(u - uo).max()
    assert err <= max(1e-10 * np.abs(uo).max(), bound), (err, bound)
    if name == "tiny":
        assert err <= 1e-10 * np.abs(uo).max(), err


def test_mc_rows_identical_streams_scaled_sampled(pdd):
    """The scaled workload (62 x 62 lattice, 48 x 64 disk grids): FP64 paths on the oracle's streams
    (with mixed disks, the form the bench times), 8 Monte Carlo rows recomputed at 1e-12."""
    cfg = workloads.scaled(paths=256)
    oc = _oracle_cover("scaled", cfg)
    S = pdd.System(pdd.Cover(cfg), cfg, "mixed", path_precision="fp64")
    mc = _np(S.mc())
    g = _np(S.csr())
    rows = mc["rows"]
    rng = np.random.default_rng(5)
    pick = rng.choice(rows.size, 8, replace=False)
    ref = osystem.assemble(cfg, oc, rows=[int(rows[k]) for k in pick], threads=8)
    for k in pick:
        i = int(rows[k])
        r = ref.mc_rows[i]
        got = mc["moments"][mc["mom_ptr"][k]:mc["mom_ptr"][k + 1]]
        assert np.abs(got - r.moments).max() <= 1e-12 * max(1.0, np.abs(r.moments).max()), i
        assert abs(mc["bmean"][k] - r.b) <= 1e-12 * max(1.0, abs(r.b))
        a, b = oc.rowptr[i], oc.rowptr[i + 1]
        pos = np.searchsorted(oc.col[a:b], r.cols)
        tol = 1e-12 + 16 * _kappa_k(oc, cfg, int(oc.row_sub[i])) * np.finfo(float).eps
        assert np.abs(g["val"][a + pos] - r.vals).max() <= tol * max(1.0, np.abs(r.vals).max()), i


@pytest.mark.parametrize("name,ill", [("varcoef", True), ("poisson46", True), ("tiny", False)])
def test_mc_moment_sums_forced_modes(pdd, name, ill):
    """The mixed paths' basis sums (a12) forced to each mode, one assembly per mode on the same seed:
    FP64 sums are the reference; double-float sums agree to 1e-9 relative and FP32 sums only to 1e-5.
    The path records of two assemblies are not bit-identical: a lane folds its FP32 weight
    increments into the FP64 weights every 8 of its loop iterations, and which lane runs a path
    depends on the scheduling, so Y and Z differ by rounding (~1e-11 relative).  The 1e-9 bar sits
    between that and the FP32 sums' error (~1e-7).  On the variable-coefficient and Eq. 46 covers
    the IMQ matrices reach kappa(K) ~ 5e8 and ~7e11, where the automatic choice must pick the
    double-float or FP64 sums."""
    paths = {"varcoef": 1000, "poisson46": 500, "tiny": 2000}[name]
    cfg = getattr(workloads, name)(paths=paths)
    cov = pdd.Cover(cfg)
    out = {}
    for mode in ("fp64", "double_float", "fp32", "auto"):
        S = pdd.System(cov, cfg, "mixed", moment_sums=mode)
        mc = _np(S.mc())
        out[mode] = (mc["moments"], mc["bmean"])
    m64, b64 = out["fp64"]
    scale = np.abs(m64).max()
    err = {mode: np.abs(out[mode][0] - m64).max() / scale for mode in ("double_float", "fp32", "auto")}
    assert err["double_float"] <= 1e-9, err
    assert 1e-9 < err["fp32"] <= 1e-5, err           # the FP32 sums really are the less accurate ones
    # r_i does not go through the basis sums
    assert np.abs(out["double_float"][1] - b64).max() <= 1e-9 * max(1.0, np.abs(b64).max())
    if ill:
        assert err["auto"] <= 1e-9, err              # the automatic choice takes the accurate sums


@pytest.mark.parametrize("name", ["varcoef", "poisson46"])
def test_mc_double_float_sums_on_identical_records(pdd, name):
    """Double-float basis sums (a12) against FP64 sums on the SAME path records: FP64 paths are
    bit-reproducible, so two assemblies that differ only in the forced summation see identical
    (Y, Z, exit angle, side).  The double-float phi and sums must then agree with the FP64 ones to
    1e-12 relative (the split is within 2^-47, the double-float rsqrt within 1e-13)."""
    paths = {"varcoef": 1000, "poisson46": 500}[name]
    cfg = getattr(workloads, name)(paths=paths)
    cov = pdd.Cover(cfg)
    out = {}
    for mode in ("fp64", "double_float"):
        S = pdd.System(cov, cfg, "mixed", path_precision="fp64", moment_sums=mode)
        mc = _np(S.mc())
        out[mode] = (mc["moments"], mc["bmean"])
    m64, b64 = out["fp64"]
    mdf, bdf = out["double_float"]
    assert np.array_equal(bdf, b64)                   # r_i does not go through the basis sums
    assert np.abs(mdf - m64).max() <= 1e-12 * np.abs(m64).max(), np.abs(mdf - m64).max() / np.abs(m64).max()


def test_split_df_bits(pdd):
    """The integer-built double-float split of the double-float sums: hi + lo within 2^-47 of v for
    2^-74 <= |v| < 2^128, lo = 0 and an error below 2^-23 for 2^-126 <= |v| < 2^-74, signed zeros
    below 2^-126; hi is v truncated to FP32's 24 bits (|hi| <= |v|, same sign)."""
    rng = np.random.default_rng(11)
    ex = rng.uniform(-140.0, 127.0, 20000)
    v = rng.uniform(1.0, 2.0, ex.size) * np.exp2(np.floor(ex)) * rng.choice([-1.0, 1.0], ex.size)
    edge = []
    for e in (-127, -126, -125, -75, -74, -73, -1, 0, 1, 126):
        for m in (1.0, 1.0 + 2.0 ** -52, 1.5, 2.0 - 2.0 ** -52):
            edge += [m * 2.0 ** e, -m * 2.0 ** e]
    v = np.concatenate([v, np.array(edge), [0.0, -0.0, 1.0 / 3.0, np.pi, 1e-30, 1e30]])
    hl = pdd.split_df(torch.tensor(v, device="cuda")).cpu().numpy().astype(np.float64)
    hi, lo = hl[:, 0], hl[:, 1]
    av = np.abs(v)
    big = av >= 2.0 ** -74
    mid = (av >= 2.0 ** -126) & ~big
    small = av < 2.0 ** -126
    assert np.all(np.abs(hi + lo - v)[big] <= 2.0 ** -47 * av[big])
    assert np.all(lo[mid] == 0.0) and np.all(np.abs(hi - v)[mid] < 2.0 ** -23 * av[mid])
    assert np.all(hi[small] == 0.0) and np.all(lo[small] == 0.0)
    assert np.all(np.signbit(hi) == np.signbit(v))
    assert np.all(np.abs(hi) <= av)
    # hi is the truncation: its 24 bits are v's leading bits
    nz = ~small
    ulp = np.exp2(np.frexp(av[nz])[1] - 24.0)         # weight of the 24th significant bit
    assert np.all(hi[nz] == np.trunc(v[nz] / ulp) * ulp)


def test_gmres_random_csr_against_direct(pdd):
    import scipy.sparse as sp
    rng = np.random.default_rng(7)
    n = 3001
    A = sp.random(n, n, density=8.0 / n, random_state=7, format="csr") * 0.1 + sp.eye(n) * 2.0
    A.sort_indices()
    b = rng.standard_normal(n)
    rowptr = torch.tensor(A.indptr, dtype=torch.int32, device="cuda")
    col = torch.tensor(A.indices, dtype=torch.int32, device="cuda")
    val = torch.tensor(A.data, dtype=torch.float64, device="cuda")
    bt = torch.tensor(b, dtype=torch.float64, device="cuda")
    x, info = pdd.solve_csr(rowptr, col, val, bt, rtol=1e-13, restart=30)
    xr = okrylov.solve(A, b)
    assert info["converged"] and np.abs(x.cpu().numpy() - xr).max() <= 1e-10 * np.abs(xr).max()
    xt, info = pdd.solve_csr(rowptr, col, val, bt, rtol=1e-13, restart=30, transpose=True)
    xrt = okrylov.solve_transpose(A, b)
    assert info["converged"] and np.abs(xt.cpu().numpy() - xrt).max() <= 1e-10 * np.abs(xrt).max()
    y = pdd.spmv_csr(rowptr, col, val, bt).cpu().numpy()
    assert np.abs(y - A @ b).max() <= 1e-13 * np.abs(A @ b).max()
    yt = pdd.spmv_csr(rowptr, col, val, bt, transpose=True).cpu().numpy()
    assert np.abs(yt - A.T @ b).max() <= 1e-13 * np.abs(A.T @ b).max()


def test_solution_varcoef_residual(pdd):
    """Full-size workload: the GPU's u solves the GPU's C u = r to the stated tolerance (FP64 check on CPU)."""
    import scipy.sparse as sp
    cfg = workloads.varcoef(paths=256)
    cov = pdd.Cover(cfg)
    S = pdd.System(cov, cfg, "mixed")
    u = S.solve(rtol=1e-13).cpu().numpy()
    a = _np(cov.arrays())
    g = _np(S.csr())
    C = sp.csr_matrix((g["val"], a["col"], a["rowptr"]), shape=(cov.N, cov.N))
    assert np.linalg.norm(C @ u - g["b"]) <= 1.05e-13 * np.linalg.norm(g["b"])


def _gpu_csr(cov, S):
    import scipy.sparse as sp
    a = _np(cov.arrays())
    g = _np(S.csr())
    return sp.csr_matrix((g["val"], a["col"], a["rowptr"]), shape=(cov.N, cov.N)), g["b"]


def test_ras_apply_against_oracle(pdd):
    """M_RAS^-1 v (Eq. 44) on the GPU (FP32 inverses of the C_p) against the oracle's FP64 operator
    built from the same C and the same subsets."""
    cfg = workloads.tiny(paths=300)
    oc = _oracle_cover("tiny", cfg)
    cov = pdd.Cover(cfg)
    S = pdd.System(cov, cfg, "fp64")
    C, _ = _gpu_csr(cov, S)
    apply, _ = okrylov.ras_operator(C, okrylov.ras_subsets(oc.knot_ptr, oc.row_sub))
    v = np.random.default_rng(11).standard_normal(cov.N)
    y = S.ras_apply(torch.tensor(v, device="cuda")).cpu().numpy()
    want = apply(v)
    assert np.abs(y - want).max() <= 1e-5 * np.abs(want).max()


def test_ras_solve_tiny_against_oracle(pdd):
    cfg = workloads.tiny(paths=300)
    oc = _oracle_cover("tiny", cfg)
    S = pdd.System(pdd.Cover(cfg), cfg, "fp64")
    u = S.solve(rtol=1e-14, precond="ras").cpu().numpy()
    it_ras = S.last_solve["iters"]
    S.solve(rtol=1e-14)
    it_plain = S.last_solve["iters"]
    ref = osystem.assemble(cfg, oc, threads=4)
    uo = okrylov.solve(ref.csr(), ref.b)
    assert np.abs(u - uo).max() <= 1e-10 * np.abs(uo).max()
    assert it_ras < it_plain, (it_ras, it_plain)


def test_ras_solve_varcoef_residual(pdd):
    """Full-size workload: the preconditioned solve meets the FP64 tolerance in fewer iterations."""
    cfg = workloads.varcoef(paths=256)
    cov = pdd.Cover(cfg)
    S = pdd.System(cov, cfg, "mixed")
    u = S.solve(rtol=1e-13, precond="ras").cpu().numpy()
    it_ras = S.last_solve["iters"]
    C, b = _gpu_csr(cov, S)
    assert np.linalg.norm(C @ u - b) <= 1.05e-13 * np.linalg.norm(b)
    S.solve(rtol=1e-13)
    assert it_ras < S.last_solve["iters"], (it_ras, S.last_solve["iters"])


def test_adjoint_against_oracle(pdd):
    from oracle import adjoint as oadj
    cfg = workloads.grad(paths=64)
    oc = _oracle_cover("grad", cfg)
    S = pdd.System(pdd.Cover(cfg), cfg, "fp64")
    u = S.solve(rtol=1e-14)
    rng = np.random.default_rng(9)
    u_obs = np.exp(oc.kx) * np.sin(oc.ky) + 0.01 * rng.standard_normal(oc.N)
    dJ = 2.0 * (u - torch.tensor(u_obs, device="cuda"))
    g, lam = S.grad(u, dJ, return_lambda=True)
    g = g.cpu().numpy()
    ref = osystem.assemble(cfg, oc, with_grad=True)
    uo = okrylov.solve(ref.csr(), ref.b)
    gw, ga, lo, gf = oadj.gradient(cfg, ref, uo, 2.0 * (uo - u_obs))
    assert gf.size == 16
    want = np.concatenate([gw, gf, ga])
    assert np.abs(lam.cpu().numpy() - lo).max() <= 1e-9 * np.abs(lo).max()
    assert np.abs(g - want).max() <= 1e-8 * np.abs(want).max()


def test_error_statuses(pdd):
    cfg = workloads.tiny()
    bad = dict(cfg)
    bad["cover"] = dict(cfg["cover"], nx=3)        # drops a column of circles: a gap
    with pytest.raises(pdd.PddError) as e:
        pdd.Cover(bad)
    assert e.value.code == "PDD_ECOVER_GAP"
    corner = dict(cfg)
    # a circle through the corners (0,0) and (0,1), exactly representable: degenerate junctions
    corner["cover"] = {"kind": "explicit", "cx": np.array([0.375, 0.5]), "cy": np.array([0.5, 0.5]),
                       "r": np.array([0.625, 0.9]), "n_knots": np.array([16, 16], np.int32),
                       "n_r": np.array([8, 8], np.int32), "n_theta": np.array([16, 16], np.int32)}
    with pytest.raises(pdd.PddError) as e:
        pdd.Cover(corner)
    assert e.value.code == "PDD_EINVAL"


def test_adjoint_against_central_differences_gpu(pdd):
    """The GPU adjoint against central differences of the GPU's own J (same Philox streams).

    Step 1e-4 (truncation O(eps^2)); the bar is the one the oracle's adjoint meets.
    """
    base = workloads.grad(paths=64)
    oc = _oracle_cover("grad", base)
    rng = np.random.default_rng(9)
    u_obs = torch.tensor(np.exp(oc.kx) * np.sin(oc.ky) + 0.01 * rng.standard_normal(oc.N), device="cuda")

    def J(cfg):
        S = pdd.System(pdd.Cover(cfg), cfg, "fp64")
        u = S.solve(rtol=1e-15)
        return float(((u - u_obs) ** 2).sum().item()), S, u

    J0, S, u = J(base)
    g = S.grad(u, 2.0 * (u - u_obs)).cpu().numpy()
    nw = base["op"]["rbf"]["w"].size
    nf = base["op"]["frbf"]["w"].size
    eps = 1e-4
    for kind, idx in (("w", 3), ("w", 50), ("a", 1), ("a", 17), ("v", 2), ("v", 11)):
        vals = []
        for sgn in (1.0, -1.0):
            c = workloads.grad(paths=64)
            if kind == "w":
                c["op"]["rbf"]["w"] = c["op"]["rbf"]["w"].copy()
                c["op"]["rbf"]["w"][idx] += sgn * eps
            elif kind == "v":
                c["op"]["frbf"]["w"] = c["op"]["frbf"]["w"].copy()
                c["op"]["frbf"]["w"][idx] += sgn * eps
            else:
                c["op"]["g_coef"] = c["op"]["g_coef"].copy()
                c["op"]["g_coef"][idx] += sgn * eps
            vals.append(J(c)[0])
        fd = (vals[0] - vals[1]) / (2 * eps)
        got = {"w": g[idx] if kind == "w" else None, "v": g[nw + idx] if kind == "v" else None,
               "a": g[nw + nf + idx] if kind == "a" else None}[kind]
        assert abs(fd - got) <= 1e-6 * max(1e-2, abs(fd)), (kind, idx, fd, got)


def test_adaptive_cover_and_rows(pdd):
    """Batching workload: unit disk, 7,108 circles of log-normal radii, grids 16^2..64^2, c from 64
    Gaussians.  Cover bit-exact; one disk of every grid shape and 4 Monte Carlo rows (FP64,
    identical streams) recomputed by the oracle."""
    cfg = workloads.adaptive(paths=200, paths_max=0)
    oc = _oracle_cover("adaptive", cfg)
    cov = pdd.Cover(cfg)
    a = _np(cov.arrays())
    assert (cov.M, cov.N, cov.nnz) == (oc.M, oc.N, oc.col.size)
    for k in ("knot_ptr", "kowner", "row_sub", "rowptr", "col"):
        assert np.array_equal(a[k].astype(np.int64), getattr(oc, k).astype(np.int64)), k
    from oracle import problem, spectral
    op = problem.Operator(cfg["op"], oc.domain)
    for prec in ("mixed", "fp64"):
        S = pdd.System(cov, cfg, prec)
        g = _np(S.csr())
        st = S.stats()
        assert st["unconverged_disks"] == 0
        if prec == "mixed":
            seen = {}
            for m in range(oc.M):
                if oc.floating[m] and oc.sub_rows(m).size and oc.n_r[m] not in seen:
                    seen[oc.n_r[m]] = m
            assert len(seen) >= 5
            for nr, m in seen.items():
                if nr > 40:
                    continue                   # the oracle's QR of n >= 2304 is checked on one grid below
                for i, (cols, v, bi) in spectral.floating_rows(oc, op, int(m)).items():
                    pos = oc.rowptr[i] + np.searchsorted(oc.col[oc.rowptr[i]:oc.rowptr[i + 1]], cols)
                    assert _row_err(g["val"][pos], v) < 1e-10, (nr, m, i)
            m = seen[max(seen)]
            for i, (cols, v, bi) in spectral.floating_rows(oc, op, int(m)).items():
                pos = oc.rowptr[i] + np.searchsorted(oc.col[oc.rowptr[i]:oc.rowptr[i + 1]], cols)
                assert _row_err(g["val"][pos], v) < 1e-10, (max(seen), m, i)
        else:
            mc = _np(S.mc())
            rows = mc["rows"]
            pick = np.random.default_rng(3).choice(rows.size, 4, replace=False)
            ref = osystem.assemble(cfg, oc, rows=[int(rows[k]) for k in pick], threads=4)
            for k in pick:
                r = ref.mc_rows[int(rows[k])]
                got = mc["moments"][mc["mom_ptr"][k]:mc["mom_ptr"][k + 1]]
                assert np.abs(got - r.moments).max() <= 1e-12 * max(1.0, np.abs(r.moments).max())
                assert abs(mc["bmean"][k] - r.b) <= 1e-12 * max(1.0, abs(r.b))


def test_autograd_function_matches_pdd_grad(pdd):
    """torch.autograd through MisfitSolve (forward: assemble + solve; backward: pdd_grad)."""
    cfg = workloads.grad(paths=64)
    w = torch.tensor(cfg["op"]["rbf"]["w"], dtype=torch.float64, device="cuda", requires_grad=True)
    a = torch.tensor(cfg["op"]["g_coef"], dtype=torch.float64, device="cuda", requires_grad=True)
    v = torch.tensor(cfg["op"]["frbf"]["w"], dtype=torch.float64, device="cuda", requires_grad=True)
    u = pdd.MisfitSolve.apply(w, a, cfg, "fp64", v)
    oc = _oracle_cover("grad", cfg)
    u_obs = torch.tensor(np.exp(oc.kx) * np.sin(oc.ky), device="cuda")
    J = ((u - u_obs) ** 2).sum()
    J.backward()
    S = pdd.System(pdd.Cover(cfg), cfg, "fp64")
    u2 = S.solve(rtol=1e-14)
    g = S.grad(u2, 2.0 * (u2 - u_obs))
    nw, nf = w.numel(), v.numel()
    assert torch.allclose(w.grad, g[:nw], rtol=1e-9, atol=1e-12)
    assert torch.allclose(v.grad, g[nw:nw + nf], rtol=1e-9, atol=1e-12)
    assert torch.allclose(a.grad, g[nw + nf:], rtol=1e-9, atol=1e-12)
