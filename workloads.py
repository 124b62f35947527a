"""Seeded synthetic inputs for the six workloads of the circle-cover interfacial system.

This module only describes problems: domains, cover lattices (or, for the
adaptive cover, explicitly drawn centres and radii), coefficient families,
coefficient parameters and Monte Carlo settings.  It holds none of the
method's arithmetic (no cover classification, no knots, no operators, no
paths); both the CUDA library and the FP64 oracle take these descriptions and
carry out every step of the method on their own.

Workloads (the problem is Eq. 1 with L = 1/2 Laplacian + b.grad, sigma = I):

* ``tiny``      -- Omega=[0,1]^2, L=1/2 Lap, f=0, g=e^x sin y; 4x4 lattice of circles
                   (radius 0.2, spacing 0.25); 16 knots per circle; 16(r)x16(theta)
                   disk grid; 1,000 paths per Monte Carlo knot, h=1e-4.
* ``varcoef``   -- Omega=[0,2]^2, b=(sin x, cos y), c=-(1+x^2+y^2), f and g from the
                   manufactured u=sin(pi x)cos(pi y); hexagonal lattice (R=0.05,
                   spacing 0.07, ~940 circles); 32 knots; 32x32 grid; 10^4 paths,
                   h=1e-5.
* ``scaled``    -- the ``tiny`` operator and data on [0,4]^2 with a 62x62 lattice
                   (radius/spacing = 0.8 as in ``tiny``); 48(r)x64(theta) grid,
                   16 knots; 1,000 paths, h=1e-5.
* ``adaptive``  -- unit disk, c(x) from 64 Gaussian RBFs (clipped to <= 0), f=0,
                   g=e^x sin y; ~10^4 circles with log-normal radii in [0.02, 0.1];
                   per-circle grids 16^2..64^2 chosen by radius; 10^3 pilot paths per
                   Monte Carlo knot, up to 10^5 where its standard error exceeds 2e-3.
* ``grad``      -- ``tiny`` geometry; parameters are 64 RBF weights of c, 16 RBF
                   weights of the source f and 32 Fourier coefficients of g along the
                   boundary arclength.
* ``poisson46`` -- the paper's Poisson test (Sec. 4, Eq. 46) on [-50,50]^2: f and g from
                   its exact solution u46, L = 1/2 Lap (so 1/2 Lap u = F/2 with
                   F = Lap u46); 10x10 square lattice of circles of radius 9 (the
                   paper's radii lie in [8.55, 9.43]; its layout figure is not
                   available); 44 knots per circle; 22(r)x44(theta) disk grid (968
                   nodes); 5,000 paths per Monte Carlo knot, h = 0.015, boundary
                   shift on (Gobet-Menozzi), pathwise variance reduction on (the
                   regression control variate on the monomials of degree <= 4);
                   c^2 = 1.5.

The random draws a workload needs (RBF centres and weights, adaptive radii,
observation noise) are made here with numpy's seeded generators and passed to
both sides as plain arrays.  The Monte Carlo normals are the one exception: they
are drawn inside each side by Philox4x32-10 from (seed, knot, path, step).
"""
from __future__ import annotations

import math

import numpy as np

# --------------------------------------------------------------------------
# Coefficient-family vocabulary shared by both sides (names only).
#   b:  "zero" | "sinx_cosy"                   b = (sin x, cos y)
#   c:  "zero" | "quadratic" | "rbf"           c = -(1+x^2+y^2) | min(0, sum_p w_p psi_p(x))
#   f:  "zero" | "one" | "manufactured" | "eq46" | "rbf"
#                                              manufactured from u = sin(pi x) cos(pi y) |
#                                              from u46, the exact solution of Eq. 46 |
#                                              sum_q v_q exp(-|x-x_q|^2/(2 s_f^2))
#   g:  "exp_sin" | "sin_cos" | "boundary_fourier" | "one" | "zero" | "eq46"
# --------------------------------------------------------------------------


def _square(x0, y0, x1, y1):
    return {"kind": "square", "p": [float(x0), float(y0), float(x1), float(y1)]}


def _disk(cx, cy, r):
    return {"kind": "disk", "p": [float(cx), float(cy), float(r), 0.0]}


def tiny(paths: int = 1000, h: float = 1e-4, seed: int = 0) -> dict:
    """4x4 square lattice on the unit square, harmonic e^x sin y."""
    return {
        "name": "tiny",
        "domain": _square(0, 0, 1, 1),
        "cover": {"kind": "square_lattice", "nx": 4, "ny": 4, "x_origin": 0.125,
                  "y_origin": 0.125, "spacing": 0.25, "radius": 0.2},
        "n_knots": 16, "n_r": 16, "n_theta": 16,
        "op": {"b": "zero", "c": "zero", "f": "zero", "g": "exp_sin"},
        "mc": {"paths": paths, "h": h, "seed": seed},
        "imq_c2": 1.5,
    }


def varcoef(paths: int = 10000, h: float = 1e-5, seed: int = 0) -> dict:
    """Hexagonal lattice on [0,2]^2 with variable drift and killing rate."""
    s = 0.07
    # rows k >= 0 at y = k*s*sqrt(3)/2, columns i >= 0; circles that miss the
    # domain are dropped by the cover step, so the index box may overshoot.
    return {
        "name": "varcoef",
        "domain": _square(0, 0, 2, 2),
        "cover": {"kind": "hex_lattice", "nx": 30, "ny": 35, "x_origin": 0.0,
                  "y_origin": 0.0, "spacing": s, "radius": 0.05},
        "n_knots": 32, "n_r": 32, "n_theta": 32,
        "op": {"b": "sinx_cosy", "c": "quadratic", "f": "manufactured", "g": "sin_cos"},
        "mc": {"paths": paths, "h": h, "seed": seed},
        "imq_c2": 1.5,
    }


def scaled(paths: int = 1000, h: float = 1e-5, seed: int = 0) -> dict:
    """``tiny`` scaled to [0,4]^2 with a 62x62 lattice and a 48x64 disk grid."""
    s = 4.0 / 62.0
    return {
        "name": "scaled",
        "domain": _square(0, 0, 4, 4),
        "cover": {"kind": "square_lattice", "nx": 62, "ny": 62, "x_origin": 0.5 * s,
                  "y_origin": 0.5 * s, "spacing": s, "radius": 0.8 * s},
        "n_knots": 16, "n_r": 48, "n_theta": 64,
        "op": {"b": "zero", "c": "zero", "f": "zero", "g": "exp_sin"},
        "mc": {"paths": paths, "h": h, "seed": seed},
        "imq_c2": 1.5,
    }


def rbf_field(n: int = 64, seed: int = 1, sigma: float = 0.2, negative: bool = False,
              domain: dict | None = None) -> dict:
    """Gaussian RBF parameters for c(x) = min(0, sum_p w_p exp(-|x-x_p|^2/(2 sigma^2))).

    Centres are uniform in the domain (rejection sampling for a disk); weights
    are N(0,1), or -|N(0,1)| when ``negative`` (then the clip is never active).
    """
    rng = np.random.default_rng(seed)
    domain = domain or _disk(0, 0, 1)
    p = domain["p"]
    xs, ys = [], []
    while len(xs) < n:
        if domain["kind"] == "disk":
            x, y = rng.uniform(-1, 1, 2)
            if x * x + y * y < 1.0:
                xs.append(p[0] + p[2] * x)
                ys.append(p[1] + p[2] * y)
        else:
            xs.append(rng.uniform(p[0], p[2]))
            ys.append(rng.uniform(p[1], p[3]))
    w = rng.standard_normal(n)
    if negative:
        w = -np.abs(w)
    return {"x": np.array(xs), "y": np.array(ys), "w": np.asarray(w, dtype=np.float64),
            "sigma": float(sigma)}


def adaptive(paths: int = 1000, h: float = 1e-5, seed: int = 0, cells: int = 16,
             paths_max: int = 100000, se_target: float = 2e-3) -> dict:
    """Unit disk with an adaptive cover of log-normal radii (drawn here, seed 0).

    The domain's bounding box [-1,1]^2 is cut into ``cells`` x ``cells`` macro
    cells.  Each cell draws r ~ LogNormal(ln 0.025, 0.5) clipped to
    [0.02, 0.1] and is filled by an evenly spaced sub-lattice whose spacing is
    at most 0.9 r (so the cell, its edges included, is covered by its own
    circles).  Circles that do not meet the unit disk are dropped by the cover
    step.  Grid and knot counts grow with the radius: n_r = n_theta = knots =
    16 + 8*round(6 (r-0.02)/0.08).
    """
    rng = np.random.default_rng(seed)
    cw = 2.0 / cells
    cx, cy, rr = [], [], []
    for j in range(cells):
        for i in range(cells):
            r = float(np.clip(rng.lognormal(math.log(0.025), 0.5), 0.02, 0.1))
            m = int(math.ceil(cw / (0.9 * r)))
            sp = cw / m
            for b in range(m):
                for a in range(m):
                    cx.append(-1.0 + i * cw + (a + 0.5) * sp)
                    cy.append(-1.0 + j * cw + (b + 0.5) * sp)
                    rr.append(r)
    rr = np.array(rr)
    nper = 16 + 8 * np.rint(6.0 * (rr - 0.02) / 0.08).astype(np.int64)
    nper = np.clip(nper, 16, 64)
    return {
        "name": "adaptive",
        "domain": _disk(0, 0, 1),
        "cover": {"kind": "explicit", "cx": np.array(cx), "cy": np.array(cy), "r": rr,
                  "n_knots": nper.astype(np.int32), "n_r": nper.astype(np.int32),
                  "n_theta": nper.astype(np.int32)},
        "n_knots": 0, "n_r": 0, "n_theta": 0,
        "op": {"b": "zero", "c": "rbf", "f": "zero", "g": "exp_sin",
               "rbf": rbf_field(64, seed=1, sigma=0.2, negative=False)},
        # pilot of `paths` per Monte Carlo knot, then up to paths_max where the largest
        # standard error of the row exceeds se_target
        "mc": {"paths": paths, "h": h, "seed": seed, "paths_max": paths_max, "se_target": se_target},
        "imq_c2": 1.5,
    }


def boundary_fourier_fit(domain: dict, n_cos: int = 16, n_sin: int = 16,
                         samples: int = 4096) -> np.ndarray:
    """Least-squares Fourier coefficients of e^x sin y along the square's arclength.

    The boundary is walked counter-clockwise from (x0, y0); with perimeter P,
    g(s) = sum_{k<n_cos} a_k cos(2 pi k s/P) + sum_{k=1..n_sin} b_k sin(2 pi k s/P).
    This is input preparation (the base coefficients of the ``grad`` workload).
    """
    x0, y0, x1, y1 = domain["p"]
    w, hgt = x1 - x0, y1 - y0
    per = 2 * (w + hgt)
    s = (np.arange(samples) + 0.5) * per / samples
    x = np.empty(samples)
    y = np.empty(samples)
    e0 = s < w
    e1 = (s >= w) & (s < w + hgt)
    e2 = (s >= w + hgt) & (s < 2 * w + hgt)
    e3 = s >= 2 * w + hgt
    x[e0], y[e0] = x0 + s[e0], y0
    x[e1], y[e1] = x1, y0 + (s[e1] - w)
    x[e2], y[e2] = x1 - (s[e2] - w - hgt), y1
    x[e3], y[e3] = x0, y1 - (s[e3] - 2 * w - hgt)
    cols = [np.cos(2 * np.pi * k * s / per) for k in range(n_cos)]
    cols += [np.sin(2 * np.pi * k * s / per) for k in range(1, n_sin + 1)]
    a = np.stack(cols, 1)
    coef, *_ = np.linalg.lstsq(a, np.exp(x) * np.sin(y), rcond=None)
    return coef


def grad(paths: int = 1000, h: float = 1e-4, seed: int = 0, perturbed: bool = False,
         with_f: bool = True) -> dict:
    """``tiny`` geometry with c from 64 negative-weight RBFs, Fourier boundary data and (with_f)
    a source f from 16 Gaussian RBFs (width 0.25, weights 0.5 N(0,1), seed 3).

    ``perturbed`` gives the parameter set the observations are made from:
    w_p (1 + 0.1 N(0,1)) with seed 1, the g coefficients shifted by 0.01 N(0,1) with seed 1
    and the f weights v_q (1 + 0.1 N(0,1)) with seed 4.
    """
    cfg = tiny(paths, h, seed)
    cfg["name"] = "grad"
    rbf = rbf_field(64, seed=0, sigma=0.2, negative=True, domain=cfg["domain"])
    gco = boundary_fourier_fit(cfg["domain"])
    frbf = rbf_field(16, seed=3, sigma=0.25, negative=False, domain=cfg["domain"])
    frbf["w"] = 0.5 * frbf["w"]
    if perturbed:
        rng = np.random.default_rng(1)
        rbf = dict(rbf)
        rbf["w"] = rbf["w"] * (1.0 + 0.1 * rng.standard_normal(rbf["w"].shape[0]))
        gco = gco + 0.01 * rng.standard_normal(gco.shape[0])
        frbf = dict(frbf)
        frbf["w"] = frbf["w"] * (1.0 + 0.1 * np.random.default_rng(4).standard_normal(frbf["w"].shape[0]))
    cfg["op"] = {"b": "zero", "c": "rbf", "f": "rbf" if with_f else "zero", "g": "boundary_fourier",
                 "rbf": rbf, "g_coef": gco}
    if with_f:
        cfg["op"]["frbf"] = frbf
    return cfg


def observation_noise(n: int, seed: int = 2, variance: float = 1e-4) -> np.ndarray:
    """N(0, variance) noise added to the observed interfacial solution."""
    return np.random.default_rng(seed).normal(0.0, math.sqrt(variance), n)


def floating_only_disk(radius: float = 0.3, n_knots: int = 16, n_r: int = 16,
                       n_theta: int = 16) -> dict:
    """A single floating circle inside a large square (used by the closed-form checks)."""
    return {
        "name": "one_disk",
        "domain": _square(-1, -1, 1, 1),
        "cover": {"kind": "explicit", "cx": np.array([0.1]), "cy": np.array([-0.05]),
                  "r": np.array([radius]), "n_knots": np.array([n_knots], np.int32),
                  "n_r": np.array([n_r], np.int32), "n_theta": np.array([n_theta], np.int32)},
        "n_knots": 0, "n_r": 0, "n_theta": 0,
        "op": {"b": "zero", "c": "zero", "f": "zero", "g": "exp_sin"},
        "mc": {"paths": 1000, "h": 1e-4, "seed": 0},
        "imq_c2": 1.5,
    }


def poisson46(paths: int = 5000, h: float = 0.015, seed: int = 0, half_width: float = 50.0,
              boundary_shift: bool = True, cv_degree: int = 4) -> dict:
    """Poisson's equation with the exact solution of Eq. 46 on [-L, L]^2, L = half_width.

    Circles of radius 9 on a square lattice of pitch 10 (centres at -L + 5, ..., L - 5),
    44 knots each, 22 x 44 pseudospectral nodes on the floating disks, as in Sec. 4.
    """
    n = int(round(2.0 * half_width / 10.0))
    return {
        "name": "poisson46",
        "domain": _square(-half_width, -half_width, half_width, half_width),
        "cover": {"kind": "square_lattice", "nx": n, "ny": n, "x_origin": -half_width + 5.0,
                  "y_origin": -half_width + 5.0, "spacing": 10.0, "radius": 9.0},
        "n_knots": 44, "n_r": 22, "n_theta": 44,
        "op": {"b": "zero", "c": "zero", "f": "eq46", "g": "eq46"},
        "mc": {"paths": paths, "h": h, "seed": seed, "boundary_shift": boundary_shift,
               "cv_degree": cv_degree},
        "imq_c2": 1.5,
    }


WORKLOADS = {"tiny": tiny, "varcoef": varcoef, "scaled": scaled, "adaptive": adaptive,
             "grad": grad, "poisson46": poisson46}
