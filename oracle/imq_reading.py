"""Which length does theta measure in the IMQ basis of Eq. 19?  Test infrastructure only.

Eq. 19 writes phi_j(theta) = ((theta - theta_j)^2 + c^2)^(-1/2) with c^2 = 1.5 (Sec. 4) on
circles of radius about 9 with 44 knots.  Two readings:

  * "radians":   theta is the angle itself; the knot spacing is 2 pi / 44 = 0.143 and
                 c = 1.22 is 8.6 spacings wide, close to the flat limit;
  * "arclength": theta is measured along the interface (s = r theta, in the length units of
                 Omega); the spacing is 9 * 0.143 = 1.29 and c = 1.22 is about one spacing.

Sec. 2.2 states that the ill-conditioning RBF interpolation is known for (stencils of
thousands of knots) does not arise here.  This script puts numbers on both readings with the
oracle alone: kappa(K) of every perimeter stencil; the largest error of the IMQ interpolant of
the exact solution u46 along every perimeter arc (the floor the method's accuracy cannot go
below); and the statistics of Table 1 (rho(C - I), the largest off-diagonal entry, kappa_2(C),
and the RMS error of u against Eq. 46) computed from ONE set of Monte Carlo path records, so
that the readings differ only in the cardinal functions.  Under the arclength reading
phi_l(s) = r^-1 ((u - u_l)^2 + c^2 / r^2)^(-1/2) with u the local angle: the cardinal
functions (Eq. 22) are those of the angle with c^2 / r^2.

Result (1,000 paths): kappa(K) ~7e11 (radians) against ~46 (arclength), but the interpolation
error of u46 is 6e-5 (radians) against 7e-2 (arclength): only the radian reading can reach the
RMS error of 3.7e-5 that Table 1 reports, so the oracle and the library take it.

    python -m oracle.imq_reading [--paths 1000] [--threads 8]
"""
from __future__ import annotations

import argparse
import math
import os
import sys

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    __package__ = "oracle"

from . import cover as cover_mod  # noqa: E402
from . import imq  # noqa: E402
from . import system  # noqa: E402
from .cover import unwrap  # noqa: E402
from .problem import Operator  # noqa: E402


def poisson46_cfg(paths: int) -> dict:
    """The Eq. 46 workload of Sec. 4 at [-50, 50]^2 (radius-9 circles on a pitch-10 lattice)."""
    return {
        "name": "poisson46",
        "domain": {"kind": "square", "p": [-50.0, -50.0, 50.0, 50.0]},
        "cover": {"kind": "square_lattice", "nx": 10, "ny": 10, "x_origin": -45.0, "y_origin": -45.0,
                  "spacing": 10.0, "radius": 9.0},
        "n_knots": 44, "n_r": 22, "n_theta": 44,
        "op": {"b": "zero", "c": "zero", "f": "eq46", "g": "eq46"},
        "mc": {"paths": paths, "h": 0.015, "seed": 0, "boundary_shift": True},
        "imq_c2": 1.5,
    }


def c2_angle(reading: str, c2: float, r: float) -> float:
    """c^2 in squared radians for the cardinal functions of the local angle."""
    return c2 if reading == "radians" else c2 / (r * r)


def rows_under(cov, S, reading: str, c2: float):
    """The Monte Carlo rows' C entries recomputed from the stored path records."""
    vals = S.vals.copy()
    kap = []
    for i, row in S.mc_rows.items():
        m = int(cov.row_sub[i])
        a, b = int(cov.knot_ptr[m]), int(cov.knot_ptr[m + 1])
        us = cov.ku[a:b]
        if not us.size:
            continue
        ce = c2_angle(reading, c2, float(cov.r[m]))
        Kinv = imq.inverse(us, ce)
        rec = row.records
        ut = np.array([unwrap(t, float(cov.theta_s[m])) for t in rec.etheta])
        phi = np.where((rec.side == 0)[:, None], imq.imq(ut, us, ce), 0.0)
        mom = (phi * rec.Y[:, None]).sum(0) / rec.Y.size
        system._put_row(cov, vals, i, np.arange(a, b), -(Kinv.T @ mom))
        kap.append(imq.condition(us, ce))
    return vals, np.array(kap)


def interpolation_error(cov, reading: str, c2: float):
    """Largest |IMQ interpolant - u46| along each perimeter arc (400 points between its end knots)."""
    errs = []
    for m in range(cov.M):
        a, b = int(cov.knot_ptr[m]), int(cov.knot_ptr[m + 1])
        if cov.floating[m] or b - a < 3:
            continue
        us, r = cov.ku[a:b], float(cov.r[m])
        ce = c2_angle(reading, c2, r)
        t = np.linspace(us[0], us[-1], 400)
        th = t + float(cov.theta_s[m])
        x, y = cov.cx[m] + r * np.cos(th), cov.cy[m] + r * np.sin(th)
        inside = cov.domain.inside_open(x, y) | (np.abs(np.abs(x) - 50.0) < 1e-9) | (np.abs(np.abs(y) - 50.0) < 1e-9)
        f = Operator.u46(cov.kx[a:b], cov.ky[a:b])[0]
        fi = imq.cardinal(t[inside], us, ce) @ f
        errs.append(float(np.abs(fi - Operator.u46(x[inside], y[inside])[0]).max()))
    return max(errs), float(np.median(errs))


def statistics(cov, vals, b):
    import scipy.sparse as sp
    N = cov.N
    C = sp.csr_matrix((vals, cov.col, cov.rowptr), shape=(N, N)).toarray()
    off = C - np.diag(np.diag(C))
    sv = np.linalg.svd(C, compute_uv=False)
    rho = float(np.abs(np.linalg.eigvals(C - np.eye(N))).max())
    u = np.linalg.solve(C, b)
    err = u - Operator.u46(cov.kx, cov.ky)[0]
    return {"rho_C_minus_I": rho, "max_offdiag_C": float(off.max()), "kappa2_C": float(sv[0] / sv[-1]),
            "rms_error": float(np.sqrt(np.mean(err * err)))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--paths", type=int, default=1000)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    cfg = poisson46_cfg(a.paths)
    cov = cover_mod.full_cover(cfg)
    S = system.assemble(cfg, cov, threads=a.threads)
    print(f"# Eq. 46 on [-50,50]^2: M = {cov.M}, N = {cov.N}, {len(S.mc_rows)} Monte Carlo rows, "
          f"{a.paths} paths per knot (one set of path records for both readings)")
    print("reading    kappa(K) min/median/max        interp. err of u46 max/median   "
          "rho(C-I)  max offdiag  kappa2(C)  RMS error")
    for reading in ("radians", "arclength"):
        vals, kap = rows_under(cov, S, reading, 1.5)
        st = statistics(cov, vals, S.b)
        ie = interpolation_error(cov, reading, 1.5)
        print(f"{reading:10s} {kap.min():9.3g} {np.median(kap):9.3g} {kap.max():9.3g}   {ie[0]:10.3g} {ie[1]:10.3g}      "
              f"{st['rho_C_minus_I']:8.4f}  {st['max_offdiag_C']:10.4f}  {st['kappa2_C']:9.1f}  "
              f"{st['rms_error']:9.3g}")
    print("Table 1 ([-50,50]^2 column)                                                   "
          "0.9558      0.0445       84.0    3.72e-05")
    sp = 2.0 * math.pi / 44
    print(f"# knot spacing: {sp:.4f} rad; c = {math.sqrt(1.5):.4f} = {math.sqrt(1.5) / sp:.2f} spacings (radians), "
          f"{math.sqrt(1.5) / (9 * sp):.2f} spacings (arclength, r = 9)")


if __name__ == "__main__":
    main()
