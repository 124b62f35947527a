"""Problem data of Eq. 1-3 in FP64: the domain Omega and the coefficient families.

The boundary value problem is  L u + c u + f = 0 in Omega, u = g on dOmega
(Eq. 1) with L = (1/2) a:grad^2 + b.grad (Eq. 2) and a = sigma sigma^T (Eq. 3).
Every workload uses sigma = I, so L = (1/2) Laplacian + b.grad.

Families (names are shared with ``workloads.py``):
  b: zero | sinx_cosy                 b = (sin x, cos y)
  c: zero | quadratic | rbf           c = -(1+x^2+y^2) | min(0, sum_p w_p exp(-|x-x_p|^2/(2 s^2)))
  f: zero | one | manufactured | eq46
       manufactured: f = -(L u* + c u*) for u* = sin(pi x) cos(pi y)
       eq46:         f = -(L u46 + c u46) for u46, the exact solution of the Poisson
                     test (Eq. 46); with b = c = 0 this is -(1/2) Lap u46, i.e. the
                     paper's Lap u = F with f = -F/2
  g: exp_sin | sin_cos | boundary_fourier | one | zero | eq46 (g = u46)

Pins: tests check both manufactured sources against finite differences of
their exact solutions, u46 at points where it has a closed value, and that
e^x sin y is harmonic (the Laplacian of the closed form vanishes).
Test infrastructure only.
"""
from __future__ import annotations

import math

import numpy as np


class Domain:
    """Omega: an axis-aligned square (x0, y0, x1, y1) or a disk (cx, cy, R)."""

    def __init__(self, spec: dict):
        self.kind = spec["kind"]
        self.p = [float(v) for v in spec["p"]]
        if self.kind not in ("square", "disk"):
            raise ValueError("domain kind must be square or disk")

    # -- membership ---------------------------------------------------------
    def inside_open(self, x, y):
        """True where (x, y) lies in the open set Omega."""
        if self.kind == "square":
            x0, y0, x1, y1 = self.p
            return (x > x0) & (x < x1) & (y > y0) & (y < y1)
        cx, cy, r = self.p[:3]
        dx = x - cx
        dy = y - cy
        return dx * dx + dy * dy < r * r

    def dist_closed(self, x, y):
        """Euclidean distance from (x, y) to the closed set Omega-bar (0 inside)."""
        if self.kind == "square":
            x0, y0, x1, y1 = self.p
            dx = np.maximum(np.maximum(x0 - x, 0.0), x - x1)
            dy = np.maximum(np.maximum(y0 - y, 0.0), y - y1)
            return np.sqrt(dx * dx + dy * dy)
        cx, cy, r = self.p[:3]
        dx = x - cx
        dy = y - cy
        return np.maximum(np.sqrt(dx * dx + dy * dy) - r, 0.0)

    def contains_closed_disk(self, cx, cy, r):
        """True when the closed disk of centre (cx, cy) and radius r lies in open Omega."""
        if self.kind == "square":
            x0, y0, x1, y1 = self.p
            return (cx - r > x0) & (cx + r < x1) & (cy - r > y0) & (cy + r < y1)
        ox, oy, rr = self.p[:3]
        dx = cx - ox
        dy = cy - oy
        return np.sqrt(dx * dx + dy * dy) + r < rr

    def perimeter(self):
        if self.kind == "square":
            x0, y0, x1, y1 = self.p
            return 2.0 * ((x1 - x0) + (y1 - y0))
        return 2.0 * math.pi * self.p[2]

    def arclength(self, x, y, edge):
        """Arclength of a boundary point, counter-clockwise from (x0, y0).

        ``edge`` is 0 (bottom), 1 (right), 2 (top), 3 (left) for the square;
        the disk measures from angle 0.
        """
        if self.kind == "square":
            x0, y0, x1, y1 = self.p
            w = x1 - x0
            h = y1 - y0
            return np.where(edge == 0, x - x0,
                   np.where(edge == 1, w + (y - y0),
                   np.where(edge == 2, w + h + (x1 - x),
                            2 * w + h + (y1 - y))))
        cx, cy, r = self.p[:3]
        t = np.arctan2(y - cy, x - cx)
        t = np.where(t < 0, t + 2 * math.pi, t)
        return r * t


class Operator:
    """b, c, f and g of Eq. 1 for one workload (all evaluations in FP64)."""

    def __init__(self, op: dict, domain: Domain):
        self.b_kind = op["b"]
        self.c_kind = op["c"]
        self.f_kind = op["f"]
        self.g_kind = op["g"]
        self.domain = domain
        rbf = op.get("rbf")
        if rbf is not None:
            self.rbf_x = np.asarray(rbf["x"], np.float64)
            self.rbf_y = np.asarray(rbf["y"], np.float64)
            self.rbf_w = np.asarray(rbf["w"], np.float64)
            self.rbf_sigma = float(rbf["sigma"])
        else:
            self.rbf_x = self.rbf_y = self.rbf_w = np.zeros(0)
            self.rbf_sigma = 1.0
        gc = op.get("g_coef")
        self.g_coef = np.zeros(0) if gc is None else np.asarray(gc, np.float64)
        if self.c_kind == "rbf" and self.rbf_w.size == 0:
            raise ValueError("c=rbf needs RBF parameters")
        # f = sum_q v_q exp(-|x - x_q|^2 / (2 s_f^2)) (the source family whose weights the adjoint
        # differentiates)
        frbf = op.get("frbf")
        if frbf is not None:
            self.frbf_x = np.asarray(frbf["x"], np.float64)
            self.frbf_y = np.asarray(frbf["y"], np.float64)
            self.frbf_w = np.asarray(frbf["w"], np.float64)
            self.frbf_sigma = float(frbf["sigma"])
        else:
            self.frbf_x = self.frbf_y = self.frbf_w = np.zeros(0)
            self.frbf_sigma = 1.0
        if self.f_kind == "rbf" and self.frbf_w.size == 0:
            raise ValueError("f=rbf needs RBF parameters")

    # -- drift -----------------------------------------------------------------
    def b(self, x, y):
        if self.b_kind == "zero":
            return np.zeros_like(x), np.zeros_like(y)
        if self.b_kind == "sinx_cosy":
            return np.sin(x), np.cos(y)
        raise ValueError(self.b_kind)

    # -- killing rate c <= 0 ---------------------------------------------------
    def rbf_psi(self, x, y):
        """psi_p(x) = exp(-|x - x_p|^2 / (2 sigma^2)), shape (..., n_rbf)."""
        x = np.asarray(x, np.float64)[..., None]
        y = np.asarray(y, np.float64)[..., None]
        dx = x - self.rbf_x
        dy = y - self.rbf_y
        return np.exp(-(dx * dx + dy * dy) / (2.0 * self.rbf_sigma * self.rbf_sigma))

    def frbf_psi(self, x, y):
        """psi^f_q(x) = exp(-|x - x_q|^2 / (2 s_f^2)), shape (..., n_frbf)."""
        x = np.asarray(x, np.float64)[..., None]
        y = np.asarray(y, np.float64)[..., None]
        dx = x - self.frbf_x
        dy = y - self.frbf_y
        return np.exp(-(dx * dx + dy * dy) / (2.0 * self.frbf_sigma * self.frbf_sigma))

    def c(self, x, y):
        if self.c_kind == "zero":
            return np.zeros_like(np.asarray(x, np.float64))
        if self.c_kind == "quadratic":
            return -(1.0 + x * x + y * y)
        if self.c_kind == "rbf":
            s = self.rbf_psi(x, y) @ self.rbf_w
            return np.minimum(s, 0.0)
        raise ValueError(self.c_kind)

    # -- manufactured solution u* = sin(pi x) cos(pi y) -----------------------
    @staticmethod
    def u_star(x, y):
        return np.sin(math.pi * x) * np.cos(math.pi * y)

    # -- exact solution of the Poisson test, Eq. 46 -----------------------------
    @staticmethod
    def u46(x, y):
        """u46 = 3 + sin(s)/3 + tanh(w)/3 with s = sqrt(1 + x^2/100 + y^2/50) and
        w = sin(3x/25 + y/20) + sin(x/20 - 3y/25) (Eq. 46); returns u, u_x, u_y, Lap u.

        Chain rule: Lap sin(s) = cos(s) Lap s - sin(s) |grad s|^2 with
        Lap s = (1/100 + 1/50 - |grad s|^2) / s, and Lap tanh(w) = sech^2(w)
        (Lap w - 2 tanh(w) |grad w|^2) with Lap w = -((3/25)^2 + (1/20)^2) w.
        """
        x = np.asarray(x, np.float64)
        y = np.asarray(y, np.float64)
        s = np.sqrt(1.0 + x * x / 100.0 + y * y / 50.0)
        sx = x / (100.0 * s)
        sy = y / (50.0 * s)
        g2s = sx * sx + sy * sy
        lap_s = (1.0 / 100.0 + 1.0 / 50.0 - g2s) / s
        a = 3.0 * x / 25.0 + y / 20.0
        b = x / 20.0 - 3.0 * y / 25.0
        w = np.sin(a) + np.sin(b)
        wx = 3.0 / 25.0 * np.cos(a) + np.cos(b) / 20.0
        wy = np.cos(a) / 20.0 - 3.0 / 25.0 * np.cos(b)
        lap_w = -((3.0 / 25.0) ** 2 + (1.0 / 20.0) ** 2) * w
        t = np.tanh(w)
        sech2 = 1.0 - t * t
        u = 3.0 + np.sin(s) / 3.0 + t / 3.0
        ux = (np.cos(s) * sx + sech2 * wx) / 3.0
        uy = (np.cos(s) * sy + sech2 * wy) / 3.0
        lap = (np.cos(s) * lap_s - np.sin(s) * g2s + sech2 * (lap_w - 2.0 * t * (wx * wx + wy * wy))) / 3.0
        return u, ux, uy, lap

    def f(self, x, y):
        x = np.asarray(x, np.float64)
        y = np.asarray(y, np.float64)
        if self.f_kind == "zero":
            return np.zeros_like(x)
        if self.f_kind == "one":
            return np.ones_like(x)
        if self.f_kind == "manufactured":
            pi = math.pi
            u = np.sin(pi * x) * np.cos(pi * y)
            ux = pi * np.cos(pi * x) * np.cos(pi * y)
            uy = -pi * np.sin(pi * x) * np.sin(pi * y)
            half_lap = -pi * pi * u            # (1/2)(u_xx + u_yy) = (1/2)(-2 pi^2 u)
            bx, by = self.b(x, y)
            return -(half_lap + bx * ux + by * uy + self.c(x, y) * u)
        if self.f_kind == "eq46":
            u, ux, uy, lap = self.u46(x, y)
            bx, by = self.b(x, y)
            return -(0.5 * lap + bx * ux + by * uy + self.c(x, y) * u)
        if self.f_kind == "rbf":
            return self.frbf_psi(x, y) @ self.frbf_w
        raise ValueError(self.f_kind)

    # -- Dirichlet data --------------------------------------------------------
    def g_fourier_basis(self, s):
        """Boundary Fourier basis at arclength s: [cos(2 pi k s/P)]_{k<K} + [sin]_{k=1..K}."""
        per = self.domain.perimeter()
        n = self.g_coef.size
        kc = (n + 1) // 2
        ks = n - kc
        s = np.asarray(s, np.float64)[..., None]
        cols = [np.cos(2 * math.pi * np.arange(kc) * s / per),
                np.sin(2 * math.pi * np.arange(1, ks + 1) * s / per)]
        return np.concatenate(cols, -1)

    def g(self, x, y, edge=None):
        x = np.asarray(x, np.float64)
        y = np.asarray(y, np.float64)
        if self.g_kind == "exp_sin":
            return np.exp(x) * np.sin(y)
        if self.g_kind == "sin_cos":
            return self.u_star(x, y)
        if self.g_kind == "eq46":
            return self.u46(x, y)[0]
        if self.g_kind == "one":
            return np.ones_like(x)
        if self.g_kind == "zero":
            return np.zeros_like(x)
        if self.g_kind == "boundary_fourier":
            if edge is None:
                edge = self.nearest_edge(x, y)
            s = self.domain.arclength(x, y, edge)
            return self.g_fourier_basis(s) @ self.g_coef
        raise ValueError(self.g_kind)

    def nearest_edge(self, x, y):
        """Index of the square's edge closest to (x, y) (0 bottom, 1 right, 2 top, 3 left)."""
        if self.domain.kind != "square":
            return np.zeros(np.shape(x), np.int64)
        x0, y0, x1, y1 = self.domain.p
        d = np.stack([np.abs(y - y0), np.abs(x - x1), np.abs(y - y1), np.abs(x - x0)], -1)
        return np.argmin(d, -1)
