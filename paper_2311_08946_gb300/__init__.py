"""Python binding of the GB300 library for the circle-cover interfacial system.

Argument marshalling only: every step runs in the CUDA kernels of
``libpdd_gb300.so`` through the C ABI of ``include/pdd.h``.  There is no CPU
fallback: importing this package fails loudly when the library is missing
or when no CUDA device is present at the first call.

    cov = Cover(workload)                         # a1-a5   pdd_build_cover
    sys = System(cov, workload, "mixed")          # a6-a12  pdd_assemble_G
    u = sys.solve()                               # a13     pdd_solve
    g = sys.grad(u, dJdu)                         # a14     pdd_grad

``workload`` is a description from ``workloads.py`` (domain, cover,
discretisation, coefficient families and Monte Carlo settings).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpdd_gb300.so")

PDD_STATUS = {0: "PDD_OK", 1: "PDD_EINVAL", 2: "PDD_ECOVER_GAP", 3: "PDD_ECIRCLE_OUTSIDE",
              4: "PDD_EKNOT_UNCOVERED", 5: "PDD_ENOCONV", 6: "PDD_EPATH_CAP", 7: "PDD_ENOMEM",
              8: "PDD_ECUDA", 9: "PDD_EDUPLICATE_KNOT"}

_B = {"zero": 0, "sinx_cosy": 1}
_C = {"zero": 0, "quadratic": 1, "rbf": 2}
_F = {"zero": 0, "one": 1, "manufactured": 2, "eq46": 3, "rbf": 4}
_G = {"exp_sin": 0, "sin_cos": 1, "boundary_fourier": 2, "one": 3, "zero": 4, "eq46": 5}
_COVER = {"square_lattice": 0, "hex_lattice": 1, "explicit": 2}
PREC = {"fp64": 0, "mixed": 1}


class PddError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{PDD_STATUS.get(status, status)}: {msg}")
        self.status = status
        self.code = PDD_STATUS.get(status, str(status))


# ---------------------------------------------------------------------------
# C structs (mirror include/pdd.h)
# ---------------------------------------------------------------------------
class _Domain(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("p", ctypes.c_double * 4)]


class _Operator(ctypes.Structure):
    _fields_ = [("b_kind", ctypes.c_int), ("c_kind", ctypes.c_int), ("f_kind", ctypes.c_int),
                ("g_kind", ctypes.c_int), ("n_rbf", ctypes.c_int), ("rbf_x", ctypes.c_void_p),
                ("rbf_y", ctypes.c_void_p), ("rbf_w", ctypes.c_void_p), ("rbf_sigma", ctypes.c_double),
                ("n_gcoef", ctypes.c_int), ("g_coef", ctypes.c_void_p), ("n_frbf", ctypes.c_int),
                ("frbf_x", ctypes.c_void_p), ("frbf_y", ctypes.c_void_p), ("frbf_w", ctypes.c_void_p),
                ("frbf_sigma", ctypes.c_double)]


class _CoverSpec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x_origin", ctypes.c_double), ("y_origin", ctypes.c_double),
                ("spacing", ctypes.c_double), ("radius", ctypes.c_double),
                ("n_knots", ctypes.c_int), ("n_r", ctypes.c_int), ("n_theta", ctypes.c_int),
                ("n_explicit", ctypes.c_int), ("cx", ctypes.c_void_p), ("cy", ctypes.c_void_p),
                ("r", ctypes.c_void_p), ("n_knots_per", ctypes.c_void_p),
                ("n_r_per", ctypes.c_void_p), ("n_theta_per", ctypes.c_void_p),
                ("row_mode", ctypes.c_int)]


ROW_MODE = {"farthest": 0, "averaged": 1}


class _AssemblyOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("floating_method", ctypes.c_int),
                ("paths", ctypes.c_int), ("h", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("imq_c2", ctypes.c_double), ("max_refine", ctypes.c_int),
                ("refine_tol", ctypes.c_double), ("factor", ctypes.c_int),
                ("lu_leaf_width", ctypes.c_int), ("lu_tensor_min", ctypes.c_int),
                ("paths_max", ctypes.c_int), ("se_target", ctypes.c_double), ("boundary_shift", ctypes.c_int),
                ("max_steps", ctypes.c_int), ("disk_precision", ctypes.c_int), ("path_precision", ctypes.c_int),
                ("moment_sums", ctypes.c_int), ("cv_degree", ctypes.c_int)]


STAGE = {None: 0, "fp64": 1, "mixed": 2}
SUMS = {"auto": 0, "fp32": 1, "double_float": 2, "fp64": 3}


class _AssemblyStats(ctypes.Structure):
    _fields_ = [("floating_disks", ctypes.c_int), ("floating_rows", ctypes.c_int),
                ("mc_rows", ctypes.c_int), ("path_steps", ctypes.c_int64),
                ("capped_paths", ctypes.c_int64), ("paths_total", ctypes.c_int64),
                ("extended_rows", ctypes.c_int), ("max_refine_sweeps", ctypes.c_int),
                ("unconverged_disks", ctypes.c_int), ("ms_cover_rows", ctypes.c_double),
                ("ms_disks", ctypes.c_double), ("ms_paths", ctypes.c_double),
                ("ms_finalize", ctypes.c_double), ("ms_operator", ctypes.c_double),
                ("ms_factor", ctypes.c_double), ("ms_refine", ctypes.c_double),
                ("ms_eval", ctypes.c_double), ("lu_blocked", ctypes.c_int), ("lu_leaf_width", ctypes.c_int),
                ("lu_tensor_min", ctypes.c_int), ("ms_trisolve", ctypes.c_double), ("ms_tc_gemm", ctypes.c_double),
                ("disk_solves", ctypes.c_int64), ("tc_gemm_flop", ctypes.c_double),
                ("lu_pivoted_fallback", ctypes.c_int), ("ms_gemm_fused", ctypes.c_double),
                ("gemm_fused_flop", ctypes.c_double), ("gemm_fused_bytes", ctypes.c_double),
                ("gemm_pipe_launches", ctypes.c_int64)]


class _SolveOpts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_iters", ctypes.c_int), ("rtol", ctypes.c_double),
                ("transpose", ctypes.c_int), ("precond", ctypes.c_int)]


PRECOND = {"none": 0, "ras": 1}


class _SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_residual", ctypes.c_double), ("converged", ctypes.c_int)]


EXPORTS = ["pdd_build_cover", "pdd_cover_info", "pdd_cover_arrays", "pdd_destroy_cover",
           "pdd_assemble_G", "pdd_system_csr", "pdd_system_mc", "pdd_system_stats",
           "pdd_destroy_system", "pdd_solve", "pdd_solve_csr", "pdd_solve_csr_noalloc",
           "pdd_spmv_csr", "pdd_batched_gemm_sub_tf32x3", "pdd_batched_gemm_tf32x3", "pdd_grad", "pdd_ras_apply",
           "pdd_cover_rows", "pdd_system_mc_subs", "pdd_split_df",
           "pdd_last_error", "pdd_launch_count", "pdd_version"]

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2311_08946_gb300/build.py "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    for name in EXPORTS:
        getattr(lib, name).restype = i32
    lib.pdd_last_error.restype = ctypes.c_char_p
    lib.pdd_version.restype = ctypes.c_char_p
    lib.pdd_launch_count.restype = i64
    lib.pdd_destroy_cover.restype = None
    lib.pdd_destroy_system.restype = None
    lib.pdd_build_cover.argtypes = [vp, vp, ctypes.POINTER(vp), vp]
    lib.pdd_cover_info.argtypes = [vp, vp, vp, vp, vp]
    lib.pdd_cover_arrays.argtypes = [vp] + [ctypes.POINTER(vp)] * 13
    lib.pdd_destroy_cover.argtypes = [vp]
    lib.pdd_assemble_G.argtypes = [vp, vp, vp, ctypes.POINTER(vp), vp]
    lib.pdd_system_csr.argtypes = [vp] + [ctypes.POINTER(vp)] * 4
    lib.pdd_system_mc.argtypes = [vp, ctypes.POINTER(i32)] + [ctypes.POINTER(vp)] * 4
    lib.pdd_system_stats.argtypes = [vp, vp]
    lib.pdd_destroy_system.argtypes = [vp]
    lib.pdd_solve.argtypes = [vp, vp, vp, vp, vp]
    lib.pdd_solve_csr.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.pdd_solve_csr_noalloc.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.pdd_spmv_csr.argtypes = [i32, vp, vp, vp, vp, vp, i32, vp]
    lib.pdd_split_df.argtypes = [vp, vp, i64, vp]
    i64_ = ctypes.c_longlong
    lib.pdd_batched_gemm_sub_tf32x3.argtypes = [i32, i32, i32, i32, vp, i64_, i32, vp, i64_, i32, vp, i64_,
                                                i32, vp]
    lib.pdd_batched_gemm_tf32x3.argtypes = [i32, i32, i32, i32, vp, i64_, i32, vp, i64_, i32, vp, i64_, i32, i32, vp]
    lib.pdd_grad.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
    _lib = lib
    return lib


def _check(st: int):
    if st != 0:
        raise PddError(st, load().pdd_last_error().decode())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required (the library has no CPU path)")


class _DevArray:
    """A borrowed device array exposed through __cuda_array_interface__."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def _to_tensor(ptr, n: int, dtype) -> torch.Tensor:
    tmap = {torch.float64: "<f8", torch.int32: "<i4", torch.uint8: "|u1"}
    if n == 0 or not ptr:
        return torch.zeros(n, dtype=dtype, device="cuda")
    v = torch.as_tensor(_DevArray(int(ptr), n, tmap[dtype]), device="cuda")
    return v.clone()


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------------------
# marshalling of workload descriptions
# ---------------------------------------------------------------------------
def domain_struct(dom: dict) -> _Domain:
    return _Domain(0 if dom["kind"] == "square" else 1, (ctypes.c_double * 4)(*dom["p"]))


def operator_struct(op: dict):
    """pdd_operator plus the numpy arrays it points to (keep both alive)."""
    keep = []
    rbf = op.get("rbf")
    n_rbf, rx, ry, rw, sig = 0, None, None, None, 1.0
    if rbf is not None and op["c"] == "rbf":
        rx, ry, rw = _f64(rbf["x"]), _f64(rbf["y"]), _f64(rbf["w"])
        keep += [rx, ry, rw]
        n_rbf, sig = rx.size, float(rbf["sigma"])
    gco = op.get("g_coef")
    n_g, gp = 0, None
    if gco is not None and op["g"] == "boundary_fourier":
        gp = _f64(gco)
        keep.append(gp)
        n_g = gp.size
    frbf = op.get("frbf")
    n_f, fx, fy, fw, fsig = 0, None, None, None, 1.0
    if frbf is not None and op["f"] == "rbf":
        fx, fy, fw = _f64(frbf["x"]), _f64(frbf["y"]), _f64(frbf["w"])
        keep += [fx, fy, fw]
        n_f, fsig = fx.size, float(frbf["sigma"])

    def p(a):
        return a.ctypes.data if a is not None else None

    s = _Operator(_B[op["b"]], _C[op["c"]], _F[op["f"]], _G[op["g"]], n_rbf, p(rx), p(ry), p(rw), sig,
                  n_g, p(gp), n_f, p(fx), p(fy), p(fw), fsig)
    return s, keep


def cover_struct(cfg: dict):
    c = cfg["cover"]
    keep = []
    if c["kind"] == "explicit":
        cx, cy, r = _f64(c["cx"]), _f64(c["cy"]), _f64(c["r"])
        nk = np.ascontiguousarray(c["n_knots"], np.int32)
        nr = np.ascontiguousarray(c["n_r"], np.int32)
        nt = np.ascontiguousarray(c["n_theta"], np.int32)
        keep = [cx, cy, r, nk, nr, nt]
        s = _CoverSpec(2, 0, 0, 0.0, 0.0, 0.0, 0.0, 0, 0, 0, cx.size, cx.ctypes.data, cy.ctypes.data,
                       r.ctypes.data, nk.ctypes.data, nr.ctypes.data, nt.ctypes.data,
                       ROW_MODE[c.get("rows", "farthest")])
    else:
        s = _CoverSpec(_COVER[c["kind"]], int(c["nx"]), int(c["ny"]), float(c["x_origin"]),
                       float(c["y_origin"]), float(c["spacing"]), float(c["radius"]),
                       int(cfg["n_knots"]), int(cfg["n_r"]), int(cfg["n_theta"]), 0, None, None, None,
                       None, None, None, ROW_MODE[c.get("rows", "farthest")])
    return s, keep


FACTOR = {"recursive_tc": 0, "blocked": 1, "pivoted_tc": 2}


def assembly_opts(cfg: dict, precision: str = "fp64", floating_method: str = "ps",
                  max_refine: int = 12, refine_tol: float = 1e-12, factor: str = "recursive_tc",
                  lu_leaf_width: int = 0, lu_tensor_min: int = 0, disk_precision: str | None = None,
                  path_precision: str | None = None, moment_sums: str = "auto") -> _AssemblyOpts:
    """pdd_assembly_opts from a workload; disk_precision / path_precision ("fp64" or "mixed")
    override `precision` for one stage, moment_sums picks the mixed paths' basis sums."""
    mc = cfg["mc"]
    return _AssemblyOpts(PREC[precision], 0 if floating_method == "ps" else 1, int(mc["paths"]),
                         float(mc["h"]), int(mc["seed"]), float(cfg.get("imq_c2", 1.5)),
                         int(max_refine), float(refine_tol), FACTOR[factor], int(lu_leaf_width),
                         int(lu_tensor_min), int(mc.get("paths_max", 0)), float(mc.get("se_target", 0.0)),
                         1 if mc.get("boundary_shift", False) else 0, int(mc.get("max_steps", 0)),
                         STAGE[disk_precision], STAGE[path_precision], SUMS[moment_sums],
                         int(mc.get("cv_degree", 0)))


# ---------------------------------------------------------------------------
# handles
# ---------------------------------------------------------------------------
class Cover:
    """pdd_build_cover: cover, interfaces, knots, row owners and the CSR pattern."""

    def __init__(self, cfg: dict, stream=None):
        _require_cuda()
        lib = load()
        self.cfg = cfg
        dom = domain_struct(cfg["domain"])
        spec, keep = cover_struct(cfg)
        h = ctypes.c_void_p()
        _check(lib.pdd_build_cover(ctypes.byref(dom), ctypes.byref(spec), ctypes.byref(h), _stream(stream)))
        self._h = h
        M, Mf, N = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        nnz = ctypes.c_int64()
        _check(lib.pdd_cover_info(h, ctypes.byref(M), ctypes.byref(Mf), ctypes.byref(N), ctypes.byref(nnz)))
        self.M, self.M_floating, self.N, self.nnz = M.value, Mf.value, N.value, nnz.value

    @property
    def handle(self):
        return self._h

    def arrays(self) -> dict:
        """Copies of the cover's device arrays as torch tensors on the current device."""
        ps = [ctypes.c_void_p() for _ in range(13)]
        _check(load().pdd_cover_arrays(self._h, *[ctypes.byref(p) for p in ps]))
        M, N, nnz = self.M, self.N, self.nnz
        names = [("cx", M, torch.float64), ("cy", M, torch.float64), ("r", M, torch.float64),
                 ("floating", M, torch.uint8), ("knot_ptr", M + 1, torch.int32),
                 ("kx", N, torch.float64), ("ky", N, torch.float64), ("ku", N, torch.float64),
                 ("kowner", N, torch.int32), ("kdir", N, torch.uint8), ("row_sub", N, torch.int32),
                 ("rowptr", N + 1, torch.int32), ("col", nnz, torch.int32)]
        npairs = ctypes.c_int()
        pp = [ctypes.c_void_p() for _ in range(2)]
        _check(load().pdd_cover_rows(self._h, ctypes.byref(npairs), *[ctypes.byref(p) for p in pp]))
        torch.cuda.synchronize()
        out = {nm: _to_tensor(p.value, n, dt) for (nm, n, dt), p in zip(names, ps)}
        out["pi_ptr"] = _to_tensor(pp[0].value, N + 1, torch.int32)
        out["pi_sub"] = _to_tensor(pp[1].value, npairs.value, torch.int32)
        return out

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.pdd_destroy_cover(self._h)
            self._h = None


class System:
    """pdd_assemble_G: C (in the cover's CSR pattern) and r."""

    def __init__(self, cov: Cover, cfg: dict | None = None, precision: str = "fp64",
                 floating_method: str = "ps", stream=None, max_refine: int = 12,
                 refine_tol: float = 1e-12, factor: str = "recursive_tc", lu_leaf_width: int = 0,
                 lu_tensor_min: int = 0, disk_precision: str | None = None, path_precision: str | None = None,
                 moment_sums: str = "auto"):
        lib = load()
        self.cov = cov
        self.cfg = cfg or cov.cfg
        self.precision = precision
        self.floating_method = floating_method
        self._op, self._keep = operator_struct(self.cfg["op"])
        self._opts = assembly_opts(self.cfg, precision, floating_method, max_refine, refine_tol, factor,
                                   lu_leaf_width, lu_tensor_min, disk_precision, path_precision, moment_sums)
        h = ctypes.c_void_p()
        _check(lib.pdd_assemble_G(cov.handle, ctypes.byref(self._op), ctypes.byref(self._opts),
                                  ctypes.byref(h), _stream(stream)))
        self._h = h

    def csr(self) -> dict:
        ps = [ctypes.c_void_p() for _ in range(4)]
        _check(load().pdd_system_csr(self._h, *[ctypes.byref(p) for p in ps]))
        n, nnz = self.cov.N, self.cov.nnz
        torch.cuda.synchronize()
        return {"val": _to_tensor(ps[0].value, nnz, torch.float64),
                "b": _to_tensor(ps[1].value, n, torch.float64),
                "se": _to_tensor(ps[2].value, nnz, torch.float64),
                "se_b": _to_tensor(ps[3].value, n, torch.float64)}

    def mc(self) -> dict:
        n = ctypes.c_int()
        ps = [ctypes.c_void_p() for _ in range(4)]
        _check(load().pdd_system_mc(self._h, ctypes.byref(n), *[ctypes.byref(p) for p in ps]))
        k = n.value
        torch.cuda.synchronize()
        rows = _to_tensor(ps[0].value, k, torch.int32)
        mp = _to_tensor(ps[1].value, k + 1, torch.int32)
        nm = int(mp[-1].item()) if k else 0
        sp = ctypes.c_void_p()
        _check(load().pdd_system_mc_subs(self._h, ctypes.byref(sp)))
        return {"rows": rows, "subs": _to_tensor(sp.value, k, torch.int32), "mom_ptr": mp,
                "moments": _to_tensor(ps[2].value, nm, torch.float64),
                "bmean": _to_tensor(ps[3].value, k, torch.float64)}

    def stats(self) -> dict:
        s = _AssemblyStats()
        _check(load().pdd_system_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def solve(self, rtol: float = 1e-13, restart: int = 64, max_iters: int = 20000, out=None,
              stream=None, precond: str = "none"):
        """GMRES(restart) on C u = r; precond "ras": right-preconditioned by the RAS operator (Eq. 45)."""
        u = out if out is not None else torch.empty(self.cov.N, dtype=torch.float64, device="cuda")
        info = _SolveInfo()
        o = _SolveOpts(restart, max_iters, rtol, 0, PRECOND[precond])
        _check(load().pdd_solve(self._h, ctypes.byref(o), _ptr(u), ctypes.byref(info), _stream(stream)))
        self.last_solve = {"iters": info.iters, "rel_residual": info.rel_residual,
                           "converged": info.converged}
        return u

    def ras_apply(self, v: torch.Tensor, stream=None) -> torch.Tensor:
        """y = M_RAS^-1 v (Eq. 44), the operator of solve(precond="ras")."""
        v = v.contiguous()
        y = torch.empty_like(v)
        _check(load().pdd_ras_apply(self._h, _ptr(v), _ptr(y), _stream(stream)))
        return y

    def grad(self, u: torch.Tensor, dJdu: torch.Tensor, stream=None, return_lambda=False):
        """dJ/d(theta) = [RBF weights of c, RBF weights of f, boundary Fourier coefficients of g]
        (a family the operator does not use has no entries)."""
        op = self.cfg["op"]
        n_w = len(op["rbf"]["w"]) if (op["c"] == "rbf" and op.get("rbf") is not None) else 0
        n_f = len(op["frbf"]["w"]) if (op["f"] == "rbf" and op.get("frbf") is not None) else 0
        n_g = len(op["g_coef"]) if (op["g"] == "boundary_fourier" and op.get("g_coef") is not None) else 0
        g = torch.zeros(max(1, n_w + n_f + n_g), dtype=torch.float64, device="cuda")
        lam = torch.empty(self.cov.N, dtype=torch.float64, device="cuda")
        u = u.contiguous()
        dJdu = dJdu.contiguous()
        _check(load().pdd_grad(self.cov.handle, ctypes.byref(self._op), ctypes.byref(self._opts), self._h,
                               _ptr(u), _ptr(dJdu), _ptr(g), _ptr(lam), _stream(stream)))
        g = g[:n_w + n_f + n_g]
        return (g, lam) if return_lambda else g

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.pdd_destroy_system(self._h)
            self._h = None


def solve_csr(rowptr, col, val, b, rtol=1e-13, restart=64, max_iters=20000, transpose=False, stream=None):
    """GMRES on any CSR matrix already in device memory (int32 rowptr/col, float64 val/b)."""
    n = b.numel()
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    info = _SolveInfo()
    o = _SolveOpts(restart, max_iters, rtol, 1 if transpose else 0, 0)
    _check(load().pdd_solve_csr(n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(b), _ptr(u), ctypes.byref(o),
                                ctypes.byref(info), _stream(stream)))
    return u, {"iters": info.iters, "rel_residual": info.rel_residual, "converged": info.converged}


def solve_csr_noalloc(rowptr, col, val, b, u, rtol=1e-13, restart=64, max_iters=20000, stream=None):
    """pdd_solve_csr_noalloc: the CSR GMRES solve on the library's fixed device workspace.

    For callers that cannot allocate device memory while they run; ``u`` is
    a caller-owned float64 device tensor of length n.  Calls that overlap on
    one device race on the shared workspace.
    """
    n = b.numel()
    info = _SolveInfo()
    o = _SolveOpts(restart, max_iters, rtol, 0, 0)
    _check(load().pdd_solve_csr_noalloc(n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(b), _ptr(u),
                                        ctypes.byref(o), ctypes.byref(info), _stream(stream)))
    return {"iters": info.iters, "rel_residual": info.rel_residual, "converged": info.converged}


def spmv_csr(rowptr, col, val, x, transpose=False, stream=None):
    n = x.numel()
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    _check(load().pdd_spmv_csr(n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(x), _ptr(y), 1 if transpose else 0,
                               _stream(stream)))
    return y


def split_df(v, stream=None):
    """The double-float split (hi, lo) of a float64 CUDA tensor, as the double-float moment sums
    apply it: returns a float32 tensor of shape v.shape + (2,)."""
    assert v.dtype == torch.float64 and v.is_cuda and v.is_contiguous()
    out = torch.empty(v.shape + (2,), dtype=torch.float32, device=v.device)
    _check(load().pdd_split_df(_ptr(v), _ptr(out), v.numel(), _stream(stream)))
    return out


def gemm_sub_tf32x3(C, A, B, stream=None):
    """C -= A @ B in place for batched row-major float32 CUDA tensors (b, M, K) x (b, K, N)."""
    b, M, K = A.shape
    N = B.shape[2]
    assert C.shape == (b, M, N) and all(t.is_contiguous() and t.dtype == torch.float32 for t in (A, B, C))
    _check(load().pdd_batched_gemm_sub_tf32x3(b, M, N, K, _ptr(A), M * K, K, _ptr(B), K * N, N, _ptr(C), M * N,
                                              N, _stream(stream)))
    return C


def gemm_tf32x3(C, A, B, subtract=True, stream=None):
    """C -= A @ B (or C = A @ B) through the pipelined kernel, batched row-major float32 tensors."""
    b, M, K = A.shape
    N = B.shape[2]
    assert C.shape == (b, M, N) and all(t.is_contiguous() and t.dtype == torch.float32 for t in (A, B, C))
    _check(load().pdd_batched_gemm_tf32x3(b, M, N, K, _ptr(A), M * K, K, _ptr(B), K * N, N, _ptr(C), M * N, N,
                                          1 if subtract else 0, _stream(stream)))
    return C


def launch_count() -> int:
    return int(load().pdd_launch_count())


class MisfitSolve(torch.autograd.Function):
    """u(theta) with theta = (RBF weights of c, boundary Fourier coefficients of g, and -- when the
    workload's f is "rbf" -- RBF weights of f).

    forward: assemble C, r at theta and solve; backward: the hand-written
    adjoint (pdd_grad).  ``cfg`` is the workload description (its c must be
    "rbf" and its g "boundary_fourier").  ``v`` (f's weights) may be None.
    """

    @staticmethod
    def forward(ctx, w, a, cfg, precision="fp64", v=None):
        c = dict(cfg)
        c["op"] = dict(cfg["op"])
        c["op"]["rbf"] = dict(cfg["op"]["rbf"])
        c["op"]["rbf"]["w"] = w.detach().cpu().numpy()
        c["op"]["g_coef"] = a.detach().cpu().numpy()
        if v is not None:
            c["op"]["frbf"] = dict(cfg["op"]["frbf"])
            c["op"]["frbf"]["w"] = v.detach().cpu().numpy()
        cov = Cover(c)
        sys_ = System(cov, c, precision)
        u = sys_.solve(rtol=1e-14)
        ctx.sys = sys_
        ctx.n_w = w.numel()
        ctx.n_f = len(c["op"]["frbf"]["w"]) if c["op"]["f"] == "rbf" else 0
        ctx.has_v = v is not None
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        (u,) = ctx.saved_tensors
        g = ctx.sys.grad(u, grad_u.to(torch.float64)).to(grad_u.device)
        nw, nf = ctx.n_w, ctx.n_f
        gv = g[nw:nw + nf] if ctx.has_v else None
        return g[:nw], g[nw + nf:], None, None, gv
