"""Failure paths of the CUDA library, each made to fire on purpose without faulting the GPU.

* a Monte Carlo path that reaches its step cap (max_steps) -> PDD_EPATH_CAP;
* an iterative refinement that cannot meet its tolerance -> PDD_ENOCONV;
* a GMRES solve stopped by its iteration cap -> PDD_ENOCONV;
* a grid barrier of the fused Arnoldi kernel that cannot complete (a host-side injection
  makes it wait for one block more than the grid holds): every block gives up after its
  bounded wait and returns, the solve reports PDD_ECUDA, and the next solve on the same
  context succeeds;
* options out of range -> PDD_EINVAL before any device work.
"""
import os

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pdd():
    import paper_2311_08946_gb300 as pkg
    from paper_2311_08946_gb300 import build
    build.build()
    pkg.load()
    return pkg


def test_path_step_cap(pdd):
    cfg = workloads.tiny(paths=64)
    cfg["mc"]["max_steps"] = 5                  # far below the mean exit time (~r^2 / (2 h) = 200 steps)
    cov = pdd.Cover(cfg)
    with pytest.raises(pdd.PddError) as e:
        pdd.System(cov, cfg, "fp64")
    assert e.value.code == "PDD_EPATH_CAP"
    assert "step cap" in str(e.value)
    # the same cover assembles once the cap is the default 50 r^2 / h
    cfg["mc"]["max_steps"] = 0
    S = pdd.System(cov, cfg, "fp64")
    assert S.stats()["capped_paths"] == 0


def test_refinement_not_converging(pdd):
    cfg = workloads.tiny(paths=64)
    cov = pdd.Cover(cfg)
    with pytest.raises(pdd.PddError) as e:
        pdd.System(cov, cfg, "mixed", max_refine=1, refine_tol=1e-16)
    assert e.value.code == "PDD_ENOCONV"
    assert "refinement" in str(e.value)


def test_gmres_iteration_cap(pdd):
    cfg = workloads.tiny(paths=64)
    S = pdd.System(pdd.Cover(cfg), cfg, "fp64")
    with pytest.raises(pdd.PddError) as e:
        S.solve(rtol=1e-14, restart=2, max_iters=2)
    assert e.value.code == "PDD_ENOCONV"
    assert S.solve(rtol=1e-13).shape[0] > 0


def test_grid_barrier_timeout_is_reported(pdd):
    import scipy.sparse as sp
    n = 5000
    A = sp.random(n, n, density=8.0 / n, random_state=2, format="csr") * 0.1 + sp.eye(n) * 2.0
    A.sort_indices()
    dev = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")
    rp, ci, va = dev(A.indptr, torch.int32), dev(A.indices, torch.int32), dev(A.data, torch.float64)
    b = dev(np.random.default_rng(2).standard_normal(n), torch.float64)
    os.environ["PDD_INJECT_BARRIER_TIMEOUT"] = "1"
    try:
        with pytest.raises(pdd.PddError) as e:
            pdd.solve_csr(rp, ci, va, b, rtol=1e-12)
    finally:
        del os.environ["PDD_INJECT_BARRIER_TIMEOUT"]
    assert e.value.code == "PDD_ECUDA" and "barrier" in str(e.value)
    # the context is still usable: the same solve without the injection converges
    u, info = pdd.solve_csr(rp, ci, va, b, rtol=1e-12)
    assert info["converged"]
    r = A @ u.cpu().numpy() - b.cpu().numpy()
    assert np.linalg.norm(r) <= 1.05e-12 * np.linalg.norm(b.cpu().numpy())


def test_options_out_of_range(pdd):
    cfg = workloads.tiny(paths=64)
    cov = pdd.Cover(cfg)
    for kw in ({"disk_precision": "fp64"}, {"path_precision": "mixed"}, {"moment_sums": "fp64"}):
        pdd.System(cov, cfg, "mixed", **kw)       # valid choices run
    import ctypes
    for field, value in (("max_steps", -1), ("disk_precision", 7), ("path_precision", -2), ("moment_sums", 9)):
        o = pdd.assembly_opts(cfg, "fp64")
        setattr(o, field, value)
        op, keep = pdd.operator_struct(cfg["op"])
        h = ctypes.c_void_p()
        st = pdd.load().pdd_assemble_G(cov.handle, ctypes.byref(op), ctypes.byref(o), ctypes.byref(h), None)
        assert st == 1, field
        assert not h.value
