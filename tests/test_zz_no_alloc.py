"""The allocation-free CSR solve against the allocating one (GPU, through the C ABI).

pdd_solve_csr_noalloc serves callers that cannot allocate device memory while
they run; it runs the GMRES kernels on a fixed device array.  Two calls in a
row must each match pdd_solve_csr within the solver tolerance used by the other
tests, the shared array's leftover contents must not leak into the next call,
and oversized requests must be refused before any work.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2311_08946_gb300 as pkg
    from paper_2311_08946_gb300 import build
    build.build()
    return pkg.load()


def _csr(n, seed):
    import scipy.sparse as sp
    A = sp.random(n, n, density=8.0 / n, random_state=seed, format="csr") * 0.1 + sp.eye(n) * 2.0
    A.sort_indices()
    b = np.random.default_rng(seed).standard_normal(n)
    dev = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")
    return (A, dev(A.indptr, torch.int32), dev(A.indices, torch.int32), dev(A.data, torch.float64),
            dev(b, torch.float64))


def _call(fn, n, rp, ci, va, b, u, restart=30, rtol=1e-13, transpose=0):
    import paper_2311_08946_gb300 as pkg
    info = pkg._SolveInfo()
    o = pkg._SolveOpts(restart, 20000, rtol, transpose)
    st = fn(n, ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(ci.data_ptr()),
            ctypes.c_void_p(va.data_ptr()), ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(u.data_ptr()),
            ctypes.byref(o), ctypes.byref(info), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, info


def test_noalloc_matches_allocating_solve_twice(lib):
    rel_tol = 1e-10          # the solver tolerance of the other parity tests
    # small, large, then small again: leftovers of a larger solve in the shared array must not
    # reach a smaller one
    for seed, n in ((3, 3001), (5, 20011), (7, 3001)):
        A, rp, ci, va, b = _csr(n, seed)
        ref = torch.empty(n, dtype=torch.float64, device="cuda")
        st, info = _call(lib.pdd_solve_csr, n, rp, ci, va, b, ref)
        assert st == 0 and info.converged
        for _ in range(2):                 # two calls in a row on the shared array
            u = torch.full((n,), 7.0, dtype=torch.float64, device="cuda")
            st, info2 = _call(lib.pdd_solve_csr_noalloc, n, rp, ci, va, b, u)
            assert st == 0 and info2.converged, lib.pdd_last_error()
            torch.cuda.synchronize()
            d = (u - ref).abs().max().item() / ref.abs().max().item()
            assert d <= rel_tol
            assert info2.iters == info.iters
            r = A @ u.cpu().numpy() - b.cpu().numpy()
            assert np.linalg.norm(r) <= 1.05e-13 * np.linalg.norm(b.cpu().numpy())


def test_noalloc_rejects_oversized_and_transposed(lib):
    A, rp, ci, va, b = _csr(64, 1)
    u = torch.zeros(64, dtype=torch.float64, device="cuda")
    # a request whose workspace exceeds the fixed array is refused before any work
    st, _ = _call(lib.pdd_solve_csr_noalloc, 4_000_000, rp, ci, va, b, u, restart=64)
    assert st == 1 and b"exceeds" in lib.pdd_last_error()
    st, _ = _call(lib.pdd_solve_csr_noalloc, 64, rp, ci, va, b, u, transpose=1)
    assert st == 1


def test_noalloc_allocates_no_device_memory(lib):
    """After one warm-up call, further calls leave the device's free memory unchanged."""
    n = 20011
    A, rp, ci, va, b = _csr(n, 9)
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, info = _call(lib.pdd_solve_csr_noalloc, n, rp, ci, va, b, u)
    assert st == 0 and info.converged
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        st, info = _call(lib.pdd_solve_csr_noalloc, n, rp, ci, va, b, u)
        assert st == 0 and info.converged
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
