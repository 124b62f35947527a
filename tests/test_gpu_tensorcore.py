"""The tcgen05 split-TF32 GEMM (Schur update of the disk LU) against an FP64 reference.

Bar: |C_gpu - C_ref| <= 2^-19 * (|C0| + |A||B|) elementwise -- the split keeps
about 21 bits per product (the dropped lo*lo term is ~2^-22 relative), plus
FP32 accumulation over K.
"""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pdd():
    import paper_2311_08946_gb300 as pkg
    from paper_2311_08946_gb300 import build
    build.build()
    pkg.load()
    return pkg


# aligned shapes take the 16-byte staging path (ragged tiles at the M, N and K edges included:
# 260 x 132 x 68, 96 x 200 x 36); odd extents take the scalar path
@pytest.mark.parametrize("b,M,N,K", [(1, 128, 128, 32), (3, 256, 128, 64), (2, 300, 200, 96),
                                     (4, 512, 384, 512), (3, 260, 132, 68), (2, 96, 200, 36),
                                     (2, 129, 65, 33), (1, 1, 1, 1)])
def test_gemm_sub_matches_fp64(pdd, b, M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(b, M, K, device="cuda", generator=g, dtype=torch.float32)
    B = torch.randn(b, K, N, device="cuda", generator=g, dtype=torch.float32)
    C0 = torch.randn(b, M, N, device="cuda", generator=g, dtype=torch.float32)
    C = C0.clone()
    pdd.gemm_sub_tf32x3(C, A, B)
    ref = C0.double() - torch.bmm(A.double(), B.double())
    bound = 2.0 ** -19 * (C0.double().abs() + torch.bmm(A.double().abs(), B.double().abs()))
    err = (C.double() - ref).abs()
    assert bool((err <= bound).all()), float((err / bound).max())


# the kernel of the pivot-free LU (operands split inside the kernel; tiles of 128 x 64/128/256 by
# N): several tiles per CTA (the persistent grid wraps), ragged M/N/K, the scalar operand path
# (odd leading dimensions), both C -= A B and C = A B
@pytest.mark.parametrize("b,M,N,K", [(1, 128, 128, 32), (3, 256, 128, 64), (2, 300, 200, 96),
                                     (4, 512, 384, 512), (3, 260, 132, 68), (2, 96, 200, 36),
                                     (2, 129, 65, 33), (1, 1, 1, 1), (40, 640, 640, 320), (7, 1536, 64, 64)])
@pytest.mark.parametrize("subtract", [True, False])
def test_pipelined_gemm_matches_fp64(pdd, b, M, N, K, subtract):
    g = torch.Generator(device="cuda").manual_seed(M * 5 + N * 11 + K + (1 if subtract else 0))
    A = torch.randn(b, M, K, device="cuda", generator=g, dtype=torch.float32)
    B = torch.randn(b, K, N, device="cuda", generator=g, dtype=torch.float32)
    C0 = torch.randn(b, M, N, device="cuda", generator=g, dtype=torch.float32)
    C = C0.clone()
    pdd.gemm_tf32x3(C, A, B, subtract=subtract)
    prod = torch.bmm(A.double(), B.double())
    ref = C0.double() - prod if subtract else prod
    bound = 2.0 ** -19 * ((C0.double().abs() if subtract else 0.0) + torch.bmm(A.double().abs(), B.double().abs()))
    err = (C.double() - ref).abs()
    assert bool((err <= bound).all()), float((err / bound).max())


def test_pipelined_gemm_in_place_product(pdd):
    """C = A B with C aliasing A (the leaf panel update L21 = A21 U^-1 of the pivot-free LU)."""
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn(5, 700, 64, device="cuda", generator=g, dtype=torch.float32)
    B = torch.randn(5, 64, 64, device="cuda", generator=g, dtype=torch.float32)
    want = torch.bmm(A.double(), B.double())
    bound = 2.0 ** -19 * torch.bmm(A.double().abs(), B.double().abs())
    pdd.gemm_tf32x3(A, A, B, subtract=False)
    err = (A.double() - want).abs()
    assert bool((err <= bound).all()), float((err / bound).max())


@pytest.mark.parametrize("M,N", [(64, 700), (200, 300)])
def test_pipelined_gemm_in_place_rhs(pdd, M, N):
    """C = A B with C aliasing B (the leaf triangular solve X = L^-1 X of the pivot-free LU): one row
    tile with K = 64 goes through the fused kernel, two row tiles (M = K = 200) through the pre-split
    tiles."""
    g = torch.Generator(device="cuda").manual_seed(M + N)
    A = torch.randn(3, M, M, device="cuda", generator=g, dtype=torch.float32)
    B = torch.randn(3, M, N, device="cuda", generator=g, dtype=torch.float32)
    want = torch.bmm(A.double(), B.double())
    bound = 2.0 ** -19 * torch.bmm(A.double().abs(), B.double().abs())
    pdd.gemm_tf32x3(B, A, B, subtract=False)
    err = (B.double() - want).abs()
    assert bool((err <= bound).all()), float((err / bound).max())


@pytest.mark.parametrize("K", [200, 300])
def test_pipelined_gemm_in_place_lhs_wide(pdd, K):
    """C = A B with C aliasing A and N = K > 64: through the pre-split tiles, which are read in full
    before C is written (in the fused kernel a tile would overwrite columns another tile reads)."""
    g = torch.Generator(device="cuda").manual_seed(K)
    A = torch.randn(2, 333, K, device="cuda", generator=g, dtype=torch.float32)
    B = torch.randn(2, K, K, device="cuda", generator=g, dtype=torch.float32)
    want = torch.bmm(A.double(), B.double())
    bound = 2.0 ** -19 * torch.bmm(A.double().abs(), B.double().abs())
    pdd.gemm_tf32x3(A, A, B, subtract=False)
    err = (A.double() - want).abs()
    assert bool((err <= bound).all()), float((err / bound).max())


def test_gemm_sub_is_not_plain_tf32(pdd):
    # a plain single-pass TF32 product would miss this bar by ~2^8
    A = torch.full((1, 128, 64), 1.0 + 2.0 ** -15, device="cuda")
    B = torch.full((1, 64, 128), 1.0 + 2.0 ** -14, device="cuda")
    C = torch.zeros(1, 128, 128, device="cuda")
    pdd.gemm_sub_tf32x3(C, A, B)
    want = -64.0 * (1.0 + 2.0 ** -15) * (1.0 + 2.0 ** -14)
    assert abs(C[0, 5, 7].item() - want) <= 64 * 2.0 ** -20
