"""The tcgen05 GEMM of the MLP's 256-wide layers (C = A B^T, bf16 operands,
fp32 accumulation in tensor memory, TMA-loaded tiles) against an fp32
product of the same bf16 values, entry by entry: sizes with ragged M and K
tails (TMA fills beyond the edges with zeros), several N tiles, and split K
summed in a fixed order."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    from paper_2303_08879_gb300 import build
    build.build()
    from paper_2303_08879_gb300 import fockdiag
    return fockdiag


def run(fd, A, B, ksplit=1):
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    part = None
    if ksplit > 1:
        part = torch.empty((ksplit, M, N), dtype=torch.float32, device="cuda")
    st = fd.lib().fk_tc_gemm_bf16(M, N, K, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                  ctypes.c_void_p(C.data_ptr()),
                                  ctypes.c_void_p(part.data_ptr()) if part is not None else None, ksplit,
                                  ctypes.c_void_p(status.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return C


@pytest.mark.parametrize("M,N,K,ksplit", [(128, 256, 64, 1), (256, 256, 256, 1), (300, 256, 328, 1),
                                          (1000, 512, 256, 1), (37, 256, 256, 1), (256, 256, 8192, 8),
                                          (256, 256, 20000, 16)])
def test_tc_gemm_matches_fp32_product(fd, M, N, K, ksplit):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + K)
    A = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
    C = run(fd, A, B, ksplit)
    ref = A.double() @ B.double().T
    bound = A.double().abs() @ B.double().abs().T
    err = (C.double() - ref).abs()
    # fp32 accumulation of exact bf16 products: a few ulp of fp32 per term sum
    assert bool((err <= 1e-5 * bound + 1e-6).all()), float((err / (bound + 1e-30)).max())
    # a wrong tile or a dropped K step is far outside that
    assert float(err.max()) < 1e-3 * float(bound.max())
