"""The tcgen05 BF16 GEMM (C = A B^T + bias, optional SiLU; FP32 accumulate)
against a plain PyTorch FP32 reference of the same operation."""
import ctypes as C

import numpy as np
import pytest

from gpu_util import ff

pytestmark = pytest.mark.gpu


def _gemm(A, B, bias=None, act=0, k_chunk=0, want=("Z", "Cf", "Cb")):
    import torch
    f = ff()
    lib = f.library()
    lib.fedfem_gemm_bf16.restype = C.c_int
    lib.fedfem_gemm_bf16.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int,
                                     C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                     C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    M, K = A.shape
    N = B.shape[0]
    dev = A.device
    Z = torch.full((M, N), float("nan"), device=dev)
    Cf = torch.full((M, N), float("nan"), device=dev)
    Cb = torch.zeros((M, N), dtype=torch.bfloat16, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    kc = k_chunk or K
    splits = (K + kc - 1) // kc
    part = torch.empty(max(1, splits * M * N) if splits > 1 else 1, device=dev)
    rc = lib.fedfem_gemm_bf16(A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), M, N, K, k_chunk,
                              bias.data_ptr() if bias is not None else None, act,
                              Z.data_ptr(), N, Cf.data_ptr(), Cb.data_ptr(), N,
                              part.data_ptr() if splits > 1 else None, status.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return Z, Cf, Cb


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (1, 16, 64), (300, 64, 192), (1331, 64, 128),
                                   (257, 192, 64), (520, 256, 128), (4100, 64, 192)])
@pytest.mark.parametrize("act", [0, 1])
def test_gemm_matches_fp32_reference(M, N, K, act):
    import torch
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g)
    Z, Cf, Cb = _gemm(A, B, bias, act)
    ref = A.float() @ B.float().T + bias
    tol = 1e-5 * K
    assert torch.max(torch.abs(Z - ref)).item() <= tol
    y = torch.nn.functional.silu(ref) if act else ref
    assert torch.max(torch.abs(Cf - y)).item() <= tol * 1.5
    assert torch.max(torch.abs(Cb.float() - y) / (1 + torch.abs(y))).item() <= 1e-2


def test_gemm_split_k_is_deterministic_and_matches():
    import torch
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn(64, 4096, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(192, 4096, device="cuda", generator=g).to(torch.bfloat16)
    Z1, _, _ = _gemm(A, B, k_chunk=512)
    Z2, _, _ = _gemm(A, B, k_chunk=512)
    ref = A.float() @ B.float().T
    assert torch.equal(Z1, Z2)
    assert torch.max(torch.abs(Z1 - ref)).item() <= 1e-5 * 4096
