"""Tensor-core product of the mixed-precision path (rsvd_gemm_tc: tcgen05.mma,
TMEM accumulation, TMA-fed) against a plain PyTorch reference of the same op.

Both operands are exactly representable in the kernel's input type, so the
reference is the FP64 product of the same values; the bound is relative to
|A| |B|^T (the sum of absolute products), i.e. pure accumulation/rounding error:
1e-5 for BF16 inputs (FP32 accumulation), 4e-3 for FP32 inputs read as TF32.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    need_gpu()
    from paper_1710_01463_gb300 import _lib
    return _lib


def run(_lib, A, B, prec):
    M, K = A.shape
    N = B.shape[0]
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = _lib.load().rsvd_gemm_tc(M, N, K, prec, ctypes.c_void_p(A.data_ptr()), A.stride(0),
                                  ctypes.c_void_p(B.data_ptr()), B.stride(0), ctypes.c_void_p(C.data_ptr()),
                                  C.stride(0), ctypes.c_void_p(err.data_ptr()), 0,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return C


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (300, 80, 200), (513, 48, 1000), (4096, 80, 4096), (256, 256, 128)])
@pytest.mark.parametrize("kind", ["bf16", "tf32"])
def test_tc_gemm_matches_reference(lib, M, N, K, kind):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    if kind == "bf16":
        A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
        B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
        prec, tol = lib.RSVD_BF16, 1e-5
    else:
        A = torch.randn(M, K, device="cuda", generator=g)
        B = torch.randn(N, K, device="cuda", generator=g)
        prec, tol = lib.RSVD_TF32, 4e-3
    C = run(lib, A, B, prec).double()
    Ad, Bd = A.double(), B.double()
    ref = Ad @ Bd.T
    scale = Ad.abs() @ Bd.abs().T
    assert torch.isfinite(C).all()
    assert bool(((C - ref).abs() <= tol * scale + 1e-30).all()), float(((C - ref).abs() / scale).max())


def test_tc_gemm_rejects_unaligned_stride(lib):
    A = torch.zeros(64, 100, dtype=torch.bfloat16, device="cuda")  # lda * 2 bytes = 200, not a multiple of 16
    B = torch.zeros(16, 100, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(64, 16, dtype=torch.float32, device="cuda")
    rc = lib.load().rsvd_gemm_tc(64, 16, 100, lib.RSVD_BF16, ctypes.c_void_p(A.data_ptr()), 100,
                                 ctypes.c_void_p(B.data_ptr()), 100, ctypes.c_void_p(C.data_ptr()), 16, None, 0, None)
    assert rc == lib.RSVD_ERR_INVALID_SIZE


def test_pipeline_wait_limit_reports_error(lib):
    # no loads are issued, so the MMA thread's wait runs out (about one second);
    # the kernel finishes, reports the timeout, and the context stays usable
    A = torch.zeros(128, 64, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(16, 64, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(128, 16, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.load().rsvd_gemm_tc(128, 16, 64, lib.RSVD_BF16, ctypes.c_void_p(A.data_ptr()), 64,
                                 ctypes.c_void_p(B.data_ptr()), 64, ctypes.c_void_p(C.data_ptr()), 16,
                                 ctypes.c_void_p(err.data_ptr()), 1, None)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 1
    # the device still works
    A2 = torch.ones(128, 64, dtype=torch.bfloat16, device="cuda")
    C2 = run(lib, A2, torch.ones(16, 64, dtype=torch.bfloat16, device="cuda"), lib.RSVD_BF16)
    assert torch.allclose(C2, torch.full_like(C2, 64.0))
