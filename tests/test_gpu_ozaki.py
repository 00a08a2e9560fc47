"""FP64 products on the tensor cores by exact slicing (rsvd_gemm_f64_tc).

Compared with an extended-precision product (numpy longdouble) of the same
FP64 inputs: the error of every entry is within 4 * 2^-53 * K * max|A_r| *
max|B_c| (the normwise class of an FP64 GEMM), for K in one chunk (<= 256) and
over several chunks (up to 1024); integer inputs give exact results; a row
holding NaN gives NaN in its row of C only.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import need_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    need_gpu()
    from paper_1710_01463_gb300 import _lib
    return _lib.load()


def run(lib, A, B):
    M, K = A.shape
    N = B.shape[0]
    At = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    Bt = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    C = torch.full((M, N), -1.0, dtype=torch.float64, device="cuda")
    ws = lib.rsvd_gemm_f64_tc_workspace_size(M, N, K)
    work = torch.empty(max(ws, 1), dtype=torch.uint8, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.rsvd_gemm_f64_tc(M, N, K, ctypes.c_void_p(At.data_ptr()), K, ctypes.c_void_p(Bt.data_ptr()), K,
                              ctypes.c_void_p(C.data_ptr()), N, ctypes.c_void_p(work.data_ptr()), work.numel(),
                              ctypes.c_void_p(err.data_ptr()), None)
    torch.cuda.synchronize()
    assert rc == 0 and int(err.item()) == 0
    return C.cpu().numpy()


def bound(A, B):
    K = A.shape[1]
    ra = np.max(np.abs(A), axis=1)
    rb = np.max(np.abs(B), axis=1)
    return 4.0 * 2.0 ** -53 * K * ra[:, None] * rb[None, :]


@pytest.mark.parametrize("M,N,K", [(256, 144, 256), (300, 138, 256), (128, 256, 256), (37, 5, 1), (200, 64, 250),
                                   (1, 1, 7), (513, 200, 129), (512, 138, 512), (384, 144, 384), (130, 48, 1024),
                                   (257, 100, 257), (64, 17, 700)])
def test_sliced_product_within_fp64_bound(lib, M, N, K):
    rng = np.random.default_rng(M * 1000 + N + K)
    # rows of widely different scales, entries spanning several binades within a row
    A = rng.standard_normal((M, K)) * np.exp2(rng.integers(-40, 40, size=(M, 1))) * np.exp2(rng.integers(-6, 6, size=(M, K)))
    B = rng.standard_normal((N, K)) * np.exp2(rng.integers(-40, 40, size=(N, 1)))
    if M > 3:
        A[2] = 0.0  # a zero row
    C = run(lib, A, B)
    ref = (A.astype(np.longdouble) @ B.astype(np.longdouble).T)
    diff = np.abs(C.astype(np.longdouble) - ref).astype(np.float64)
    assert np.all(diff <= bound(A, B)), float(np.max(diff / np.maximum(bound(A, B), 1e-300)))
    if M > 3:
        assert np.all(C[2] == 0.0)


def test_integer_inputs_exact(lib):
    rng = np.random.default_rng(3)
    A = rng.integers(-1000, 1000, size=(192, 256)).astype(np.float64)
    B = rng.integers(-1000, 1000, size=(96, 256)).astype(np.float64)
    C = run(lib, A, B)
    np.testing.assert_array_equal(C, (A.astype(np.int64) @ B.astype(np.int64).T).astype(np.float64))


def test_nan_row_propagates(lib):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((130, 64))
    B = rng.standard_normal((48, 64))
    A[129, 5] = np.nan
    C = run(lib, A, B)
    assert np.all(np.isnan(C[129]))
    assert np.all(np.isfinite(C[:129]))


def test_integer_inputs_exact_over_chunks(lib):
    # K = 768: three chunks of 256, each level sum exact, chunks added in FP64 (integers
    # below 2^53 stay exact)
    rng = np.random.default_rng(5)
    A = rng.integers(-1000, 1000, size=(130, 768)).astype(np.float64)
    B = rng.integers(-1000, 1000, size=(40, 768)).astype(np.float64)
    C = run(lib, A, B)
    np.testing.assert_array_equal(C, (A.astype(np.int64) @ B.astype(np.int64).T).astype(np.float64))


def test_rejects_long_k(lib):
    A = torch.zeros((4, 1100), dtype=torch.float64, device="cuda")
    C = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    work = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    rc = lib.rsvd_gemm_f64_tc(4, 4, 1100, ctypes.c_void_p(A.data_ptr()), 1100, ctypes.c_void_p(A.data_ptr()), 1100,
                              ctypes.c_void_p(C.data_ptr()), 4, ctypes.c_void_p(work.data_ptr()), work.numel(), None, None)
    assert rc == -1  # RSVD_ERR_INVALID_SIZE: K <= 1024
