"""rsvd_truncate_noalloc: the truncated factorization of rsvd_truncate with its
scratch in the library's fixed device array instead of a caller workspace.

It serves callers that cannot allocate or own device memory (a framework that
pre-reserves all GPU memory, a fixed-budget real-time loop, a plain C caller
without an allocator).  The entry point is called through the C ABI twice in
a row - on two different inputs, so the second call runs on scratch the first
one left behind - and each result is checked against rsvd_truncate on the same
input within the FP64 parity tolerance used by the other GPU tests.  This file
is collected last so that a run stopping at the first failure has run every
other test before it.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import need_gpu, sigma_tol, torch
from paper_1710_01463_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    need_gpu()
    from paper_1710_01463_gb300 import _lib, api
    return _lib, api


def call_noalloc(_lib, A, k, p, q, seed, stream, cuda_stream=None):
    lib = _lib.load()
    m, n = A.shape
    U = torch.empty((m, k), dtype=A.dtype, device=A.device)
    S = torch.empty((k,), dtype=torch.float64, device=A.device)
    Vt = torch.empty((k, n), dtype=A.dtype, device=A.device)
    info = torch.zeros((1, _lib.INFO_INTS), dtype=torch.int32, device=A.device)
    prec = _lib.RSVD_F64 if A.dtype == torch.float64 else _lib.RSVD_F32
    par = _lib.RsvdParams(k, p, q, prec, seed, stream, 0, 0)
    rc = lib.rsvd_truncate_noalloc(m, n, ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.byref(par),
                                   ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(U.data_ptr()), U.stride(0),
                                   ctypes.c_void_p(Vt.data_ptr()), Vt.stride(0), ctypes.c_void_p(info.data_ptr()),
                                   ctypes.c_void_p((cuda_stream or torch.cuda.current_stream()).cuda_stream))
    return rc, U, S, Vt, info


def compare(api, got, A, k, p, q, seed, stream):
    rc, U, S, Vt, info = got
    assert rc == 0
    U0, S0, Vt0, info0 = api.rsvd_truncate(A, k, p, q, seed, stream)
    torch.cuda.synchronize()
    s, s0 = S.cpu().numpy(), S0.cpu().numpy()
    assert np.all(np.abs(s - s0) <= sigma_tol(s0))
    np.testing.assert_allclose(U.cpu().numpy(), U0.cpu().numpy(), atol=1e-8)
    np.testing.assert_allclose(Vt.cpu().numpy(), Vt0.cpu().numpy(), atol=1e-8)
    assert api.info_dicts(info)[0]["status"] == 0


def test_two_calls_in_a_row_match_workspace_path(mods):
    _lib, api = mods
    A1 = torch.from_numpy(inputs.dense_case()).cuda()
    A2 = torch.from_numpy(inputs.spectral_matrix(300, 200, inputs.exp_spectrum(200, 8.0), 12)).cuda()
    first = call_noalloc(_lib, A1, 32, 8, 2, 201, 0)
    second = call_noalloc(_lib, A2, 20, 6, 2, 7, 3)
    torch.cuda.synchronize()
    compare(api, first, A1, 32, 8, 2, 201, 0)
    compare(api, second, A2, 20, 6, 2, 7, 3)


def test_back_to_back_on_one_stream_same_shape(mods):
    # two calls queued on one non-default stream with no synchronisation between them,
    # same shape and different data: the second call's kernels (and the side streams
    # each call forks from and joins back to that stream) start only after the first
    # call's work on the shared array is done, so both results are right
    _lib, api = mods
    A1 = torch.from_numpy(inputs.dense_case(256, 256, seed=101)).cuda()
    A2 = torch.from_numpy(inputs.spectral_matrix(256, 256, inputs.exp_spectrum(256, 9.0), 33)).cuda()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        first = call_noalloc(_lib, A1, 32, 8, 2, 201, 0, side)
        second = call_noalloc(_lib, A2, 32, 8, 2, 11, 2, side)
    torch.cuda.synchronize()
    compare(api, first, A1, 32, 8, 2, 201, 0)
    compare(api, second, A2, 32, 8, 2, 11, 2)


def test_size_beyond_the_fixed_scratch_is_rejected(mods):
    _lib, api = mods
    lib = _lib.load()
    limit = lib.rsvd_noalloc_scratch_bytes()
    assert limit == 16 << 20
    A = torch.zeros((4096, 4096), dtype=torch.float64, device="cuda")
    rc, *_ = call_noalloc(_lib, A, 64, 16, 2, 0, 0)
    assert rc == _lib.RSVD_ERR_SCRATCH_LIMIT


def test_tensor_core_slices_that_do_not_fit_fall_back_to_fma_products(mods):
    # 768 x 768 at l = 138: the FP64 tensor-core path's slices of A and A^T need about 32 MiB,
    # the FP64-FMA products about 10 MiB: the call runs, with the factorization of the
    # workspace path within the FP64 bar
    _lib, api = mods
    A = torch.from_numpy(inputs.spectral_matrix(768, 768, inputs.exp_spectrum(768, 10.0), 21)).cuda()
    res = call_noalloc(_lib, A, 128, 10, 2, 5, 1)
    torch.cuda.synchronize()
    assert res[0] == 0
    compare(api, res, A, 128, 10, 2, 5, 1)

