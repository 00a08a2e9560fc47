"""GPU parity of rsvd_truncate_complex (Alg. RSVD for complex A, Sec. II.B; the paper's
runs use complex double, Sec. IV) against the oracle's complex Alg. RSVD with the same
real Philox test matrix.

* Complex spectra with Haar-like unitary factors (square, tall, wide, and a size that
  takes the FP64 tensor-core products): singular values within the FP64 bar
  (1e-10 sigma_i + 1e-14 sigma_1), U and V^H within 1e-8 after the phase rule (largest-
  modulus entry of u_i real positive), orthonormal factors.
* Real data in complex storage gives the real algorithm (the oracle's real Alg. RSVD).
* FP32 (complex64): values within 2e-5 sigma_1.
* Alg. TSVD of a complex matrix on the same engine (RSVD_FLAG_FULL_SVD) equals the oracle's
  complex TSVD.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, sigma_tol, torch
from oracle import rsvd as orsvd
from paper_1710_01463_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    need_gpu()
    from paper_1710_01463_gb300 import _lib, api
    return _lib, api


@pytest.mark.parametrize("m,n,k,p,q", [(96, 80, 12, 6, 2), (200, 120, 20, 8, 2), (64, 180, 10, 6, 1),
                                       (300, 300, 40, 10, 2)])
def test_complex_matches_oracle(mods, m, n, k, p, q):
    _lib, api = mods
    A = inputs.complex_spectral_matrix(m, n, inputs.exp_spectrum(min(m, n), 10.0), 40 + m)
    U, S, Vh, info = api.rsvd_truncate_complex(torch.from_numpy(A).cuda(), k, p, q, 201, 3)
    torch.cuda.synchronize()
    assert api.info_dicts(info)[0]["status"] == 0
    Uo, So, Vho = orsvd.rsvd_complex(A, k, p, q, 201, 3)
    s = S.cpu().numpy()
    assert np.all(np.abs(s - So) <= sigma_tol(So))
    u, vh = U.cpu().numpy(), Vh.cpu().numpy()
    np.testing.assert_allclose(u, Uo, atol=1e-8)
    np.testing.assert_allclose(vh, Vho, atol=1e-8)
    np.testing.assert_allclose(u.conj().T @ u, np.eye(k), atol=1e-12)
    np.testing.assert_allclose(vh @ vh.conj().T, np.eye(k), atol=1e-12)
    # the phase rule: the largest-modulus entry of every u_i is real and positive
    j = np.argmax(np.abs(u), axis=0)
    piv = u[j, np.arange(k)]
    assert np.all(piv.real > 0) and np.all(np.abs(piv.imag) <= 1e-14)


def test_real_data_gives_the_real_algorithm(mods):
    _lib, api = mods
    A = inputs.dense_case(120, 100, seed=9)
    U, S, Vh, info = api.rsvd_truncate_complex(torch.from_numpy(A.astype(np.complex128)).cuda(), 16, 8, 2, 5, 0)
    torch.cuda.synchronize()
    Ur, Sr, Vtr = orsvd.rsvd(A, 16, 8, 2, 5, 0)
    assert np.all(np.abs(S.cpu().numpy() - Sr) <= sigma_tol(Sr))
    np.testing.assert_allclose(U.cpu().numpy(), Ur, atol=1e-8)
    np.testing.assert_allclose(Vh.cpu().numpy(), Vtr, atol=1e-8)


def test_complex64_within_fp32_bar(mods):
    _lib, api = mods
    A = inputs.complex_spectral_matrix(160, 140, inputs.exp_spectrum(140, 10.0), 77).astype(np.complex64)
    U, S, Vh, info = api.rsvd_truncate_complex(torch.from_numpy(A).cuda(), 16, 8, 2, 11, 0)
    torch.cuda.synchronize()
    assert api.info_dicts(info)[0]["status"] == 0
    _, So, _ = orsvd.rsvd_complex(A.astype(np.complex128), 16, 8, 2, 11, 0)
    assert np.max(np.abs(S.cpu().numpy() - So)) <= 2e-5 * So[0]


def test_complex_tsvd_on_the_engine(mods):
    _lib, api = mods
    A = inputs.complex_spectral_matrix(70, 90, inputs.exp_spectrum(70, 8.0), 5)
    U, S, Vh, info = api.rsvd_truncate_complex(torch.from_numpy(A).cuda(), 12, 0, 0, 0, 0,
                                               flags=_lib.RSVD_FLAG_FULL_SVD)
    torch.cuda.synchronize()
    assert api.info_dicts(info)[0]["status"] == 0
    Uo, So, Vho = orsvd.tsvd_complex(A, 12)
    assert np.all(np.abs(S.cpu().numpy() - So) <= sigma_tol(So))
    np.testing.assert_allclose(U.cpu().numpy(), Uo, atol=1e-8)
    np.testing.assert_allclose(Vh.cpu().numpy(), Vho, atol=1e-8)
