"""GPU parity of the RSVD path (C ABI through the Python binding) against the FP64 oracle.

Parity is GPU-RSVD vs oracle-RSVD on the same Philox test matrix (Alg. RSVD),
FP64: singular values within 1e-10 relative (+ 1e-14 sigma_1), singular vectors
within 1e-8 after sign alignment; FP32 products: 1e-4 relative to sigma_1.
"""
import numpy as np
import pytest

from gpu_util import align_columns, need_gpu, sigma_tol, torch
from oracle import philox
from oracle import rsvd as orsvd
from paper_1710_01463_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    need_gpu()
    from paper_1710_01463_gb300 import api as a
    return a


@pytest.mark.parametrize("n,l,seed,stream", [(256, 40, 201, 0), (37, 9, 5, 3), (1, 1, 0, 0), (1000, 17, 2**63 + 5, 77)])
def test_gaussian_matches_oracle(api, n, l, seed, stream):
    om = api.rsvd_gaussian(n, l, seed, stream).cpu().numpy()
    ref = philox.gaussian_test_matrix(n, l, seed, stream)
    np.testing.assert_allclose(om, ref, rtol=1e-13, atol=1e-14)


def check_rsvd(api, A, k, p, q, seed=201, stream=0, dtype=torch.float64, svtol=None, vtol=1e-8):
    At = torch.from_numpy(np.ascontiguousarray(A)).to(dtype).cuda()
    U, S, Vt, info = api.rsvd_truncate(At, k, p, q, seed, stream)
    torch.cuda.synchronize()
    Uo, So, Vto = orsvd.rsvd(At.double().cpu().numpy(), k, p, q, seed, stream)
    s = S.cpu().numpy()
    tol = sigma_tol(So) if svtol is None else svtol * np.max(So)
    assert np.all(np.abs(s - So) <= tol), np.max(np.abs(s - So) / So)
    u = U.double().cpu().numpy()
    vt = Vt.double().cpu().numpy()
    gap_ok = np.ones(k, dtype=bool)
    rel = np.abs(np.diff(So)) / So[0]
    # vectors are compared where the singular value is separated from its neighbours
    for i in range(k):
        near = [rel[i - 1] if i > 0 else 1.0, rel[i] if i < k - 1 else 1.0]
        gap_ok[i] = min(near) > 1e-6 and So[i] > 1e-8 * So[0]
    ua = align_columns(u, Uo)
    np.testing.assert_allclose(ua[:, gap_ok], Uo[:, gap_ok], atol=vtol)
    va = align_columns(vt.T, Vto.T)
    np.testing.assert_allclose(va[:, gap_ok], Vto.T[:, gap_ok], atol=vtol)
    kk = u.shape[1]
    otol = 1e-12 if dtype == torch.float64 else 1e-5
    np.testing.assert_allclose(u.T @ u, np.eye(kk), atol=otol)
    np.testing.assert_allclose(vt @ vt.T, np.eye(kk), atol=otol)
    st = api.info_dicts(info)[0]
    return s, u, vt, st


def test_dense_fp64_256(api):
    A = inputs.dense_case()
    s, u, vt, st = check_rsvd(api, A, 32, 8, 2)
    assert st["status"] == 0 and st["l"] == 40 and st["path"] == 0
    assert st["jacobi_sweeps"] >= 2
    # canonical sign: largest-|.| entry of every u_i positive
    idx = np.argmax(np.abs(u), axis=0)
    assert np.all(u[idx, np.arange(u.shape[1])] > 0)


@pytest.mark.parametrize("m,n,k,p,q", [(37, 23, 5, 4, 1), (100, 300, 10, 6, 2), (300, 100, 10, 6, 2),
                                       (257, 255, 33, 7, 0), (129, 65, 64, 8, 1)])
def test_ragged_shapes_fp64(api, m, n, k, p, q):
    r = min(m, n)
    A = inputs.spectral_matrix(m, n, inputs.exp_spectrum(r, 8.0), 7 + m + n)
    check_rsvd(api, A, k, p, q, seed=11, stream=m)


def test_exact_path_small(api):
    # m <= l: Q = I, the result is the TSVD of A
    A = inputs.random_dense(5, 7, 3)
    At = torch.from_numpy(A).cuda()
    U, S, Vt, info = api.rsvd_truncate(At, 4, 8, 2, 1)
    torch.cuda.synchronize()
    Ut, St, Vtt = orsvd.tsvd(A, 4)
    np.testing.assert_allclose(S.cpu().numpy(), St, rtol=1e-12)
    np.testing.assert_allclose(U.cpu().numpy(), Ut, atol=1e-12)
    np.testing.assert_allclose(Vt.cpu().numpy(), Vtt, atol=1e-12)
    st = api.info_dicts(info)[0]
    assert st["path"] & 1


def test_fp32_products(api):
    A = inputs.spectral_matrix(512, 384, inputs.harmonic_spectrum(384), 5)
    check_rsvd(api, A, 16, 8, 2, dtype=torch.float32, svtol=2e-5, vtol=2e-3)


def test_rank_deficient_takes_householder(api):
    A = inputs.spectral_matrix(120, 90, np.linspace(2.0, 1.0, 5), 17)
    At = torch.from_numpy(A).cuda()
    U, S, Vt, info = api.rsvd_truncate(At, 10, 8, 2, 3)
    torch.cuda.synchronize()
    st = api.info_dicts(info)[0]
    assert st["path"] & 2 and st["chol_fallbacks"] >= 1
    s = S.cpu().numpy()
    np.testing.assert_allclose(s[:5], np.linspace(2.0, 1.0, 5), rtol=1e-12)
    assert np.all(s[5:] < 1e-13 * s[0])
    u = U.cpu().numpy()
    np.testing.assert_allclose(u[:, :5].T @ u[:, :5], np.eye(5), atol=1e-12)
    # the leading factors reproduce A
    np.testing.assert_allclose((u[:, :5] * s[:5]) @ Vt.cpu().numpy()[:5], A, atol=1e-12)


def test_nonfinite_input_reported(api):
    A = inputs.random_dense(40, 30, 1)
    A[3, 4] = np.nan
    U, S, Vt, info = api.rsvd_truncate(torch.from_numpy(A).cuda(), 5, 4, 1, 0)
    torch.cuda.synchronize()
    assert api.info_dicts(info)[0]["status"] == -6


def test_jacobi_exchange_timeout_reported(api):
    # the failure path of the Jacobi SVD's cluster exchange: with the test flag no CTA
    # sends its partials, every CTA's first wait runs out (about 0.13 s), the cluster
    # leaves the iteration together and the status says so; the context stays usable
    from paper_1710_01463_gb300 import _lib
    A = inputs.dense_case(96, 80, seed=101)
    Ad = torch.from_numpy(A).cuda()
    U, S, Vt, info = api.rsvd_truncate(Ad, 12, 6, 2, 201, flags=_lib.RSVD_FLAG_TEST_NO_EXCHANGE)
    torch.cuda.synchronize()
    assert api.info_dicts(info)[0]["status"] == _lib.RSVD_ERR_TIMEOUT
    U, S, Vt, info = api.rsvd_truncate(Ad, 12, 6, 2, 201)
    torch.cuda.synchronize()
    assert api.info_dicts(info)[0]["status"] == 0
    _, So, _ = orsvd.rsvd(A, 12, 6, 2, 201)
    assert np.all(np.abs(S.cpu().numpy() - So) <= sigma_tol(So))


def test_sweep_cap_reported(api):
    A = inputs.dense_case()
    U, S, Vt, info = api.rsvd_truncate(torch.from_numpy(A).cuda(), 32, 8, 2, 201, max_sweeps=1)
    torch.cuda.synchronize()
    st = api.info_dicts(info)[0]
    assert st["status"] == 1 and st["jacobi_sweeps"] == 1


@pytest.mark.parametrize("m,n,k", [(256, 256, 32), (200, 150, 20), (256, 96, 40)])
def test_fp64_product_paths_agree(api, m, n, k):
    # the products with A on the tensor cores by exact slicing (default for m, n <= 256)
    # and on FP64 FMAs (flag) give the oracle's factorization within the FP64 bar
    A = inputs.spectral_matrix(m, n, inputs.exp_spectrum(min(m, n), 12.0), 31 + m)
    At = torch.from_numpy(A).cuda()
    Uo, So, Vto = orsvd.rsvd(A, k, 8, 2, 5, 9)
    out = {}
    for simt in (False, True):
        U, S, Vt, info = api.rsvd_truncate(At, k, 8, 2, 5, 9, simt=simt)
        torch.cuda.synchronize()
        s = S.cpu().numpy()
        assert np.all(np.abs(s - So) <= sigma_tol(So))
        assert api.info_dicts(info)[0]["status"] == 0
        out[simt] = (s, U.cpu().numpy(), Vt.cpu().numpy())
    np.testing.assert_allclose(out[False][0], out[True][0], rtol=1e-11, atol=1e-14 * So[0])
    u0, u1 = out[False][1], out[True][1]
    np.testing.assert_allclose(u0.T @ u0, np.eye(k), atol=1e-12)
    np.testing.assert_allclose(np.abs(np.sum(u0 * u1, axis=0))[:k // 2], 1.0, atol=1e-9)


@pytest.mark.parametrize("m", [384, 512])
def test_blocked_householder_tall_samples(api, m):
    # the bond-matrix heights of the spin-1 chain (3 * 128) and the two-leg cylinder
    # (4 * 128): a spectrum falling through the FP64 floor within l = 138 columns makes
    # CholeskyQR2 fail, so the samples are orthonormalised by the blocked Householder
    # kernel with m rows in shared memory
    A = inputs.spectral_matrix(m, m, inputs.exp_spectrum(m, 4.0), 41 + m)
    s, u, vt, st = check_rsvd(api, A, 128, 10, 2, seed=7, stream=m)
    assert st["status"] == 0 and st["path"] & 2 and st["l"] == 138
