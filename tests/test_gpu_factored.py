"""GPU parity of Alg. RSVD on a matrix given as a product X Y (rsvd_truncate_factored,
Sec. II.A) against the FP64 oracle's Alg. RSVD of the formed product, same Omega.

Tolerances as for rsvd_truncate: FP64 singular values within 1e-10 relative (+ 1e-14
sigma_1), singular vectors within 1e-8 where separated; FP32 2e-5 sigma_1.
"""
import numpy as np
import pytest

from gpu_util import align_columns, need_gpu, sigma_tol, torch
from oracle import rsvd as orsvd
from paper_1710_01463_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    need_gpu()
    from paper_1710_01463_gb300 import api as a
    return a


def factors(m, r, n, seed):
    # X Y with a decaying spectrum: X = U_m diag(s) G, Y = H V_n^T (G, H seeded Gaussian)
    rng = np.random.default_rng(seed)
    c = min(m, n, r)
    A = inputs.spectral_matrix(m, n, inputs.exp_spectrum(min(m, n), 10.0), seed)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    G = rng.standard_normal((c, r)) / np.sqrt(r)
    X = (U[:, :c] * s[:c]) @ G
    Y = np.linalg.pinv(G) @ Vt[:c]
    return X, Y


@pytest.mark.parametrize("m,r,n,k,p,q", [(300, 40, 200, 20, 8, 2), (512, 256, 512, 128, 10, 2), (37, 5, 23, 4, 3, 1),
                                         (4, 8, 16, 4, 10, 2), (129, 300, 65, 30, 8, 0)])
def test_factored_matches_oracle(api, m, r, n, k, p, q):
    X, Y = factors(m, r, n, 7 + m + r)
    A = X @ Y
    Uo, So, Vto = orsvd.rsvd(A, k, p, q, 13, 5)
    U, S, Vt, info = api.rsvd_truncate_factored(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), k, p, q, 13, 5)
    torch.cuda.synchronize()
    assert api.info_dicts(info)[0]["status"] == 0
    s = S.cpu().numpy()
    assert np.all(np.abs(s - So) <= sigma_tol(So)), np.max(np.abs(s - So) / So)
    u, vt = U.cpu().numpy(), Vt.cpu().numpy()
    rel = np.abs(np.diff(So)) / So[0]
    sep = np.array([min(rel[i - 1] if i > 0 else 1.0, rel[i] if i < k - 1 else 1.0) > 1e-6 and So[i] > 1e-8 * So[0]
                    for i in range(k)])
    np.testing.assert_allclose(align_columns(u, Uo)[:, sep], Uo[:, sep], atol=1e-8)
    np.testing.assert_allclose(align_columns(vt.T, Vto.T)[:, sep], Vto.T[:, sep], atol=1e-8)
    np.testing.assert_allclose(u.T @ u, np.eye(k), atol=1e-12)


def test_factored_fp32(api):
    X, Y = factors(256, 64, 300, 3)
    Uo, So, Vto = orsvd.rsvd(X.astype(np.float32).astype(np.float64) @ Y.astype(np.float32).astype(np.float64),
                             16, 8, 2, 1, 0)
    U, S, Vt, info = api.rsvd_truncate_factored(torch.from_numpy(X).float().cuda(), torch.from_numpy(Y).float().cuda(),
                                                16, 8, 2, 1, 0)
    torch.cuda.synchronize()
    assert np.all(np.abs(S.cpu().numpy() - So) <= 2e-5 * So[0])


def test_factored_equals_dense_call(api):
    # the same Alg. RSVD (same Omega) on X Y and on the formed A: the same factorization
    X, Y = factors(200, 64, 180, 11)
    A = torch.from_numpy(X @ Y).cuda()
    U1, S1, V1, _ = api.rsvd_truncate_factored(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), 24, 8, 2, 4, 2)
    U2, S2, V2, _ = api.rsvd_truncate(A, 24, 8, 2, 4, 2)
    torch.cuda.synchronize()
    s1, s2 = S1.cpu().numpy(), S2.cpu().numpy()
    np.testing.assert_allclose(s1, s2, rtol=1e-10, atol=1e-14 * s2[0])
