"""Accuracy class of the small SVD of B (Alg. RSVD step 4) on a row-graded matrix.

B = D G with D = diag(10^-e_i), e_i evenly from 0 to E, and G an N(0,1) matrix: its
singular values span E decades.  The one-sided Jacobi on the rows of B rotates every
pair whose cosine exceeds n 2^-53, however small the rows, so it determines the singular
values to high relative accuracy (Demmel-Veselic: the error is governed by the condition
number of G, not of B) - beyond the absolute accuracy (errors of order eps ||B||) of the
LAPACK SVD the paper uses.  Rows whose norm falls below 2^-52 of the largest are deflated
to zero at a sweep head (rounding noise of a computed B), so values below that floor come
out as 0 and values a few eps ||B|| above it carry an absolute error of order eps ||B||.
The Alg. TSVD flag (B = A, all m rows; for n >= 3m on the m x m factor A Q_b, which
transforms every row on its own and so keeps the grading) and the exact path of small
matrices (m <= 16, B = A) hand A itself to the Jacobi SVD; the sampled path for larger m
forms B = Q^T A, whose entries carry absolute errors of order eps ||A||.  The reference is the SVD of the same FP64 entries in 40-digit arithmetic
(mpmath).  The factors' nonzero rows/columns are checked for orthonormality.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    need_gpu()
    from paper_1710_01463_gb300 import api as a
    return a


def graded(m, n, decades, seed):
    G = np.random.default_rng(seed).standard_normal((m, n))
    return 10.0 ** (-np.linspace(0.0, decades, m))[:, None] * G


def exact_sigma(A):
    mpmath = pytest.importorskip("mpmath")
    with mpmath.workdps(40):
        s = mpmath.svd_r(mpmath.matrix(A.tolist()), compute_uv=False)
        return np.array(sorted((float(v) for v in s), reverse=True))


@pytest.mark.parametrize("m,n,seed,decades,full", [(24, 40, 1, 12.0, True), (64, 64, 3, 12.0, True),
                                                    (24, 80, 4, 12.0, True), (16, 40, 5, 12.0, False),
                                                    (24, 40, 1, 20.0, True), (40, 64, 2, 20.0, True)])
def test_graded_rows_high_relative_accuracy(api, m, n, seed, decades, full):
    from paper_1710_01463_gb300 import _lib
    A = graded(m, n, decades, seed)
    ref = exact_sigma(A)
    U, S, Vt, info = api.rsvd_truncate(torch.from_numpy(A).cuda(), m, 8, 2, 3,
                                       flags=_lib.RSVD_FLAG_FULL_SVD if full else 0)
    torch.cuda.synchronize()
    d = api.info_dicts(info)[0]
    assert d["status"] == 0
    s = S.cpu().numpy()
    floor = 2.0 ** -52 * ref[0]
    if ref[-1] > floor:  # nothing deflated: every value to high relative accuracy
        assert np.max(np.abs(s - ref) / ref) <= 1e-12
    else:  # rows below the floor are zeroed, a perturbation of at most the floor
        assert np.all(np.abs(s - ref) <= 1e-12 * ref + 2.0 * floor)
        assert np.all(s[ref < 0.5 * floor] == 0.0)
        assert np.max(np.abs(s - ref)[ref > 1e-8 * ref[0]] / ref[ref > 1e-8 * ref[0]]) <= 1e-12
    above = ref > 1e4 * floor
    nz = s > 0
    assert nz.sum() >= above.sum()
    vt = Vt.cpu().numpy()[nz]
    np.testing.assert_allclose(vt @ vt.T, np.eye(int(nz.sum())), atol=1e-13)
    u = U.cpu().numpy()
    np.testing.assert_allclose(u.T @ u, np.eye(m), atol=1e-13)
