"""GPU parity of the fixed-error RSVD (rsvd_truncate_tol) against the oracle's
rsvd_fixed_error on the same Philox test matrices: the chosen rank bit-exact (the
tolerances are kept away from the rank boundaries), the reported error within 1e-6
relative of the oracle's and of the directly computed ||A - U S V^T||_F / ||A||_F,
singular values at the FP64 bar (1e-10 relative + 1e-14 sigma_1)."""
import numpy as np
import pytest

from gpu_util import need_gpu, sigma_tol, torch
from oracle import rsvd as orsvd
from paper_1710_01463_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    need_gpu()
    from paper_1710_01463_gb300 import api as a
    return a


def boundary_safe(A, eps):
    """True when no rank's exact error lies within 5% of eps ||A|| (no rank decision can
    flip on rounding)."""
    s = np.linalg.svd(A, compute_uv=False)
    tails = np.sqrt(np.maximum(0.0, np.cumsum((s ** 2)[::-1])[::-1])) / np.linalg.norm(A)
    return np.all(np.abs(tails / eps - 1.0) > 0.05)


@pytest.mark.parametrize("m,n,eps,k0,kmax", [(256, 256, 9.61e-5, 8, 200), (300, 180, 1e-8, 16, 180),
                                             (200, 200, 0.287, 32, 64), (130, 400, 1.07e-6, 4, 130),
                                             (12, 40, 1e-9, 4, 12), (256, 256, 1.05e-12, 8, 24)])
def test_fixed_error_matches_oracle(api, m, n, eps, k0, kmax):
    A = inputs.spectral_matrix(m, n, inputs.exp_spectrum(min(m, n), 6.0), 3 + m + n)
    assert boundary_safe(A, eps)
    Uo, so, Vto, erro = orsvd.rsvd_fixed_error(A, eps, k0, kmax, 10, 2, 17, 4)
    U, S, Vt, err, info = api.rsvd_truncate_tol(torch.from_numpy(A).cuda(), eps, k0, kmax, 10, 2, 17, 4)
    torch.cuda.synchronize()
    assert api.info_dicts(info)[0]["status"] == 0
    s = S.cpu().numpy()
    assert len(s) == len(so)
    assert np.all(np.abs(s - so) <= sigma_tol(so))
    assert err == pytest.approx(erro, rel=1e-6, abs=1e-15)
    u, vt = U.cpu().numpy(), Vt.cpu().numpy()
    direct = np.linalg.norm(A - (u * s) @ vt) / np.linalg.norm(A)
    assert err == pytest.approx(direct, rel=1e-6, abs=1e-14)
    if erro <= eps:
        assert err <= eps


def test_fixed_error_zero_matrix(api):
    U, S, Vt, err, info = api.rsvd_truncate_tol(torch.zeros((40, 30), dtype=torch.float64, device="cuda"), 1e-6, 4, 30)
    torch.cuda.synchronize()
    assert S.numel() == 1 and float(S[0]) == 0.0 and err == 0.0
