"""GPU parity of the backward of the truncated factorization
(rsvd_truncate_backward_batched, RSVDTrunc) against the oracle's full-SVD adjoint.

* At the exact factors (FP64), with cotangents on all three outputs, the
  library's Abar matches the adjoint of the full SVD with zero cotangents on the
  discarded triplets to 1e-8 relative (max-norm).
* FP32 products at the exact factors agree to 1e-3.
* The gradient of the loss sum w_i s_i + ||W^T U_k||^2 through RSVDTrunc
  (RSVD forward, library backward) matches the oracle's exact gradient.
* A conjugate-gradient cap that is too small is reported, not silent.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, torch
from oracle import grad as ograd
from paper_1710_01463_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    need_gpu()
    from paper_1710_01463_gb300 import api as a
    return a


def exact_case(m, n, k, seed):
    s_true = 1.0 / (1.0 + 0.3 * np.arange(1, min(m, n) + 1))
    A = inputs.spectral_matrix(m, n, s_true, seed)
    Uf, sf, Vtf = np.linalg.svd(A, full_matrices=False)
    rng = np.random.default_rng(seed)
    Ub = rng.standard_normal((m, k))
    Sb = rng.standard_normal(k)
    Vb = rng.standard_normal((n, k))
    return A, Uf, sf, Vtf, Ub, Sb, Vb


@pytest.mark.parametrize("m,n,k", [(90, 70, 6), (64, 100, 9), (200, 200, 20)])
def test_backward_matches_full_svd_adjoint(api, m, n, k):
    A, Uf, sf, Vtf, Ub, Sb, Vb = exact_case(m, n, k, 3 + m)
    ref = ograd.full_svd_adjoint(Uf, sf, Vtf, Ub, Sb, Vb)
    c = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    Abar, info = api.rsvd_truncate_backward_batched([c(A)], [c(Uf[:, :k])], [c(sf[:k])], [c(Vtf[:k])],
                                                    [c(Ub)], [c(Sb)], [c(Vb.T)], max_iter=400, tol=1e-11)
    torch.cuda.synchronize()
    got = Abar[0].cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-8 * np.max(np.abs(ref))
    assert api.info_dicts(info)[0]["status"] == 0


def test_backward_batched_mixed_cotangents(api):
    cases = [exact_case(60, 50, 5, 11), exact_case(80, 90, 7, 12)]
    c = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    As = [c(A) for A, *_ in cases]
    Us = [c(Uf[:, :Sb.size]) for A, Uf, sf, Vtf, Ub, Sb, Vb in cases]
    Ss = [c(sf[:Sb.size]) for A, Uf, sf, Vtf, Ub, Sb, Vb in cases]
    Vts = [c(Vtf[:Sb.size]) for A, Uf, sf, Vtf, Ub, Sb, Vb in cases]
    Ubs = [c(Ub) for A, Uf, sf, Vtf, Ub, Sb, Vb in cases]
    Abar, info = api.rsvd_truncate_backward_batched(As, Us, Ss, Vts, Ubs, None, None, max_iter=400, tol=1e-13)
    torch.cuda.synchronize()
    for (A, Uf, sf, Vtf, Ub, Sb, Vb), got in zip(cases, Abar):
        k = Sb.size
        ref = ograd.full_svd_adjoint(Uf, sf, Vtf, Ub, np.zeros(k), np.zeros((A.shape[1], k)))
        assert np.max(np.abs(got.cpu().numpy() - ref)) <= 1e-8 * np.max(np.abs(ref))


def test_loss_gradient_through_rsvd_autograd(api):
    m = n = 160
    k = 12
    s_true = 1.0 / (1.0 + 0.3 * np.arange(1, m + 1)) ** 3
    A = inputs.spectral_matrix(m, n, s_true, 41)
    rng = np.random.default_rng(5)
    w = rng.uniform(size=k)
    W = rng.standard_normal((m, 4))
    At = torch.from_numpy(A).cuda().requires_grad_(True)
    U, S, Vt = api.RSVDTrunc.apply(At, k, 20, 3, 7, 0)
    Wt = torch.from_numpy(W).cuda()
    loss = (torch.from_numpy(w).cuda() * S).sum() + ((Wt.T @ U) ** 2).sum()
    loss.backward()
    ref = ograd.loss_grad(A, k, w, W)
    got = At.grad.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-7 * np.max(np.abs(ref))


def test_fp32_backward_at_exact_factors(api):
    # FP32 products: the exact factors rounded to float, Abar within 1e-3 of the FP64 adjoint
    A, Uf, sf, Vtf, Ub, Sb, Vb = exact_case(256, 256, 32, 21)
    ref = ograd.full_svd_adjoint(Uf, sf, Vtf, Ub, Sb, Vb)
    f = lambda x: torch.from_numpy(np.ascontiguousarray(x)).float().cuda()
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    Abar, info = api.rsvd_truncate_backward_batched([f(A)], [f(Uf[:, :32])], [d(sf[:32])], [f(Vtf[:32])],
                                                    [f(Ub)], [d(Sb)], [f(Vb.T)], max_iter=300, tol=1e-6)
    torch.cuda.synchronize()
    got = Abar[0].double().cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-3 * np.max(np.abs(ref))


def test_cg_cap_is_reported(api):
    A, Uf, sf, Vtf, Ub, Sb, Vb = exact_case(90, 70, 6, 5)
    c = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    Abar, info = api.rsvd_truncate_backward_batched([c(A)], [c(Uf[:, :6])], [c(sf[:6])], [c(Vtf[:6])],
                                                    [c(Ub)], None, None, max_iter=1, tol=1e-14)
    torch.cuda.synchronize()
    assert api.info_dicts(info)[0]["status"] == 2


def test_autograd_warns_on_cg_cap(api):
    # RSVDTrunc reads the backward's status: a conjugate-gradient cap that is too small
    # reaches the caller as a RuntimeWarning, not as a silently unconverged gradient
    A = inputs.spectral_matrix(90, 70, 1.0 / (1.0 + 0.3 * np.arange(1, 71)), 5)
    At = torch.from_numpy(A).cuda().requires_grad_(True)
    U, S, Vt = api.RSVDTrunc.apply(At, 6, 10, 2, 3, 0, 1)
    with pytest.warns(RuntimeWarning, match="status 2"):
        ((U[:, :3] ** 2).sum() * 0.0 + (U ** 3).sum() + S.sum()).backward()


def test_autograd_raises_on_nonfinite_input(api):
    A = inputs.spectral_matrix(40, 30, 1.0 / np.arange(1, 31), 6)
    A[3, 4] = np.nan
    with pytest.raises(RuntimeError, match="status -6"):
        api.RSVDTrunc.apply(torch.from_numpy(A).cuda(), 4, 6, 1, 3, 0)
