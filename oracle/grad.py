"""Oracle: derivative of a loss of the truncated factorization (plain FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper has no derivative; the loss and its gradient below are a
differentiable form of the truncated factorization defined here.  Loss of the rank-k
truncation (U_k, s_k, V_k) of A:

    loss(A) = sum_{i<=k} w_i s_i + || W^T U_k ||_F^2,   W in R^{m x r}.

(Reading: ``||U_k W||^2`` with a k x r matrix W would equal ||W||_F^2 for any
A, a constant; with W of m rows it is tr(W^T U_k U_k^T W), which depends only
on the retained left subspace and is invariant under the sign gauge.)

Reference gradient = the adjoint of the FULL SVD with the cotangents of the
discarded triplets set to zero (definition written out):

    A = U S V^T (thin, r = min(m, n)),  F_ij = 1 / (s_j^2 - s_i^2), F_ii = 0
    Abar = U [ (F o (U^T Ubar - Ubar^T U)) S + diag(sbar)
              + S (F o (V^T Vbar - Vbar^T V)) ] V^T
           + (I - U U^T) Ubar S^-1 V^T + U S^-1 Vbar^T (I - V V^T)

with Ubar[:, :k] = 2 W W^T U_k, sbar[:k] = w, Vbar = 0 for this loss.
"""
import numpy as np

from .rsvd import tsvd


def loss(A, k, w, W):
    """sum_{i<=k} w_i s_i + ||W^T U_k||_F^2 from the exact TSVD of A."""
    U, s, _ = tsvd(A, k)
    return float(np.dot(w, s) + np.sum((W.T @ U) ** 2))


def full_svd_adjoint(U, s, Vt, Ubar_k, sbar_k, Vbar_k):
    """Abar for cotangents of the first k singular triplets (zero elsewhere).

    (U, s, Vt) is the thin SVD of A; the cotangents must refer to the same
    sign choice of the singular vectors as U and Vt.
    """
    m, n = U.shape[0], Vt.shape[1]
    V = Vt.T
    r = s.size
    k = sbar_k.size
    Ubar = np.zeros((m, r))
    Vbar = np.zeros((n, r))
    sbar = np.zeros(r)
    Ubar[:, :k] = Ubar_k
    Vbar[:, :k] = Vbar_k
    sbar[:k] = sbar_k
    s2 = s * s
    diff = s2[None, :] - s2[:, None]
    F = np.zeros((r, r))
    off = ~np.eye(r, dtype=bool)
    F[off] = 1.0 / diff[off]
    S = np.diag(s)
    J = F * (U.T @ Ubar - Ubar.T @ U)
    K = F * (V.T @ Vbar - Vbar.T @ V)
    core = J @ S + np.diag(sbar) + S @ K
    out = U @ core @ Vt
    sinv = 1.0 / s
    out += (np.eye(m) - U @ U.T) @ (Ubar * sinv[None, :]) @ Vt
    out += (U * sinv[None, :]) @ Vbar.T @ (np.eye(n) - V @ Vt)
    return out


def loss_cotangents(U_k, w, W):
    """(Ubar_k, sbar_k, Vbar_k) of the loss at the factors U_k (m x k)."""
    return 2.0 * W @ (W.T @ U_k), np.asarray(w, dtype=np.float64).copy(), None


def loss_grad(A, k, w, W):
    """Reference gradient d loss / d A through the full-SVD adjoint."""
    A = np.asarray(A, dtype=np.float64)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    Ub, sb, _ = loss_cotangents(U[:, :k], w, W)
    return full_svd_adjoint(U, s, Vt, Ub, sb, np.zeros((A.shape[1], k)))


def fd_directional(A, k, w, W, D, h=1e-6):
    """Central finite difference of the loss along the direction D."""
    return (loss(A + h * D, k, w, W) - loss(A - h * D, k, w, W)) / (2.0 * h)
