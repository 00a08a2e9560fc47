"""Pins of the oracle's gradient of the truncated factorization.

* central finite differences (h = 1e-6, FP64) of the loss computed from the
  exact TSVD, along random directions and entry by entry on 8 x 8;
* closed form of the singular-value term: d(sum w_i s_i)/dA = U_k diag(w) V_k^T;
* invariance: with k = n for a square A the subspace term is constant, so its
  gradient vanishes.
"""
import numpy as np
import pytest

from oracle import grad
from oracle.rsvd import tsvd
from paper_1710_01463_gb300 import inputs


@pytest.mark.parametrize("shape", [(8, 8), (12, 7), (7, 12), (40, 40)])
def test_gradient_matches_central_differences(shape):
    m, n = shape
    rng = np.random.default_rng(sum(shape))
    A = inputs.spectral_matrix(m, n, 1.0 / (1.0 + 0.3 * np.arange(1, min(m, n) + 1)), 9)
    k = 3
    w = rng.uniform(size=k)
    W = rng.standard_normal((m, 2))
    G = grad.loss_grad(A, k, w, W)
    for _ in range(4):
        D = rng.standard_normal((m, n))
        fd = grad.fd_directional(A, k, w, W, D)
        assert np.sum(G * D) == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_entrywise_fd_8x8():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((8, 8))
    k = 4
    w = rng.uniform(size=k)
    W = rng.standard_normal((8, 3))
    G = grad.loss_grad(A, k, w, W)
    for i in range(8):
        for j in range(8):
            E = np.zeros((8, 8))
            E[i, j] = 1.0
            assert G[i, j] == pytest.approx(grad.fd_directional(A, k, w, W, E), rel=1e-5, abs=1e-7)


def test_singular_value_term_closed_form():
    A = inputs.random_dense(15, 11, 2)
    k = 5
    w = np.random.default_rng(3).uniform(size=k)
    U, s, Vt = tsvd(A, k)
    np.testing.assert_allclose(grad.loss_grad(A, k, w, np.zeros((15, 2))), (U * w) @ Vt, atol=1e-12)


def test_full_rank_subspace_term_vanishes():
    A = inputs.random_dense(10, 10, 4)
    W = np.random.default_rng(5).standard_normal((10, 3))
    G = grad.loss_grad(A, 10, np.zeros(10), W)
    assert np.max(np.abs(G)) < 1e-10
