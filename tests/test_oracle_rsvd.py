"""Pins of the oracle's Alg. TSVD and Alg. RSVD (Sec. II) against mathematics.

* prescribed spectra of A = U diag(s) V^T are recovered;
* Eckart-Young-Mirsky: the Frobenius error of the rank-k truncation is
  sqrt(sum_{j>k} s_j^2) and the spectral error is s_{k+1} (Sec. II.A);
* 2 x 2 brute force: singular values from the eigenvalues of A^T A in closed form;
* exactness: l >= rank(A) reproduces the TSVD;
* interlacing: every RSVD singular value is <= the exact one (B = Q^T A with
  orthonormal Q);
* isometry of Q U~ and V~ (Sec. II.B);
* literal Alg. RSVD step 2, Y = (A A^T)^q A Omega formed without intermediate
  orthonormalisation, spans the same space as the re-orthonormalised power
  iteration (checked where Y is well conditioned);
* the Halko-Martinsson-Tropp expectation bound for the power scheme (HMT 2011,
  Cor. 10.10) holds on average over seeds, and q = 2 beats q = 0.
"""
import math

import numpy as np
import pytest

from oracle import philox
from oracle import rsvd as orsvd
from oracle.rsvd import canonical_signs, qr_pos, rsvd, rsvd_basis, tsvd
from paper_1710_01463_gb300 import inputs


def test_tsvd_recovers_prescribed_spectrum():
    A = inputs.dense_case()
    s_true = inputs.exp_spectrum(256)
    U, s, Vt = tsvd(A, 32)
    np.testing.assert_allclose(s, s_true[:32], rtol=1e-13)
    np.testing.assert_allclose(U.T @ U, np.eye(32), atol=1e-13)
    np.testing.assert_allclose(Vt @ Vt.T, np.eye(32), atol=1e-13)


def test_eckart_young_frobenius_and_spectral():
    A = inputs.dense_case()
    s_true = inputs.exp_spectrum(256)
    k = 32
    U, s, Vt = tsvd(A, k)
    R = A - (U * s) @ Vt
    assert np.linalg.norm(R, "fro") == pytest.approx(math.sqrt(np.sum(s_true[k:] ** 2)), rel=1e-11)
    assert np.linalg.norm(R, 2) == pytest.approx(s_true[k], rel=1e-11)


@pytest.mark.parametrize("seed", range(5))
def test_two_by_two_closed_form(seed):
    A = np.random.default_rng(seed).standard_normal((2, 2))
    # eigenvalues of A^T A from trace and determinant
    tr = float(np.sum(A * A))
    det = float(np.linalg.det(A)) ** 2
    disc = math.sqrt(max(tr * tr / 4 - det, 0.0))
    s1 = math.sqrt(tr / 2 + disc)
    s2 = math.sqrt(max(tr / 2 - disc, 0.0))
    _, s, _ = tsvd(A, 2)
    np.testing.assert_allclose(s, [s1, s2], rtol=1e-12, atol=1e-15)


def test_three_by_three_brute_force():
    A = np.random.default_rng(9).standard_normal((3, 3))
    # singular values = square roots of the roots of det(A^T A - x I) (cubic)
    M = A.T @ A
    c2 = -np.trace(M)
    c1 = 0.5 * (np.trace(M) ** 2 - np.trace(M @ M))
    c0 = -np.linalg.det(M)
    roots = np.sort(np.roots([1.0, c2, c1, c0]).real)[::-1]
    _, s, _ = tsvd(A, 3)
    np.testing.assert_allclose(s, np.sqrt(roots), rtol=1e-10)


def test_canonical_sign_rule():
    A = inputs.random_dense(20, 12, 3)
    U, s, Vt = tsvd(A, 5)
    for i in range(5):
        j = int(np.argmax(np.abs(U[:, i])))
        assert U[j, i] > 0
    np.testing.assert_allclose((U * s) @ Vt, (lambda u, s_, v: (u * s_) @ v)(*tsvd(A, 5)), atol=1e-14)


def test_qr_pos_unique_factor():
    Y = inputs.random_dense(30, 7, 4)
    Q = qr_pos(Y)
    R = Q.T @ Y
    np.testing.assert_allclose(Q.T @ Q, np.eye(7), atol=1e-14)
    np.testing.assert_allclose(np.tril(R, -1), 0, atol=1e-13)
    assert np.all(np.diag(R) > 0)


@pytest.mark.parametrize("shape,r", [((60, 40), 10), ((40, 60), 10), ((50, 50), 18)])
def test_rsvd_exact_when_rank_fits(shape, r):
    m, n = shape
    A = inputs.spectral_matrix(m, n, np.linspace(3.0, 0.5, r), 77)
    U, s, Vt = rsvd(A, k=8, p=12, q=1, seed=11)   # l = 20 >= r
    Ut, st, Vtt = tsvd(A, 8)
    np.testing.assert_allclose(s, st, rtol=1e-12)
    np.testing.assert_allclose(U, Ut, atol=1e-10)
    np.testing.assert_allclose(Vt, Vtt, atol=1e-10)


def test_rsvd_interlacing_and_isometry():
    A = inputs.dense_case()
    U, s, Vt = rsvd(A, 32, 8, 2, seed=201)
    s_true = inputs.exp_spectrum(256)[:32]
    assert np.all(s <= s_true * (1 + 1e-13))
    np.testing.assert_allclose(U.T @ U, np.eye(32), atol=1e-13)
    np.testing.assert_allclose(Vt @ Vt.T, np.eye(32), atol=1e-13)
    # cfg (sigma_40 / sigma_32)^(4q) = e^-4: leading values accurate, trailing ones measurably below
    assert abs(s[0] - s_true[0]) / s_true[0] < 1e-9
    assert (s_true[31] - s[31]) / s_true[31] > 1e-4


def test_literal_power_form_spans_same_space():
    # Y = (A A^T)^q A Omega without intermediate QRs is fine when Y is well conditioned
    s_true = np.linspace(1.0, 0.3, 40)
    A = inputs.spectral_matrix(80, 60, s_true, 31)
    l, q = 12, 2
    omega = philox.gaussian_test_matrix(60, l, seed=3)
    Y = A @ omega
    for _ in range(q):
        Y = A @ (A.T @ Y)
    Qlit, _ = np.linalg.qr(Y)
    Q = rsvd_basis(A, l, q, seed=3)
    # same range: projectors agree
    np.testing.assert_allclose(Q @ Q.T, Qlit @ Qlit.T, atol=1e-11)


def test_wrong_power_operand_would_be_detected():
    # A @ Q in place of A^T @ Q gives a different (worse) subspace for non-normal A
    s_true = inputs.power_spectrum(60, 0.7)
    A = inputs.spectral_matrix(60, 60, s_true, 32)
    l, q = 10, 2
    omega = philox.gaussian_test_matrix(60, l, seed=4)
    Q = rsvd_basis(A, l, q, seed=4)
    Qw = qr_pos(A @ omega)
    for _ in range(q):
        Qw = qr_pos(A @ Qw)
        Qw = qr_pos(A @ Qw)
    e_right = np.linalg.norm(A - Q @ (Q.T @ A), 2)
    e_wrong = np.linalg.norm(A - Qw @ (Qw.T @ A), 2)
    assert e_right < 0.9 * e_wrong


def hmt_power_bound(s, k, p, q):
    """HMT 2011, Cor. 10.10: bound on E || (I - P_Y) A || for Y = (A A^T)^q A Omega."""
    t = 2 * q + 1
    tail = s[k:]
    val = (1 + math.sqrt(k / (p - 1))) * tail[0] ** t + (math.e * math.sqrt(k + p) / p) * math.sqrt(np.sum(tail ** (2 * t)))
    return val ** (1.0 / t)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_hmt_expectation_bound(q):
    s_true = inputs.power_spectrum(100, 0.5)       # slow decay
    A = inputs.spectral_matrix(100, 100, s_true, 55)
    k, p = 10, 5
    errs = []
    for seed in range(100):
        Q = rsvd_basis(A, k + p, q, seed=seed)
        errs.append(np.linalg.norm(A - Q @ (Q.T @ A), 2))
    assert np.mean(errs) <= hmt_power_bound(s_true, k, p, q)
    assert np.mean(errs) >= s_true[k + p] * (1 - 1e-12)   # can never beat sigma_{l+1}


def test_power_iterations_improve_accuracy():
    s_true = inputs.power_spectrum(200, 0.5)
    A = inputs.spectral_matrix(200, 200, s_true, 56)
    err = {}
    for q in (0, 2):
        U, s, Vt = rsvd(A, 20, 8, q, seed=7)
        err[q] = np.linalg.norm(A - (U * s) @ Vt, 2)
    assert err[2] < 0.8 * err[0]
    assert err[2] >= s_true[20] * (1 - 1e-12)


# ---------------------------------------------------------------- fixed-error RSVD
def minimal_rank(s_full, eps):
    """Smallest k >= 1 with sqrt(sum_{i>k} s_i^2) <= eps ||s|| (Eckart-Young)."""
    tot = np.sum(s_full ** 2)
    for k in range(1, len(s_full) + 1):
        if np.sum(s_full[k:] ** 2) <= eps * eps * tot:
            return k
    return len(s_full)


@pytest.mark.parametrize("eps", [1e-1, 1e-3, 3e-6, 1e-9])
def test_fixed_error_rank_matches_eckart_young_when_exact(eps):
    # rank-40 A: once l >= 40 the sample spans the range, s(B) = s(A), and the chosen rank
    # is the TSVD's minimal rank (eps kept away from the boundaries of the exp spectrum)
    rng = np.random.default_rng(21)
    s = np.exp(-np.arange(1, 41) / 3.0)
    U = np.linalg.qr(rng.standard_normal((120, 40)))[0]
    V = np.linalg.qr(rng.standard_normal((90, 40)))[0]
    A = (U * s) @ V.T
    Ur, sr, Vtr, err = orsvd.rsvd_fixed_error(A, eps, 8, 60, 40, 1, 3)
    k = minimal_rank(s, eps)
    assert len(sr) == k
    np.testing.assert_allclose(sr, s[:k], rtol=1e-10)
    assert err <= eps


@pytest.mark.parametrize("k0,kmax,eps", [(4, 200, 1e-6), (16, 200, 1e-3), (4, 12, 1e-8), (64, 64, 1e-2)])
def test_fixed_error_reports_its_true_error_and_is_minimal(k0, kmax, eps):
    # the reported error is ||A - U S V^T|| / ||A|| computed directly (pins the
    # Pythagoras identity: a dropped residual term or an off-by-one in the tail sum fails),
    # and rank k - 1 of the same factorization misses eps
    A = inputs.spectral_matrix(200, 150, inputs.exp_spectrum(150, 6.0), 8)
    U, s, Vt, err = orsvd.rsvd_fixed_error(A, eps, k0, kmax, 8, 1, 5)
    fro = np.linalg.norm(A)
    direct = np.linalg.norm(A - (U * s) @ Vt) / fro
    assert err == pytest.approx(direct, rel=1e-6, abs=1e-15)
    k = len(s)
    if err <= eps:
        assert k == 1 or np.linalg.norm(A - (U[:, :k - 1] * s[:k - 1]) @ Vt[:k - 1]) / fro > eps
    else:
        assert k == min(kmax, 150)  # the cap was reached


def test_fixed_error_grows_from_a_small_trial_rank():
    A = inputs.spectral_matrix(160, 160, inputs.harmonic_spectrum(160), 9)
    U, s, Vt, err = orsvd.rsvd_fixed_error(A, 0.05, 2, 160, 8, 2, 1)
    assert err <= 0.05 and len(s) > 2
    # the same result as one fixed-rank RSVD at the final trial rank (nested Omega: the
    # trials differ only in their width)
    kt = 2
    while kt < len(s):
        kt *= 2
    U2, s2, Vt2 = orsvd.rsvd(A, kt, 8, 2, 1)
    np.testing.assert_allclose(s, s2[:len(s)], rtol=1e-12)


def test_fixed_error_of_zero_and_exact_rank():
    U, s, Vt, err = orsvd.rsvd_fixed_error(np.zeros((30, 20)), 1e-6, 4, 20, 4, 1, 0)
    assert len(s) == 1 and s[0] == 0.0 and err == 0.0
    A = np.outer(np.arange(1.0, 31.0), np.arange(1.0, 21.0))
    U, s, Vt, err = orsvd.rsvd_fixed_error(A, 1e-12, 4, 20, 4, 1, 0)
    assert len(s) == 1 and err <= 1e-12


# ---------------------------------------------------------------- complex A (NEXT row: oracle only)
def haar_unitary(n, rng):
    z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


def test_complex_rsvd_of_real_data_is_the_real_algorithm():
    A = inputs.spectral_matrix(120, 90, inputs.exp_spectrum(90, 8.0), 3)
    Uc, sc, Vhc = orsvd.rsvd_complex(A.astype(np.complex128), 20, 8, 2, 11, 2)
    Ur, sr, Vtr = orsvd.rsvd(A, 20, 8, 2, 11, 2)
    np.testing.assert_allclose(sc, sr, rtol=1e-12)
    np.testing.assert_allclose(Uc, Ur, atol=1e-10)
    np.testing.assert_allclose(Vhc, Vtr, atol=1e-10)


def test_complex_rsvd_recovers_a_complex_spectrum_exactly():
    # A = U diag(s) V^H of rank 30 with Haar unitary factors: with l >= 30 the sample spans the
    # range and the singular values come back exactly; a transpose in place of a conjugate
    # transpose anywhere in the power iteration or the projection breaks this
    rng = np.random.default_rng(8)
    s = np.exp(-np.arange(1, 31) / 4.0)
    U = haar_unitary(80, rng)[:, :30]
    V = haar_unitary(70, rng)[:, :30]
    A = (U * s) @ V.conj().T
    Ur, sr, Vhr = orsvd.rsvd_complex(A, 30, 10, 2, 5, 0)
    np.testing.assert_allclose(sr, s, rtol=1e-11)
    np.testing.assert_allclose(Ur.conj().T @ Ur, np.eye(30), atol=1e-12)
    np.testing.assert_allclose(Vhr @ Vhr.conj().T, np.eye(30), atol=1e-12)
    np.testing.assert_allclose((Ur * sr) @ Vhr, A, atol=1e-12)
    # the phase rule: the largest-modulus entry of every u_i is real and positive
    idx = np.argmax(np.abs(Ur), axis=0)
    top = Ur[idx, np.arange(30)]
    assert np.all(top.real > 0) and np.all(np.abs(top.imag) < 1e-14)
    # and the factors agree with the complex TSVD
    Ut, st, Vht = orsvd.tsvd_complex(A, 30)
    np.testing.assert_allclose(Ur, Ut, atol=1e-9)


def test_complex_rsvd_is_covariant_under_a_global_phase():
    # e^{i phi} A has the same singular values; the phase rule moves the phase into V^H
    rng = np.random.default_rng(9)
    A = (rng.standard_normal((60, 40)) + 1j * rng.standard_normal((60, 40))) @ np.diag(np.exp(-np.arange(40) / 5.0))
    U1, s1, V1 = orsvd.rsvd_complex(A, 10, 8, 2, 3)
    U2, s2, V2 = orsvd.rsvd_complex(np.exp(0.7j) * A, 10, 8, 2, 3)
    np.testing.assert_allclose(s2, s1, rtol=1e-12)
    np.testing.assert_allclose(U2, U1, atol=1e-9)
    np.testing.assert_allclose(V2, np.exp(0.7j) * V1, atol=1e-9)


def test_complex_power_iteration_is_the_literal_power():
    # full rank, slow decay and l < rank, so the power iteration decides the result: the
    # literal Y = (A A^H)^q A Omega spans the same space, hence the same B singular values (a
    # transpose without conjugation inside the iteration changes them)
    rng = np.random.default_rng(10)
    m, n, k, p, q = 60, 50, 8, 4, 2
    s = 1.0 / np.arange(1, n + 1)
    A = (haar_unitary(m, rng)[:, :n] * s) @ haar_unitary(n, rng).conj().T
    _, s_r, _ = orsvd.rsvd_complex(A, k, p, q, 21, 1)
    omega = philox.gaussian_test_matrix(n, k + p, 21, 1)
    Y = A @ omega
    for _ in range(q):
        Y = A @ (A.conj().T @ Y)
    Qlit, _ = np.linalg.qr(Y)
    s_lit = np.linalg.svd(Qlit.conj().T @ A, compute_uv=False)[:k]
    np.testing.assert_allclose(s_r, s_lit, rtol=1e-9)
    assert np.all(s_r <= s[:k] * (1 + 1e-12))  # interlacing: the sampled values never exceed the true ones


def test_complex_rsvd_equals_real_algorithm_on_the_real_embedding():
    # The reading the GPU path takes for complex A: Alg. RSVD of the real embedding
    # R(A) = [Re A, -Im A; Im A, Re A] with the test matrix diag(Omega, Omega) and
    # rank 2k, oversampling 2p has the complex algorithm's singular values, each twice
    # (R(A^H) = R(A)^T and every sampled subspace is a realification)
    from oracle.philox import gaussian_test_matrix
    m, n, k, p, q = 96, 80, 12, 6, 2
    A = inputs.complex_spectral_matrix(m, n, inputs.exp_spectrum(80, 10.0), 40 + m)
    R = np.block([[A.real, -A.imag], [A.imag, A.real]])
    l = min(k + p, m, n)
    om = gaussian_test_matrix(n, l, 201, 3)
    omr = np.zeros((2 * n, 2 * l))
    omr[:n, :l] = om
    omr[n:, l:] = om
    _, sr, _ = orsvd.rsvd(R, 2 * k, 2 * p, q, 201, 3, omega=omr)
    _, so, _ = orsvd.rsvd_complex(A, k, p, q, 201, 3)
    np.testing.assert_allclose(sr[0::2], so, rtol=1e-12)
    np.testing.assert_allclose(sr[1::2], so, rtol=1e-12)
    # a plain (non-block-diagonal) real test matrix of the same width samples other spaces
    _, sx, _ = orsvd.rsvd(R, 2 * k, 2 * p, q, 201, 3)
    assert np.max(np.abs(sx[0::2] - so) / so) > 1e-12
