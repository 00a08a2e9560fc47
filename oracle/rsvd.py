"""Oracle: Alg. TSVD and Alg. RSVD of Kohn et al. (Sec. II), plain FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Library primitives used as steps: ``numpy.linalg.svd`` (LAPACK gesdd) for
every "compute the SVD" step and ``numpy.linalg.qr`` (LAPACK Householder
geqrf/orgqr) for every "orthonormalise" step.  No blocking, fusion or
reordering beyond what the algorithms state.

Readings where the paper is silent (the CUDA path applies the same ones):

* QR sign: R_ii >= 0 (Q unique for full-rank input).
* Singular-vector sign: u_i is flipped (with v_i) so that its entry of
  largest magnitude is positive, the lowest row index winning ties.
* Power iteration: the paper's step 2 forms Y = (A A^T)^q A Omega "as a power
  iteration with subsequent QR factorizations" (Halko-Martinsson-Tropp 2011,
  Algorithm 4.4), i.e. 2q+1 orthonormalisations:
  Q0 = qr(A Omega); for j = 1..q: Z = qr(A^T Q), Q = qr(A Z).
* l = min(k + p, m, n): the sample can never have more columns than A has
  independent rows or columns.
"""
import numpy as np

from .philox import gaussian_test_matrix


def qr_pos(Y):
    """Thin QR with non-negative diagonal of R; returns Q (Alg. RSVD step 3)."""
    Q, R = np.linalg.qr(Y, mode="reduced")
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :]


def canonical_signs(U, s, Vt):
    """Flip (u_i, v_i) pairs so the largest-|.| entry of each u_i is positive."""
    U = U.copy()
    Vt = Vt.copy()
    for i in range(U.shape[1]):
        j = int(np.argmax(np.abs(U[:, i])))  # argmax returns the lowest index on ties
        if U[j, i] < 0:
            U[:, i] = -U[:, i]
            Vt[i, :] = -Vt[i, :]
    return U, s, Vt


def tsvd(A, k):
    """Alg. TSVD (Sec. II.A): full SVD of A, keep the k largest singular triplets.

    Returns (U_k, s_k, Vt_k): U_k is m-by-k, s_k descending, Vt_k is k-by-n.
    """
    U, s, Vt = np.linalg.svd(np.asarray(A, dtype=np.float64), full_matrices=False)
    return canonical_signs(U[:, :k], s[:k], Vt[:k, :])


def sample_width(m, n, k, p):
    """l = min(k + p, m, n)."""
    return min(k + p, m, n)


def rsvd_basis(A, l, q, seed, stream=0, omega=None):
    """Alg. RSVD steps 1-3: orthonormal basis Q (m-by-l) of the sampled range."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if omega is None:
        omega = gaussian_test_matrix(n, l, seed, stream)      # step 1
    Q = qr_pos(A @ omega)                                       # step 2, j = 0
    for _ in range(q):                                          # step 2, j = 1..q
        Z = qr_pos(A.T @ Q)
        Q = qr_pos(A @ Z)
    return Q                                                    # step 3


def rsvd(A, k, p, q, seed, stream=0, omega=None):
    """Alg. RSVD (Sec. II.B): approximate rank-k truncated SVD of A.

    Step 4 takes the rank-k TSVD of B = Q^T A (l-by-n); the left factor is
    lifted back as U = Q U~, the right factor is V~ itself.  Both are exact
    isometries (Sec. II.B).
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    l = sample_width(m, n, k, p)
    Q = rsvd_basis(A, l, q, seed, stream, omega)
    B = Q.T @ A                                                 # step 4
    Ub, s, Vt = np.linalg.svd(B, full_matrices=False)
    U = Q @ Ub[:, :k]
    return canonical_signs(U, s[:k], Vt[:k, :])


def truncation_error_frobenius(s_full, k):
    """Eckart-Young-Mirsky (Sec. II.A): minimal Frobenius error of a rank-k factorization."""
    s_full = np.asarray(s_full, dtype=np.float64)
    return float(np.sqrt(np.sum(s_full[k:] ** 2)))


def rsvd_fixed_error(A, eps, k0, k_max, p, q, seed, stream=0):
    """Fixed-error Alg. RSVD (the fixed-error form the paper proposes in Sec. V, after
    Halko-Martinsson-Tropp and Gu): the smallest rank k <= k_max whose factorization has
    ||A - U diag(s) V^T||_F <= eps ||A||_F.

    The error of the rank-k result Q B_k (B = Q^T A, B_k its rank-k TSVD) is known from
    the sample alone: Q Q^T is an orthogonal projector, so
        ||A - Q B_k||_F^2 = ||A - Q B||_F^2 + sum_{i > k} s_i(B)^2.
    Trial ranks k0, 2 k0, 4 k0, ... (capped at k_max and min(m, n)), each a full Alg.
    RSVD with l = min(k + p, m, n); the test matrix of a larger trial extends the
    previous one (its columns nest).  k >= 1.  Returns (U, s, Vt, err) with
    err = ||A - U diag(s) Vt||_F / ||A||_F (0 for A = 0); when no k <= k_max reaches
    eps, k is the last trial rank and err > eps."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    fro2 = float(np.sum(A * A))
    cap = min(k_max, m, n)
    kt = max(1, min(k0, cap))
    while True:
        l = sample_width(m, n, kt, p)
        Q = rsvd_basis(A, l, q, seed, stream)
        B = Q.T @ A
        Ub, s, Vt = np.linalg.svd(B, full_matrices=False)
        r2 = float(np.sum((A - Q @ B) ** 2))
        # err2[k] = r2 + sum_{i >= k} s_i^2 (0-based i), k = 0 .. len(s); summed smallest first
        err2 = np.append(r2 + np.cumsum((s ** 2)[::-1])[::-1], r2)
        ok = [k for k in range(1, kt + 1) if err2[k] <= eps * eps * fro2]
        if ok or kt >= cap:
            k = ok[0] if ok else kt
            U, s_k, Vt_k = canonical_signs(Q @ Ub[:, :k], s[:k], Vt[:k, :])
            err = float(np.sqrt(err2[k] / fro2)) if fro2 > 0 else 0.0
            return U, s_k, Vt_k, err
        kt = min(2 * kt, cap)


# ---------------------------------------------------------------- complex A
# Sec. II.A states the problem for "real- or complex-valued" A.  Readings for the
# complex form (the paper is silent): the test matrix Omega is the same real Philox
# matrix (so a real A in complex storage gives the real algorithm exactly); every
# transpose is the conjugate transpose; QR takes R_ii real and positive; the sign
# rule becomes a phase rule - the entry of largest modulus of u_i (lowest index on
# ties) is made real and positive, v_i taking the conjugate phase so that
# u_i s_i v_i^H is unchanged.

def qr_pos_complex(Y):
    """Thin QR with real non-negative diagonal of R (Alg. RSVD step 3, complex)."""
    Q, R = np.linalg.qr(Y, mode="reduced")
    d = np.diag(R)
    ph = np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1.0), 1.0)
    return Q * ph[None, :]


def canonical_phases(U, s, Vh):
    """Make the largest-modulus entry of each u_i real positive (v_i^H follows)."""
    U = U.copy()
    Vh = Vh.copy()
    for i in range(U.shape[1]):
        j = int(np.argmax(np.abs(U[:, i])))
        a = U[j, i]
        if abs(a) > 0:
            ph = a / abs(a)
            U[:, i] = U[:, i] / ph
            Vh[i, :] = Vh[i, :] * ph
    return U, s, Vh


def tsvd_complex(A, k):
    """Alg. TSVD for complex A: (U_k, s_k, V_k^H) with the phase rule."""
    U, s, Vh = np.linalg.svd(np.asarray(A, dtype=np.complex128), full_matrices=False)
    return canonical_phases(U[:, :k], s[:k], Vh[:k, :])


def rsvd_complex(A, k, p, q, seed, stream=0):
    """Alg. RSVD (Sec. II.B) for complex A: Q0 = qr(A Omega); q times Z = qr(A^H Q),
    Q = qr(A Z); B = Q^H A; rank-k TSVD of B lifted by Q.  Returns (U, s, V^H)."""
    A = np.asarray(A, dtype=np.complex128)
    m, n = A.shape
    l = sample_width(m, n, k, p)
    omega = gaussian_test_matrix(n, l, seed, stream)
    Q = qr_pos_complex(A @ omega)
    for _ in range(q):
        Z = qr_pos_complex(A.conj().T @ Q)
        Q = qr_pos_complex(A @ Z)
    B = Q.conj().T @ A
    Ub, s, Vh = np.linalg.svd(B, full_matrices=False)
    return canonical_phases(Q @ Ub[:, :k], s[:k], Vh[:k, :])

