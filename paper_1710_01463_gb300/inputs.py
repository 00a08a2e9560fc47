"""Seeded synthetic inputs shaped like the paper's compression problems.

This module holds none of the method's arithmetic: it only builds test data
(matrices with a prescribed spectrum, sector shapes, loss weights, product
states).  Both the CUDA path's tests/benchmarks and the FP64 oracle take their
inputs from here, so both see identical bytes.

Recipe (all FP64 on the host, numpy PCG64 streams):

* ``spectral_matrix``: A = U diag(s) V^T with U, V the Q factors (R_ii > 0) of
  the QR factorization of seeded N(0,1) matrices - dense, Haar-like factors.
* Dense FP64 case: 256 x 256, s_i = exp(-i/16), i = 1..256 (the paper indexes
  singular values from 1, Sec. II.A).
* TTN-shaped case: chi^2 x chi^2 = 4096 x 4096 at chi = 64 (Sec. III.A, TTN
  double-tensor update), power law s_i = i^-1.5 (slower than the decays
  gamma = 2..11 the paper fits, Sec. IV).
* Sector case: N = 32 blocks, m_b, n_b uniform in 64..2048, s_i = f_b i^-1.2
  with f_b log-uniform in [1e-3, 1] (Sec. III.A block-diagonal structure).
* Gradient case: 1024 x 1024, s_i = 1 / (1 + 0.05 i); weights w ~ U(0, 1),
  W ~ N(0, 1) of shape m x 8.
* TEBD: a random product state (Sec. III.C: "product state with randomized
  tensors of bond dimension one").
* Complex case: A = U diag(s) V^H with U, V the Q factors (R_ii > 0) of seeded
  complex Gaussian matrices (the paper runs in complex double, Sec. IV).
"""
import numpy as np

_ORTHO_CACHE = {}


def haar_like_orthogonal(n, seed):
    """Q factor (R_ii > 0) of the QR factorization of a seeded N(0,1) n x n matrix."""
    key = (n, seed)
    if key not in _ORTHO_CACHE:
        rng = np.random.default_rng(seed)
        G = rng.standard_normal((n, n))
        Q, R = np.linalg.qr(G)
        Q = Q * np.where(np.diag(R) < 0, -1.0, 1.0)[None, :]
        _ORTHO_CACHE[key] = Q
    return _ORTHO_CACHE[key]


def spectral_matrix(m, n, s, seed):
    """A = U[:, :r] diag(s) V[:, :r]^T, r = len(s) <= min(m, n), FP64."""
    s = np.asarray(s, dtype=np.float64)
    r = s.size
    U = haar_like_orthogonal(m, 2 * seed)[:, :r]
    V = haar_like_orthogonal(n, 2 * seed + 1)[:, :r]
    return (U * s[None, :]) @ V.T


def haar_like_unitary(n, seed):
    """Q factor (R_ii > 0) of the QR factorization of a seeded complex N(0,1) n x n matrix."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    d = np.diag(R)
    return Q * np.where(np.abs(d) > 0, d / np.where(np.abs(d) > 0, np.abs(d), 1.0), 1.0)[None, :]


def complex_spectral_matrix(m, n, s, seed):
    """Complex A = U[:, :r] diag(s) V[:, :r]^H with seeded Haar-like unitary factors."""
    s = np.asarray(s, dtype=np.float64)
    r = s.size
    U = haar_like_unitary(m, 2 * seed)[:, :r]
    V = haar_like_unitary(n, 2 * seed + 1)[:, :r]
    return (U * s[None, :]) @ V.conj().T


def permuted_spectral_matrix(m, n, s, base_seed, j):
    """Member j of a batch: the factors of ``base_seed`` with seeded row
    permutations and sign flips (still orthogonal, distinct per j)."""
    s = np.asarray(s, dtype=np.float64)
    r = s.size
    rng = np.random.default_rng(1_000_003 * base_seed + j)
    U = haar_like_orthogonal(m, 2 * base_seed)[:, :r]
    V = haar_like_orthogonal(n, 2 * base_seed + 1)[:, :r]
    U = U[rng.permutation(m)] * rng.choice([-1.0, 1.0], size=m)[:, None]
    V = V[rng.permutation(n)] * rng.choice([-1.0, 1.0], size=n)[:, None]
    return (U * s[None, :]) @ V.T


def exp_spectrum(r, scale=16.0):
    """s_i = exp(-i / scale), i = 1..r."""
    return np.exp(-np.arange(1, r + 1) / scale)


def power_spectrum(r, gamma, factor=1.0):
    """s_i = factor * i^-gamma, i = 1..r."""
    return factor * np.arange(1, r + 1, dtype=np.float64) ** (-gamma)


def harmonic_spectrum(r, a=0.05):
    """s_i = 1 / (1 + a i), i = 1..r."""
    return 1.0 / (1.0 + a * np.arange(1, r + 1))


def dense_case(m=256, n=256, seed=101):
    """Single dense FP64 matrix with s_i = exp(-i/16)."""
    return spectral_matrix(m, n, exp_spectrum(min(m, n)), seed)


def ttn_case(j, n=4096, base_seed=103):
    """Member j of the 4096 x 4096 power-law (i^-1.5) batch."""
    return permuted_spectral_matrix(n, n, power_spectrum(n, 1.5), base_seed, j)


def sector_shapes(N=32, lo=64, hi=2048, seed=104):
    """Block shapes m_b x n_b and per-sector factors f_b (log-uniform in [1e-3, 1])."""
    rng = np.random.default_rng(seed)
    mb = rng.integers(lo, hi + 1, size=N)
    nb = rng.integers(lo, hi + 1, size=N)
    f = 10.0 ** rng.uniform(-3.0, 0.0, size=N)
    return [(int(a), int(b)) for a, b in zip(mb, nb)], f


def sector_blocks(N=32, lo=64, hi=2048, seed=104):
    """Blocks of a block-diagonal bond matrix, block b with s_i = f_b i^-1.2."""
    shapes, f = sector_shapes(N, lo, hi, seed)
    out = []
    for b, ((m, n), fb) in enumerate(zip(shapes, f)):
        out.append(spectral_matrix(m, n, power_spectrum(min(m, n), 1.2, fb), 7919 * seed + b))
    return out


def grad_case(j, n=1024, k=128, r=8, base_seed=105):
    """Member j of the gradient batch: (A, w, W)."""
    A = permuted_spectral_matrix(n, n, harmonic_spectrum(n), base_seed, j)
    rng = np.random.default_rng(104_729 * base_seed + j)
    w = rng.uniform(0.0, 1.0, size=k)
    W = rng.standard_normal((n, r))
    return A, w, W


def product_state_vectors(L, d=2, seed=102):
    """L random local vectors (rows) of a product state, N(0,1) entries."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((L, d))


def random_dense(m, n, seed):
    """Seeded N(0,1) m x n matrix."""
    return np.random.default_rng(seed).standard_normal((m, n))
