"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def sigma_tol(ref):
    """Per-value tolerance on singular values: 1e-10 relative + 1e-14 of sigma_1.

    The relative part is the FP64 parity bar; the absolute floor is the
    rounding limit of any normwise backward-stable method (Weyl: a perturbation
    E moves every singular value by at most ||E||_2 ~ eps ||A||_2).
    """
    ref = np.asarray(ref)
    return 1e-10 * np.abs(ref) + 1e-14 * np.max(np.abs(ref))


def align_columns(X, Y):
    """Flip columns of X to best match Y (sign gauge)."""
    s = np.sign(np.sum(X * Y, axis=0))
    s[s == 0] = 1.0
    return X * s[None, :]
