"""Alg. TSVD (Sec. II.A) on the library's own engine (RSVD_FLAG_FULL_SVD): the full
one-sided Jacobi SVD of A, then truncation - the comparator of the paper's speedup
tau = T_TSVD / T_RSVD (Sec. IV).

* Dense matrices (square, tall, wide - the wide one through the orthonormalised A^T):
  the k leading singular values equal the oracle's Alg. TSVD within the FP64 bar
  (1e-10 sigma_i + 1e-14 sigma_1), the vectors within 1e-8 where the values are
  separated, and the result is exact (no sampling): the reconstruction error is the
  Eckart-Young optimum.
* TEBD with TSVD compressions matches the oracle's TSVD-TEBD step by step, and its ground
  energy equals the RSVD-TEBD energy within 1e-9 relative (the paper reports both giving
  the same energies within computational precision, Sec. IV).
"""
import numpy as np
import pytest

from gpu_util import align_columns, need_gpu, sigma_tol, torch
from oracle import rsvd as orsvd
from oracle import tebd as otebd
from paper_1710_01463_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    need_gpu()
    from paper_1710_01463_gb300 import _lib, api, tebd
    return _lib, api, tebd


@pytest.mark.parametrize("m,n,k", [(256, 256, 32), (200, 120, 20), (64, 256, 16), (40, 30, 7)])
def test_full_svd_matches_oracle_tsvd(mods, m, n, k):
    _lib, api, _ = mods
    A = inputs.spectral_matrix(m, n, inputs.exp_spectrum(min(m, n), 12.0), 31 + m)
    U, S, Vt, info = api.rsvd_truncate(torch.from_numpy(A).cuda(), k, 8, 2, 0, flags=_lib.RSVD_FLAG_FULL_SVD)
    torch.cuda.synchronize()
    st = api.info_dicts(info)[0]
    assert st["status"] == 0 and st["path"] & 1
    Uo, So, Vto = orsvd.tsvd(A, k)
    s = S.cpu().numpy()
    assert np.all(np.abs(s - So) <= sigma_tol(So))
    u, vt = U.cpu().numpy(), Vt.cpu().numpy()
    np.testing.assert_allclose(align_columns(u, Uo), Uo, atol=1e-8)
    np.testing.assert_allclose(align_columns(vt.T, Vto.T), Vto.T, atol=1e-8)
    s_full = np.linalg.svd(A, compute_uv=False)
    err = np.linalg.norm(A - (u * s) @ vt)
    assert err == pytest.approx(np.sqrt(np.sum(s_full[k:] ** 2)), rel=1e-8)


def test_tebd_tsvd_steps_match_oracle(mods):
    _, _, tebd = mods
    L, chi, dt = 10, 8, 0.05
    ch = tebd.TebdChain(L, chi, h=1.0, p=10, q=2, seed=5, tsvd=True)
    vec = inputs.product_state_vectors(L, 2, 102)
    ch.set_product_state(vec)
    ch.set_dt(dt)
    D = otebd.bond_dims(L, 2, chi)
    B, lam = otebd.product_state(vec, D)
    comp = otebd.make_compressor("tsvd")
    for s in range(4):
        ch.step(s)
        otebd.trotter_step(B, lam, L, 1.0, dt, comp, s)
    torch.cuda.synchronize()
    lam_g = ch.schmidt_values()
    for j in range(1, L):
        np.testing.assert_allclose(lam_g[j], lam[j], rtol=0, atol=1e-10 * np.max(lam[j]) + 1e-14)
    assert otebd.mps_energy(ch.tensors(), L, 1.0) == pytest.approx(otebd.mps_energy(B, L, 1.0), rel=1e-10)


def test_tebd_tsvd_and_rsvd_reach_the_same_energy(mods):
    _, _, tebd = mods
    L, chi = 16, 32
    es = []
    for tsvd in (False, True):
        ch = tebd.TebdChain(L, chi, h=1.0, p=10, q=2, seed=5, tsvd=tsvd)
        ch.set_product_state(inputs.product_state_vectors(L, 2, 102))
        ch.evolve(((0.1, 150), (0.02, 100)))
        torch.cuda.synchronize()
        assert int((ch.info[..., 0] != 0).sum()) == 0
        es.append(otebd.mps_energy(ch.tensors(), L, 1.0))
    assert es[0] == pytest.approx(es[1], rel=1e-9)
