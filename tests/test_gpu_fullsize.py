"""GPU parity at the full sizes of the batched-sector and gradient workloads.

* Sectors (Sec. III.A block-diagonal bond, global post-selection): the 32 blocks of
  the seeded sector workload (m_b, n_b uniform in 64..2048, s_i = f_b i^-1.2), FP32
  products, trial ranks k_b = min(chi, m_b, n_b), p = 16, q = 2, chi = 512.  The kept
  counts are the global top-chi selection over the GPU's own values (integer work,
  bit-exact), they add up to chi, and every kept value is within 2e-5 sigma_1 of the FP64
  oracle's Alg. RSVD of the same FP32-rounded block with the same Philox stream (FP32
  products: unit roundoff 6e-8 times the growth of a K <= 2048 sum).  These sizes take
  the paths small blocks never reach: wide B (n >= 3l), 2048-row CholeskyQR2, samples
  of up to 528 columns and the Jacobi SVD in global memory.
* Backward of the truncated factorization at the gradient workload's size: 1024 x 1024,
  k = 128, s_i = 1 / (1 + 0.05 i), whose retained and discarded values are only
  s_128^2 - s_129^2 = 2.4e-4 apart at the cut.  At the exact factors, with the loss's
  cotangents (sum w_i s_i + ||W^T U_k||^2), the library's Abar equals the adjoint of the
  full SVD: to 1e-8 (max-norm, relative) in FP64 and 1e-3 in FP32, and the
  conjugate-gradient solve of the discarded-space coupling reports convergence.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, torch
from oracle import grad as ograd
from oracle import rsvd as orsvd
from oracle.sectors import global_select
from paper_1710_01463_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    need_gpu()
    from paper_1710_01463_gb300 import api as a
    return a


def test_sectors_full_size_fp32_global_selection(api):
    blocks = [b.astype(np.float32) for b in inputs.sector_blocks(N=32, lo=64, hi=2048, seed=104)]
    chi, p, q, seed = 512, 16, 2, 103
    ks = [min(chi, *b.shape) for b in blocks]
    As = [torch.from_numpy(b).cuda() for b in blocks]
    U, S, Vt, k_out, info = api.rsvd_truncate_batched(As, ks, p=p, q=q, seed=seed, stream=0, chi_global=chi)
    torch.cuda.synchronize()
    assert all(d["status"] == 0 for d in api.info_dicts(info))
    got = k_out.cpu().tolist()
    Sg = [s.cpu().numpy() for s in S]
    assert global_select(Sg, chi) == got
    assert sum(got) == chi
    # the paths these sizes take: some wide B and some samples past 256 columns
    ls = [min(k + p, *b.shape) for k, b in zip(ks, blocks)]
    assert any(b.shape[1] >= 3 * l for b, l in zip(blocks, ls)) and max(ls) > 256
    ref = []
    for b, (blk, k) in enumerate(zip(blocks, ks)):
        _, So, _ = orsvd.rsvd(blk.astype(np.float64), k, p, q, seed, b)
        ref.append(So)
    smax = max(float(r[0]) for r in ref)
    for b in range(len(blocks)):
        kb = got[b]
        if kb == 0:
            continue
        err = np.max(np.abs(Sg[b][:kb] - ref[b][:kb]))
        assert err <= 2e-5 * smax, (b, err / smax)


def grad_problem(j):
    A, w, W = inputs.grad_case(j)
    k = 128
    return A, w, W, k


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_backward_full_size_at_exact_factors(api, dtype):
    cases = []
    for j in range(2):
        A, w, W, k = grad_problem(j)
        if dtype == "f32":
            A = A.astype(np.float32).astype(np.float64)
        Uf, sf, Vtf = np.linalg.svd(A, full_matrices=False)
        Ub, sb, _ = ograd.loss_cotangents(Uf[:, :k], w, W)
        ref = ograd.full_svd_adjoint(Uf, sf, Vtf, Ub, sb, np.zeros((A.shape[1], k)))
        assert sf[k - 1] ** 2 - sf[k] ** 2 < 3e-4  # the near-degenerate cut of this workload
        cases.append((A, Uf[:, :k], sf[:k], Vtf[:k], Ub, sb, ref))
    tdt = torch.float64 if dtype == "f64" else torch.float32
    f = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(tdt).cuda()
    d = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    Abar, info = api.rsvd_truncate_backward_batched(
        [f(c[0]) for c in cases], [f(c[1]) for c in cases], [d(c[2]) for c in cases], [f(c[3]) for c in cases],
        [f(c[4]) for c in cases], [d(c[5]) for c in cases], None,
        max_iter=400 if dtype == "f64" else 200, tol=1e-11 if dtype == "f64" else 1e-6)
    torch.cuda.synchronize()
    assert [s["status"] for s in api.info_dicts(info)] == [0, 0]
    bar = 1e-8 if dtype == "f64" else 1e-3
    for c, got in zip(cases, Abar):
        ref = c[6]
        err = np.max(np.abs(got.double().cpu().numpy() - ref)) / np.max(np.abs(ref))
        assert err <= bar, err
