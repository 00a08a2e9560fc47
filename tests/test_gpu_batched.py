"""GPU parity of rsvd_truncate_batched (uneven blocks, global top-chi, Sec. III.A)."""
import numpy as np
import pytest

from gpu_util import need_gpu, sigma_tol, torch
from oracle import rsvd as orsvd
from oracle.sectors import block_rsvd_global, global_select
from paper_1710_01463_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    need_gpu()
    from paper_1710_01463_gb300 import api as a
    return a


def small_sectors(N=7, seed=3):
    shapes, f = inputs.sector_shapes(N=N, lo=20, hi=160, seed=seed)
    return [inputs.spectral_matrix(m, n, inputs.power_spectrum(min(m, n), 1.2, fb), 100 + b)
            for b, ((m, n), fb) in enumerate(zip(shapes, f))]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_uneven_matches_per_matrix_oracle(api, dtype):
    blocks = small_sectors()
    ks = [min(12, *b.shape) for b in blocks]
    As = [torch.from_numpy(b).to(dtype).cuda() for b in blocks]
    U, S, Vt, k_out, info = api.rsvd_truncate_batched(As, ks, p=6, q=2, seed=9, stream=4)
    torch.cuda.synchronize()
    for b, (A, k) in enumerate(zip(blocks, ks)):
        Ao = As[b].double().cpu().numpy()
        _, So, _ = orsvd.rsvd(Ao, k, 6, 2, 9, 4 + b)
        s = S[b].cpu().numpy()
        if dtype == torch.float64:
            assert np.all(np.abs(s - So) <= sigma_tol(So))
        else:
            assert np.all(np.abs(s - So) <= 2e-5 * So[0])
    assert all(d["status"] == 0 for d in api.info_dicts(info))


def test_global_selection_matches_oracle(api):
    blocks = small_sectors(9, 4)
    chi = 40
    ks = [min(chi, *b.shape) for b in blocks]
    As = [torch.from_numpy(b).cuda() for b in blocks]
    U, S, Vt, k_out, info = api.rsvd_truncate_batched(As, ks, p=8, q=2, seed=5, stream=0, chi_global=chi)
    torch.cuda.synchronize()
    res, kept, ranks = block_rsvd_global(blocks, chi, p=8, q=2, seed=5, ranks=ks)
    assert k_out.cpu().tolist() == kept
    # selection over the GPU's own values reproduces its k_out exactly (integer work)
    assert global_select([s.cpu().numpy() for s in S], chi) == k_out.cpu().tolist()
    smax = max(float(r[1][0]) for r in res if r[1].size)
    for b in range(len(blocks)):
        if kept[b] == 0:
            continue
        ref = res[b][1]
        tol = 1e-10 * np.abs(ref) + 1e-14 * smax
        assert np.all(np.abs(S[b].cpu().numpy()[: kept[b]] - ref) <= tol)


def test_global_selection_ties(api):
    # identical blocks: equal values, ties go to the lower matrix index
    A = inputs.spectral_matrix(30, 30, np.linspace(1.0, 0.1, 30), 8)
    As = [torch.from_numpy(A).cuda() for _ in range(3)]
    U, S, Vt, k_out, info = api.rsvd_truncate_batched(As, [10, 10, 10], p=20, q=1, seed=1, chi_global=7)
    torch.cuda.synchronize()
    # p=20 covers the rank: every block returns the same values up to rounding
    got = k_out.cpu().tolist()
    assert sum(got) == 7
    assert got == global_select([s.cpu().numpy() for s in S], 7)
