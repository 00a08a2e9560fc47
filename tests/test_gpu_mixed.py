"""Mixed-precision RSVD (products with A on tensor cores: BF16 or TF32, FP32
accumulation; Gram / Cholesky / SVD of B in FP64) against the FP64 oracle.

The oracle factorises the same matrix as the GPU sees it (A rounded to bfloat16
for the BF16 form) with its own FP64 test matrix.  The bounds are the stated
errors of the reduced-precision forms (the thin operand is split into
high and low parts, so only A's own rounding and FP32 accumulation remain):
singular values within 1e-4 of sigma_1 (BF16 storage of A is exact input) and
2e-3 relative for TF32 (A truncated to 10 mantissa bits); U and V^T orthonormal
to 1e-5.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, torch
from oracle import rsvd as orsvd
from paper_1710_01463_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    need_gpu()
    from paper_1710_01463_gb300 import api as a
    return a


@pytest.mark.parametrize("m,n,k,p", [(1024, 768, 32, 16), (777, 1504, 20, 12), (4096, 4096, 64, 16)])
@pytest.mark.parametrize("kind", ["bf16", "tf32"])
def test_mixed_precision_rsvd(api, m, n, k, p, kind):
    A64 = inputs.spectral_matrix(m, n, inputs.power_spectrum(min(m, n), 1.5), 61 + m)
    if kind == "bf16":
        At = torch.from_numpy(A64).to(torch.bfloat16).cuda()
        U, S, Vt, info = api.rsvd_truncate(At, k, p, 2, 5, 0)
        Aref = At.double().cpu().numpy()
    else:
        At = torch.from_numpy(A64).float().cuda()
        U, S, Vt, info = api.rsvd_truncate(At, k, p, 2, 5, 0, tf32=True)
        Aref = At.double().cpu().numpy()
    torch.cuda.synchronize()
    assert api.info_dicts(info)[0]["status"] == 0
    _, So, _ = orsvd.rsvd(Aref, k, p, 2, 5, 0)
    s = S.cpu().numpy()
    if kind == "bf16":
        assert np.max(np.abs(s - So)) <= 1e-4 * So[0], np.max(np.abs(s - So)) / So[0]
    else:
        assert np.max(np.abs(s - So) / So) <= 2e-3, np.max(np.abs(s - So) / So)
    u, vt = U.double().cpu().numpy(), Vt.double().cpu().numpy()
    np.testing.assert_allclose(u.T @ u, np.eye(k), atol=1e-5)
    np.testing.assert_allclose(vt @ vt.T, np.eye(k), atol=1e-5)


def test_mixed_precision_batched(api):
    As = [torch.from_numpy(inputs.ttn_case(j, n=1024)).to(torch.bfloat16).cuda() for j in range(3)]
    U, S, Vt, k_out, info = api.rsvd_truncate_batched(As, [64] * 3, p=16, q=2, seed=103, stream=0)
    torch.cuda.synchronize()
    for j, A in enumerate(As):
        _, So, _ = orsvd.rsvd(A.double().cpu().numpy(), 64, 16, 2, 103, j)
        assert np.max(np.abs(S[j].cpu().numpy() - So)) <= 1e-4 * So[0]
    assert all(d["status"] == 0 for d in api.info_dicts(info))


def test_mixed_precision_rejects_unaligned_rows(api):
    A = torch.zeros((300, 301), dtype=torch.bfloat16, device="cuda")  # 602-byte rows: not a TMA stride
    with pytest.raises(Exception):
        api.rsvd_truncate(A, 8, 8, 1, 0, 0)


def test_mixed_precision_large_batch_chunks_concurrent(api):
    # BF16 batches are processed in chunks of 16 matrices; above that the chunks run
    # concurrently on the library's chunk streams: bit-identical to RSVD_FLAG_SERIAL (every
    # chunk on the caller's stream), and sampled members within the BF16 bound of the oracle
    shapes = [(320 + 16 * (b % 5), 256 + 8 * (b % 7)) for b in range(37)]
    A64 = [inputs.spectral_matrix(m, n, inputs.power_spectrum(min(m, n), 1.5), 900 + b)
           for b, (m, n) in enumerate(shapes)]
    As = [torch.from_numpy(a).to(torch.bfloat16).cuda() for a in A64]
    ks = [24] * len(As)
    _, S, Vt, _, info = api.rsvd_truncate_batched(As, ks, p=16, q=2, seed=21, stream=0)
    S = [s.clone() for s in S]
    Vt = [v.clone() for v in Vt]
    from paper_1710_01463_gb300 import _lib as lib_mod
    _, S2, Vt2, _, info2 = api.rsvd_truncate_batched(As, ks, p=16, q=2, seed=21, stream=0,
                                                     flags=lib_mod.RSVD_FLAG_SERIAL)
    torch.cuda.synchronize()
    for b in range(len(As)):
        assert torch.equal(S[b], S2[b]) and torch.equal(Vt[b], Vt2[b])
    assert all(d["status"] == 0 for d in api.info_dicts(info))
    for b in (0, 15, 16, 36):
        Ab = As[b].double().cpu().numpy()
        _, So, _ = orsvd.rsvd(Ab, 24, 16, 2, 21, b)
        assert np.all(np.abs(S[b].cpu().numpy() - So) <= 1e-4 * So[0]), b
