"""GPU parity of rsvd_truncate_batched (uneven blocks, global top-chi, Sec. III.A)."""
import numpy as np
import pytest

from gpu_util import need_gpu, sigma_tol, torch
from oracle import rsvd as orsvd
from oracle.sectors import block_rsvd_adaptive, block_rsvd_global, global_select
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


@pytest.mark.parametrize("start,dtype", [("ones", torch.float64), ("even", torch.float64), ("ones", torch.float32)])
def test_adaptive_sector_ranks_match_oracle(api, start, dtype):
    # per-block trial ranks grown until no block is saturated.  FP64: the same rounds,
    # final ranks and kept counts as the oracle (integer work, bit-exact) and its values at
    # the FP64 bar.  FP32: values near the cut lie closer than FP32 rounding (3.7e-5
    # sigma_1 apart), so the unique parts are checked: the counts are the selection over
    # the GPU's own values, no block ends saturated below its cap, and every kept value is
    # within 2e-5 sigma_1 of the oracle's
    blocks = small_sectors(9, 4)
    chi = 40
    r0 = [1] * len(blocks) if start == "ones" else [max(1, chi // len(blocks))] * len(blocks)
    plan = api.AdaptiveSectorsPlan([b.shape for b in blocks], chi, r0, p=8, q=2, seed=5, dtype=dtype)
    U, S, Vt, k_out = plan.run([torch.from_numpy(b).to(dtype).cuda() for b in blocks])
    torch.cuda.synchronize()
    res, kept, ranks, rounds = block_rsvd_adaptive(blocks, chi, 8, 2, 5, r0)
    got_kept = k_out.cpu().tolist()
    smax = max(float(r[1][0]) for r in res if r[1].size)
    if dtype == torch.float64:
        assert got_kept == kept
        assert plan.ranks == ranks and plan.rounds == rounds
    else:
        assert global_select([s.cpu().numpy()[:r] for s, r in zip(S, plan.ranks)], chi) == got_kept
        for kb, r, blk in zip(got_kept, plan.ranks, blocks):
            assert kb < r or r == min(chi, *blk.shape)
    for b in range(len(blocks)):
        kb = min(kept[b], got_kept[b])
        ref = res[b][1][:kb]
        got = S[b].cpu().numpy()[:kb]
        tol = (1e-10 * np.abs(ref) + 1e-14 * smax) if dtype == torch.float64 else 2e-5 * smax
        assert np.all(np.abs(got - ref) <= tol)
    assert all(d["status"] == 0 for d in api.info_dicts(plan.info))


@pytest.mark.parametrize("start,dtype", [("ones", torch.float64), ("even", torch.float64), ("ones", torch.float32)])
def test_adaptive_device_rounds_match_host_rounds(api, start, dtype):
    # the rounds decided on the device (no host synchronisation) against the host-driven
    # rounds and the oracle: the same kept counts, final ranks and number of rounds
    # (integer work, bit-exact in FP64), and the values of the two GPU forms at the FP64 bar
    # (only the cluster sizes of a round, i.e. summation orders, may differ).  FP32: the
    # counts are the selection over the device form's own values.
    blocks = small_sectors(9, 4)
    chi = 40
    r0 = [1] * len(blocks) if start == "ones" else [max(1, chi // len(blocks))] * len(blocks)
    As = [torch.from_numpy(b).to(dtype).cuda() for b in blocks]
    host = api.AdaptiveSectorsPlan([b.shape for b in blocks], chi, r0, p=8, q=2, seed=5, dtype=dtype)
    host.run(As)
    dev = api.AdaptiveSectorsPlan([b.shape for b in blocks], chi, r0, p=8, q=2, seed=5, dtype=dtype,
                                  device_rounds=True)
    dev.run(As)
    torch.cuda.synchronize()
    got_kept = dev.k_out.cpu().tolist()
    got_ranks = dev.k_final.cpu().tolist()
    got_rounds = int(dev.rounds_dev.item())
    if dtype == torch.float64:
        _, kept, ranks, rounds = block_rsvd_adaptive(blocks, chi, 8, 2, 5, r0)
        assert got_kept == kept == host.k_out.cpu().tolist()
        assert got_ranks == ranks == host.ranks
        assert got_rounds == rounds == host.rounds
        for b in range(len(blocks)):
            kb = got_kept[b]
            s_h, s_d = host.S[b].cpu().numpy()[:kb], dev.S[b].cpu().numpy()[:kb]
            assert np.all(np.abs(s_h - s_d) <= 1e-12 * max(1.0, float(np.abs(s_h).max(initial=0.0))))
    else:
        assert global_select([s.cpu().numpy()[:r] for s, r in zip(dev.S, got_ranks)], chi) == got_kept
        for kb, r, blk in zip(got_kept, got_ranks, blocks):
            assert kb < r or r == min(chi, *blk.shape)
    assert sum(got_kept) == chi
    assert all(d["status"] == 0 for d in api.info_dicts(dev.info))


def test_adaptive_device_rounds_replay_bit_identically(api):
    # the batching form of an adaptive sector bond: the 32 uneven FP32 blocks (64..2048),
    # chi = 512, every trial rank starting at 16, the whole adaptive step (all rounds, the
    # selections and the round decisions) captured as ONE CUDA graph and replayed
    blocks = [b.astype(np.float32) for b in inputs.sector_blocks(N=32, lo=64, hi=2048, seed=104)]
    As = [torch.from_numpy(b).cuda() for b in blocks]
    plan = api.AdaptiveSectorsPlan([b.shape for b in blocks], 512, [16] * len(blocks), p=16, q=2, seed=103,
                                   dtype=torch.float32, device_rounds=True)
    plan.run(As)  # eager reference (also warms up)
    torch.cuda.synchronize()
    ref = ([s.clone() for s in plan.S], [u.clone() for u in plan.U], plan.k_out.clone(), plan.k_final.clone(),
           plan.rounds_dev.clone())
    assert int(ref[2].sum()) == 512 and int(ref[4].item()) >= 2
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.run(As)
    for s in plan.S:
        s.zero_()
    plan.k_out.zero_()
    plan.k_final.zero_()
    plan.rounds_dev.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(plan.k_out, ref[2]) and torch.equal(plan.k_final, ref[3])
    assert torch.equal(plan.rounds_dev, ref[4])
    for a, b, r in zip(plan.S, ref[0], ref[3].tolist()):  # entries past a block's final rank are unset
        assert torch.equal(a[:r], b[:r])
    for a, b, r in zip(plan.U, ref[1], ref[3].tolist()):
        assert torch.equal(a[:, :r], b[:, :r])
    assert all(d["status"] == 0 for d in api.info_dicts(plan.info))


def test_large_batch_chunks_concurrent(api):
    # a batch above 64 matrices runs in chunks of 64, concurrently on the chunk streams:
    # bit-identical to the serial run (RSVD_FLAG_SERIAL, every chunk and group on the
    # caller's stream), and sampled members at the FP64 bar against the oracle
    from paper_1710_01463_gb300 import _lib
    rng = np.random.default_rng(71)
    shapes = [(int(m), int(n)) for m, n in zip(rng.integers(40, 97, 150), rng.integers(40, 97, 150))]
    blocks = [inputs.spectral_matrix(m, n, inputs.exp_spectrum(min(m, n), 6.0), 500 + b)
              for b, (m, n) in enumerate(shapes)]
    ks = [min(10, m, n) for m, n in shapes]
    As = [torch.from_numpy(b).cuda() for b in blocks]
    _, S, Vt, _, info = api.rsvd_truncate_batched(As, ks, p=6, q=2, seed=13, stream=2)
    S = [s.clone() for s in S]
    Vt = [v.clone() for v in Vt]
    _, S2, Vt2, _, info2 = api.rsvd_truncate_batched(As, ks, p=6, q=2, seed=13, stream=2,
                                                     flags=_lib.RSVD_FLAG_SERIAL)
    torch.cuda.synchronize()
    for b in range(len(blocks)):
        assert torch.equal(S[b], S2[b]) and torch.equal(Vt[b], Vt2[b])
    assert all(d["status"] == 0 for d in api.info_dicts(info))
    assert all(d["status"] == 0 for d in api.info_dicts(info2))
    for b in (0, 63, 64, 100, 127, 128, 149):
        _, So, _ = orsvd.rsvd(blocks[b], ks[b], 6, 2, 13, 2 + b)
        assert np.all(np.abs(S[b].cpu().numpy() - So) <= sigma_tol(So)), b
