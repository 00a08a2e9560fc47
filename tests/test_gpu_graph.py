"""The asynchronous entry points are graph-capturable: a call captured into a CUDA graph
and replayed gives bit-identical results to the same call run eagerly (every sum has a
fixed order, so the kernels are deterministic).  Covers rsvd_truncate (side streams for
concurrent groups, tensor maps of the sliced FP64 products) and one TEBD Trotter step
(three layers of tebd_bond_update)."""
import numpy as np
import pytest

from gpu_util import need_gpu, torch
from paper_1710_01463_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    need_gpu()
    from paper_1710_01463_gb300 import api, tebd
    return api, tebd


def test_rsvd_truncate_replays_bit_identically(mods):
    api, _ = mods
    A = torch.from_numpy(inputs.dense_case()).cuda()
    work = torch.empty(api.rsvd_workspace_size(256, 256, 32, 8, 2), dtype=torch.uint8, device="cuda")
    U0, S0, V0, _ = api.rsvd_truncate(A, 32, 8, 2, 201, work=work)  # eager (also warms up)
    torch.cuda.synchronize()
    s0, u0, v0 = S0.clone(), U0.clone(), V0.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        U, S, Vt, info = api.rsvd_truncate(A, 32, 8, 2, 201, work=work)
    S.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(S, s0) and torch.equal(U, u0) and torch.equal(Vt, v0)
    assert api.info_dicts(info)[0]["status"] == 0


def test_tebd_step_replays_bit_identically(mods):
    _, tebd = mods
    L, chi = 16, 32
    ch = tebd.TebdChain(L, chi, h=1.0, p=10, q=2, seed=3)
    ch.set_product_state(inputs.product_state_vectors(L, 2, 102))
    ch.set_dt(0.05)
    for s in range(4):
        ch.step(s)
    torch.cuda.synchronize()
    B0, lam0 = ch.B.clone(), ch.lam.clone()
    ch.step(4)  # eager reference step
    torch.cuda.synchronize()
    B1, lam1 = ch.B.clone(), ch.lam.clone()
    ch.B.copy_(B0)
    ch.lam.copy_(lam0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ch.step(4)
    ch.B.copy_(B0)  # capture runs nothing; start the replay from the same state
    ch.lam.copy_(lam0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(ch.B, B1) and torch.equal(ch.lam, lam1)
    assert int((ch.info[..., 0] != 0).sum()) == 0
    assert np.isfinite(ch.trunc_err.cpu().numpy()).all()


@pytest.mark.parametrize("policy", ["maximal", "estimate"])
def test_sector_bond_step_replays_bit_identically(mods, policy):
    # the batching form of the sector workload: the 32 uneven blocks (64..2048) of one
    # block-diagonal bond, FP32 products, with the global top-chi selection, as ONE graph
    # replay (no host synchronisation inside the step); trial ranks maximal or from a
    # previous step's kept counts + 16
    api, _ = mods
    blocks = [b.astype(np.float32) for b in inputs.sector_blocks(N=32, lo=64, hi=2048, seed=104)]
    As = [torch.from_numpy(b).cuda() for b in blocks]
    ks = [min(512, *b.shape) for b in blocks]
    plan = api.BatchedPlan([b.shape for b in blocks], ks, 16, 2, 103, 0, torch.float32, "cuda", chi_global=512)
    plan.run(As)
    torch.cuda.synchronize()
    if policy == "estimate":
        kept = plan.k_out.cpu().tolist()
        ks = [min(min(b.shape), kk + 16) for b, kk in zip(blocks, kept)]
        plan = api.BatchedPlan([b.shape for b in blocks], ks, 16, 2, 103, 0, torch.float32, "cuda", chi_global=512)
        plan.run(As)  # eager reference
        torch.cuda.synchronize()
    ref = ([s.clone() for s in plan.S], [u.clone() for u in plan.U], [v.clone() for v in plan.Vt],
           plan.k_out.clone())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.run(As)
    for s in plan.S:
        s.zero_()
    plan.k_out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(plan.k_out, ref[3]) and int(plan.k_out.sum()) == 512
    for a, b in zip(plan.S, ref[0]):
        assert torch.equal(a, b)
    for a, b in zip(plan.U, ref[1]):
        assert torch.equal(a, b)
    for a, b in zip(plan.Vt, ref[2]):
        assert torch.equal(a, b)
    assert all(d["status"] == 0 for d in api.info_dicts(plan.info))
