"""GPU parity of tebd_bond_update (Sec. III.A block update) against the oracle TEBD."""
import numpy as np
import pytest

from gpu_util import need_gpu, torch
from oracle import tebd as otebd
from paper_1710_01463_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    need_gpu()
    from paper_1710_01463_gb300 import tebd
    return tebd


def run_both(tebd, L, chi, dt, steps, p=10, q=2, seed=5):
    ch = tebd.TebdChain(L, chi, h=1.0, p=p, q=q, seed=seed)
    vec = inputs.product_state_vectors(L, 2, 102)
    ch.set_product_state(vec)
    ch.set_dt(dt)
    D = otebd.bond_dims(L, 2, chi)
    B, lam = otebd.product_state(vec, D)
    comp = otebd.make_compressor("rsvd", p=p, q=q, seed=seed)
    for s in range(steps):
        ch.step(s)
        otebd.trotter_step(B, lam, L, 1.0, dt, comp, s)
    torch.cuda.synchronize()
    return ch, B, lam


@pytest.mark.parametrize("L,chi,steps", [(8, 16, 3), (12, 8, 4)])
def test_tebd_steps_match_oracle(mods, L, chi, steps):
    ch, B, lam = run_both(mods, L, chi, 0.05, steps)
    lam_g = ch.schmidt_values()
    for j in range(1, L):
        a, b = lam_g[j], lam[j]
        np.testing.assert_allclose(a, b, atol=1e-10 * np.max(b) + 1e-14)
    e_g = otebd.mps_energy(ch.tensors(), L, 1.0)
    e_o = otebd.mps_energy(B, L, 1.0)
    assert e_g == pytest.approx(e_o, rel=1e-10)
    st = ch.info.cpu().numpy()
    assert np.all(st[..., 0] >= 0)


def test_tebd_converges_small_chain(mods):
    L = 6
    ch = mods.TebdChain(L, 8, h=1.0, p=10, q=2, seed=3)
    ch.set_product_state(inputs.product_state_vectors(L, 2, 102))
    ch.set_dt(0.1)
    for s in range(200):
        ch.step(s)
    torch.cuda.synchronize()
    e = otebd.mps_energy(ch.tensors(), L, 1.0)
    e0 = otebd.exact_ground_energy_ed(L, 1.0)
    assert 0 < e - e0 < 3e-5


def test_checkpoint_resume_is_exact(mods, tmp_path):
    L, chi = 10, 16
    a = mods.TebdChain(L, chi, seed=4)
    a.set_product_state(inputs.product_state_vectors(L, 2, 102))
    a.set_dt(0.05)
    for s in range(6):
        a.step(s)
    path = str(tmp_path / "state.npz")
    a.save(path, 6)
    for s in range(6, 10):
        a.step(s)
    b = mods.TebdChain(L, chi, seed=4)
    start = b.load(path)
    for s in range(start, 10):
        b.step(s)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a.B.cpu().numpy(), b.B.cpu().numpy())
    np.testing.assert_array_equal(a.lam.cpu().numpy(), b.lam.cpu().numpy())


def test_tebd_fp64_product_paths_agree():
    # a few Trotter steps with the products on the tensor cores (default) and on FP64 FMAs
    need_gpu()
    from paper_1710_01463_gb300.tebd import TebdChain
    from paper_1710_01463_gb300 import inputs as inp
    from oracle import tebd as ot
    L, chi = 12, 16
    res = []
    for simt in (False, True):
        ch = TebdChain(L, chi, h=1.0, p=6, q=2, seed=3, simt=simt)
        ch.set_product_state(inp.product_state_vectors(L, 2, 7))
        ch.set_dt(0.05)
        for s in range(6):
            ch.step(s)
        torch.cuda.synchronize()
        assert int((ch.info[..., 0] != 0).sum()) == 0
        res.append((ot.mps_energy(ch.tensors(), L, 1.0), ch.schmidt_values()))
    assert abs(res[0][0] - res[1][0]) <= 1e-10 * abs(res[1][0])
    for a, b in zip(res[0][1], res[1][1]):
        np.testing.assert_allclose(a, b, atol=1e-10)


def run_model(tebd, L, chi, dt, steps, S=0.5, W=None, h=1.0, p=6, q=2, seed=4):
    d = 2 ** W if W else int(2 * S) + 1
    ch = tebd.TebdChain(L, chi, h=h, p=p, q=q, seed=seed, S=S, W=W)
    vec = inputs.product_state_vectors(L, d, 77)
    ch.set_product_state(vec)
    ch.set_dt(dt)
    terms = otebd.cylinder_bond_terms(L, h, W) if W else otebd.chain_bond_terms(L, h, S)
    D = otebd.bond_dims(L, d, chi)
    B, lam = otebd.product_state(vec, D)
    comp = otebd.make_compressor("rsvd", p=p, q=q, seed=seed)
    for s in range(steps):
        ch.step(s)
        otebd.trotter_step(B, lam, L, h, dt, comp, s, terms)
    torch.cuda.synchronize()
    return ch, B, lam, terms


@pytest.mark.parametrize("S,W,L,chi,h", [(1.0, None, 8, 9, 1.2), (1.5, None, 6, 12, 1.5), (None, 2, 6, 16, 3.0)])
def test_large_d_models_match_oracle(mods, S, W, L, chi, h):
    # spin-S chains (d = 2S + 1) and the 2D cylinder (d = 2^W), Sec. III.B: the same bond
    # update with larger local dimension
    ch, B, lam, terms = run_model(mods, L, chi, 0.05, 4, S=S or 0.5, W=W, h=h)
    assert int((ch.info[..., 0] != 0).sum()) == 0
    lam_g = ch.schmidt_values()
    for j in range(1, L):
        np.testing.assert_allclose(lam_g[j], lam[j], atol=1e-10 * np.max(lam[j]) + 1e-14)
    e_g = otebd.mps_energy(ch.tensors(), L, h, terms)
    e_o = otebd.mps_energy(B, L, h, terms)
    assert e_g == pytest.approx(e_o, rel=1e-10)


def test_spin1_chain_reaches_ed_ground_energy(mods):
    # paramagnetic side (gap 1.0 at L = 6): imaginary time 7.5 reaches the ground state from
    # a product state with generic overlap
    S, L, h = 1.0, 6, 2.0
    ch = mods.TebdChain(L, 27, h=h, p=10, q=2, seed=8, S=S)
    ch.set_product_state(np.ones((L, 3)) + 0.1 * np.arange(L * 3).reshape(L, 3))
    step = 0
    for dt, n in ((0.1, 60), (0.02, 60), (0.005, 60)):
        ch.set_dt(dt)
        for _ in range(n):
            ch.step(step)
            step += 1
    torch.cuda.synchronize()
    e = otebd.mps_energy(ch.tensors(), L, h, otebd.chain_bond_terms(L, h, S))
    e0 = float(np.linalg.eigvalsh(otebd.dense_chain_hamiltonian(L, h, S))[0])
    assert abs(e - e0) <= 1e-7 * abs(e0)


@pytest.mark.parametrize("W,L,chi,steps", [(2, 6, 16, 4), (1, 8, 8, 4), (3, 4, 24, 2)])
def test_product_update_matches_oracle(mods, W, L, chi, steps):
    # the cylinder with product updates (Sec. III.A P): each bond as W gates of K = 2
    # Kronecker terms, one factored compression per gate
    h, dt, p, q, seed = 3.0, 0.05, 6, 2, 9
    d = 2 ** W
    ch = mods.TebdChain(L, chi, h=h, p=p, q=q, seed=seed, W=W, update="product")
    vec = inputs.product_state_vectors(L, d, 78)
    ch.set_product_state(vec)
    ch.set_dt(dt)
    B, lam = otebd.product_state(vec, otebd.bond_dims(L, d, chi))
    comp = otebd.make_compressor("rsvd", p=p, q=q, seed=seed)
    for s in range(steps):
        ch.step(s)
        otebd.trotter_step_product(B, lam, L, h, W, dt, comp, s)
    torch.cuda.synchronize()
    assert int((ch.info[..., 0] != 0).sum()) == 0
    lam_g = ch.schmidt_values()
    for j in range(1, L):
        np.testing.assert_allclose(lam_g[j], lam[j], atol=1e-10 * np.max(lam[j]) + 1e-14)
    terms = otebd.cylinder_bond_terms(L, h, W)
    assert otebd.mps_energy(ch.tensors(), L, h, terms) == pytest.approx(otebd.mps_energy(B, L, h, terms), rel=1e-10)
    te = ch.trunc_err.cpu().numpy()
    assert np.all(te >= 0) and np.all(te < 1e-2)


def test_product_and_block_updates_reach_the_same_ground_state(mods):
    # the two Trotter forms differ by O(dt^2) in the state; both approach the ED ground
    # energy of a small cylinder
    L, W, h = 4, 2, 3.0
    e0 = float(np.linalg.eigvalsh(otebd.dense_cylinder_hamiltonian(L, h, W))[0])
    terms = otebd.cylinder_bond_terms(L, h, W)
    out = {}
    for update in ("block", "product"):
        ch = mods.TebdChain(L, 16, h=h, p=10, q=2, seed=2, W=W, update=update)
        ch.set_product_state(np.ones((L, 4)) + 0.1 * np.arange(L * 4).reshape(L, 4))
        step = 0
        for dt, n in ((0.2, 40), (0.02, 200)):
            ch.set_dt(dt)
            for _ in range(n):
                ch.step(step)
                step += 1
        torch.cuda.synchronize()
        out[update] = otebd.mps_energy(ch.tensors(), L, h, terms)
    for e in out.values():
        assert 0 <= e - e0 < 1e-6 * abs(e0)
