"""Pins of the oracle's TEBD (Sec. III) against exact results.

* the ground energy of the open transverse-field Ising chain: free-fermion
  singular-value form, the h = 1 closed form and exact diagonalisation agree;
* the MPS energy contraction equals <psi|H|psi> of the dense state;
* the bond gates equal scipy's matrix exponential;
* TEBD without truncation converges to the exact ground energy with the
  second-order Trotter error: energy error ~ dt^4 (ratio ~ 5^4 for dt / 5);
* RSVD-TEBD equals TSVD-TEBD when l covers every bond.
"""
import numpy as np
import pytest
from scipy.linalg import expm

from oracle import tebd
from paper_1710_01463_gb300 import inputs

E0_L64 = -81.12598012314353


@pytest.mark.parametrize("L", [1, 2, 3, 5, 6, 8])
def test_ground_energy_forms_agree_with_ed(L):
    e_ed = tebd.exact_ground_energy_ed(L, 1.0)
    assert tebd.free_fermion_ground_energy(L, 1.0) == pytest.approx(e_ed, rel=1e-12)
    assert tebd.critical_ground_energy(L) == pytest.approx(e_ed, rel=1e-12)


@pytest.mark.parametrize("h", [0.3, 0.7, 1.6])
def test_free_fermion_off_critical_matches_ed(h):
    assert tebd.free_fermion_ground_energy(7, h) == pytest.approx(tebd.exact_ground_energy_ed(7, h), rel=1e-12)


def test_l64_closed_form_value():
    assert tebd.critical_ground_energy(64) == pytest.approx(E0_L64, rel=1e-14)
    assert tebd.free_fermion_ground_energy(64, 1.0) == pytest.approx(E0_L64, rel=1e-13)


def test_bond_terms_sum_to_hamiltonian():
    L = 5
    H = np.zeros((2 ** L, 2 ** L))
    for i in range(L - 1):
        H += np.kron(np.kron(np.eye(2 ** i), tebd.bond_hamiltonian(i, L, 0.8)), np.eye(2 ** (L - i - 2)))
    np.testing.assert_allclose(H, tebd.dense_hamiltonian(L, 0.8), atol=1e-13)


def test_gate_is_matrix_exponential():
    hb = tebd.bond_hamiltonian(3, 10, 1.0)
    np.testing.assert_allclose(tebd.gate(hb, 0.005), expm(-0.005 * hb), atol=1e-14)


def test_mps_energy_matches_dense():
    L, d = 6, 2
    D = tebd.bond_dims(L, d, 4)
    rng = np.random.default_rng(0)
    B = [rng.standard_normal((D[i], d, D[i + 1])) for i in range(L)]
    psi = tebd.mps_to_dense(B)
    H = tebd.dense_hamiltonian(L, 0.9)
    assert tebd.mps_energy(B, L, 0.9) == pytest.approx(psi @ H @ psi / (psi @ psi), rel=1e-12)


def run(L, chi, dt, steps, kind, h=1.0):
    D = tebd.bond_dims(L, 2, chi)
    B, lam = tebd.product_state(inputs.product_state_vectors(L, 2, 102), D)
    comp = tebd.make_compressor(kind, p=10, q=2, seed=5)
    for s in range(steps):
        tebd.trotter_step(B, lam, L, h, dt, comp, s)
    return B, lam


def test_tebd_trotter_error_scales_as_dt4():
    L = 6
    e0 = tebd.exact_ground_energy_ed(L, 1.0)
    B1, _ = run(L, 8, 0.1, 200, "tsvd")
    B2, _ = run(L, 8, 0.02, 1000, "tsvd")
    e1 = tebd.mps_energy(B1, L, 1.0) - e0
    e2 = tebd.mps_energy(B2, L, 1.0) - e0
    assert e1 > 0 and e2 > 0
    assert 400 < e1 / e2 < 900          # 5^4 = 625
    assert e2 < 1e-7


def test_tebd_rsvd_equals_tsvd_without_truncation():
    L = 6
    B1, lam1 = run(L, 8, 0.1, 30, "tsvd")
    B2, lam2 = run(L, 8, 0.1, 30, "rsvd")
    assert tebd.mps_energy(B1, L, 1.0) == pytest.approx(tebd.mps_energy(B2, L, 1.0), rel=1e-12)
    for a, b in zip(lam1, lam2):
        np.testing.assert_allclose(a, b, atol=1e-12)


def test_schmidt_values_normalised_and_entropy():
    L = 6
    _, lam = run(L, 8, 0.1, 50, "tsvd")
    for j in range(1, L):
        assert np.sum(lam[j] ** 2) == pytest.approx(1.0, rel=1e-12)
    assert tebd.entanglement_entropy([1.0]) == 0.0
    assert tebd.entanglement_entropy([2 ** -0.5, 2 ** -0.5]) == pytest.approx(np.log(2.0))


# ---- spin-S chain and 2D cylinder (Sec. III.B)

@pytest.mark.parametrize("S", [0.5, 1.0, 1.5, 2.0, 3.5])
def test_spin_ops_obey_the_spin_algebra(S):
    # pins the S^x elements (the paper's printed formula is garbled) by the algebra alone:
    # S^+ = 2 triu(S^x) raises m by one, [S^+, S^-] = 2 S^z and S.S = S(S+1)
    sx, sz = tebd.spin_ops(S)
    d = sx.shape[0]
    assert d == int(2 * S) + 1
    sp = 2.0 * np.triu(sx, 1)
    sm = sp.T
    np.testing.assert_allclose(sz @ sp - sp @ sz, sp, atol=1e-13)
    np.testing.assert_allclose(sp @ sm - sm @ sp, 2.0 * sz, atol=1e-12)
    casimir = sx @ sx - (sp - sm) @ (sp - sm) / 4.0 + sz @ sz
    np.testing.assert_allclose(casimir, S * (S + 1) * np.eye(d), atol=1e-12)
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(sx)), np.sort(np.diag(sz)), atol=1e-12)


def test_spin_half_chain_is_the_pauli_chain():
    L, h = 6, 0.8
    for i in range(L - 1):
        fl = 1.0 if i == 0 else 0.5
        fr = 1.0 if i + 1 == L - 1 else 0.5
        ref = -np.kron(tebd.PAULI_Z, tebd.PAULI_Z) - h * (fl * np.kron(tebd.PAULI_X, tebd.EYE2)
                                                          + fr * np.kron(tebd.EYE2, tebd.PAULI_X))
        np.testing.assert_allclose(tebd.bond_hamiltonian(i, L, h, 0.5), ref, atol=1e-14)
    np.testing.assert_allclose(tebd.dense_chain_hamiltonian(4, h, 0.5), tebd.dense_hamiltonian(4, h), atol=1e-13)


def embed(terms, d, L):
    H = np.zeros((d ** L, d ** L))
    for i, t in enumerate(terms):
        H += np.kron(np.kron(np.eye(d ** i), t), np.eye(d ** (L - i - 2)))
    return H


@pytest.mark.parametrize("S,L", [(1.0, 4), (1.5, 3), (2.0, 3)])
def test_spin_chain_bond_terms_sum_to_the_hamiltonian(S, L):
    h = 1.3
    d = int(2 * S) + 1
    np.testing.assert_allclose(embed(tebd.chain_bond_terms(L, h, S), d, L), tebd.dense_chain_hamiltonian(L, h, S),
                               atol=1e-11)


@pytest.mark.parametrize("W,L", [(2, 3), (3, 2)])
def test_cylinder_bond_terms_sum_to_the_hamiltonian(W, L):
    h = 3.0
    np.testing.assert_allclose(embed(tebd.cylinder_bond_terms(L, h, W), 2 ** W, L),
                               tebd.dense_cylinder_hamiltonian(L, h, W), atol=1e-11)


def test_cylinder_of_width_one_is_the_chain_shifted():
    # one spin per ring: the ring coupling Z_j Z_{j+1 mod 1} = 1 adds -1 per ring
    L, h = 5, 0.7
    np.testing.assert_allclose(tebd.dense_cylinder_hamiltonian(L, h, 1), tebd.dense_hamiltonian(L, h) - L * np.eye(2 ** L),
                               atol=1e-12)


def test_spin1_imaginary_tebd_reaches_the_ed_ground_energy():
    S, L, h = 1.0, 5, 1.2
    d = 3
    e0 = float(np.linalg.eigvalsh(tebd.dense_chain_hamiltonian(L, h, S))[0])
    terms = tebd.chain_bond_terms(L, h, S)
    D = tebd.bond_dims(L, d, 27)
    vec = np.ones((L, d)) + 0.1 * np.arange(L * d).reshape(L, d)
    B, lam = tebd.product_state(vec, D)
    comp = tebd.make_compressor("tsvd")
    step = 0
    for dt, n in ((0.1, 60), (0.02, 60), (0.005, 60)):
        for _ in range(n):
            tebd.trotter_step(B, lam, L, h, dt, comp, step, terms)
            step += 1
    e = tebd.mps_energy(B, L, h, terms)
    assert abs(e - e0) <= 1e-4 * abs(e0)


def random_bond(rng, Dl, d, Dm, Dr):
    B = [rng.standard_normal((Dl, d, Dm)), rng.standard_normal((Dm, d, Dr))]
    lam = [np.sort(rng.uniform(0.1, 1.0, Dl))[::-1], np.ones(Dm), np.ones(Dr)]
    return B, lam


def test_product_update_is_the_block_update_of_the_kronecker_sum():
    # P update with terms (uL_k, uR_k) == B update with G = sum_k uL_k (x) uR_k: pins the
    # index placement of X and Y (the random terms are neither symmetric nor equal)
    rng = np.random.default_rng(61)
    Dl, d, Dm, Dr, K = 4, 3, 5, 6, 3
    uL = rng.standard_normal((K, d, d))
    uR = rng.standard_normal((K, d, d))
    G = sum(np.kron(uL[k], uR[k]) for k in range(K))
    comp = tebd.make_compressor("tsvd")
    Bp, lp = random_bond(rng, Dl, d, Dm, Dr)
    Bb = [t.copy() for t in Bp]
    lb = [v.copy() for v in lp]
    ep = tebd.product_update(Bp, lp, 0, uL, uR, comp, 0)
    eb = tebd.bond_update(Bb, lb, 0, G, comp, 0)
    assert ep == pytest.approx(eb, rel=1e-12, abs=1e-15)
    np.testing.assert_allclose(lp[1], lb[1], atol=1e-13)
    # singular vectors up to the shared sign rule
    np.testing.assert_allclose(Bp[1], Bb[1], atol=1e-11)
    np.testing.assert_allclose(Bp[0], Bb[0], atol=1e-11)


def test_product_matrix_has_the_spectrum_of_theta():
    # the paper's (K D) x (d D') matrix R Y and theta = X Y share singular values and right
    # singular vectors
    rng = np.random.default_rng(62)
    Dl, d, Dm, Dr, K = 6, 4, 5, 7, 2
    B, lam = random_bond(rng, Dl, d, Dm, Dr)
    uL = rng.standard_normal((K, d, d))
    uR = rng.standard_normal((K, d, d))
    X, Y, RY = tebd.product_factors(B, lam, 0, uL, uR)
    assert RY.shape == (K * Dm, d * Dr)
    s1 = np.linalg.svd(X @ Y, compute_uv=False)[:K * Dm]
    s2 = np.linalg.svd(RY, compute_uv=False)
    np.testing.assert_allclose(s1, s2, rtol=1e-12, atol=1e-13 * s2[0])
    _, _, v1 = np.linalg.svd(X @ Y)
    _, _, v2 = np.linalg.svd(RY)
    np.testing.assert_allclose(np.abs(v1[:4] @ v2[:4].T), np.eye(4), atol=1e-10)


def test_gate_terms_reconstruct_the_gate():
    rng = np.random.default_rng(63)
    d = 3
    G = rng.standard_normal((d * d, d * d))
    uL, uR = tebd.gate_terms(G, d)
    assert len(uL) == d * d
    np.testing.assert_allclose(sum(np.kron(a, b) for a, b in zip(uL, uR)), G, atol=1e-12)
    # the Ising coupling gate has operator-Schmidt rank 2, a product gate rank 1
    zz = expm(0.3 * np.kron(tebd.PAULI_Z, tebd.PAULI_Z))
    assert len(tebd.gate_terms(zz, 2)[0]) == 2
    assert len(tebd.gate_terms(np.kron(rng.standard_normal((2, 2)), rng.standard_normal((2, 2))), 2)[0]) == 1


@pytest.mark.parametrize("W,i,L", [(1, 1, 4), (2, 0, 4), (3, 1, 3), (2, 2, 4)])
def test_cylinder_product_gates_are_the_symmetric_split(W, i, L):
    # the W gates multiply to exp(-tau A/2) exp(-tau C) exp(-tau A/2) (A: the rings' own
    # terms, C: the couplings along the cylinder), built here from the bond term by expm
    h, tau = 3.0, 0.07
    d = 2 ** W
    hb = tebd.cylinder_bond_hamiltonian(i, L, h, W)
    C = -sum(np.kron(z, z) for z in tebd.ring_ops(W)[0])
    A = hb - C
    want = expm(-tau / 2 * A) @ expm(-tau * C) @ expm(-tau / 2 * A)
    got = np.eye(d * d)
    for uL, uR in tebd.cylinder_product_gates(i, L, h, W, tau):
        assert len(uL) == 2
        got = sum(np.kron(a, b) for a, b in zip(uL, uR)) @ got
    np.testing.assert_allclose(got, want, atol=1e-12)
    # a second-order split of exp(-tau hb): the error falls by 8 when tau halves
    errs = []
    for t in (tau, tau / 2):
        g = np.eye(d * d)
        for uL, uR in tebd.cylinder_product_gates(i, L, h, W, t):
            g = sum(np.kron(a, b) for a, b in zip(uL, uR)) @ g
        errs.append(np.linalg.norm(g - expm(-t * hb)))
    if W > 1:
        assert 6.0 < errs[0] / errs[1] < 10.0


def test_product_tebd_reaches_the_cylinder_ground_state_at_second_order():
    # product-update TEBD of the W = 2 cylinder without truncation (chi = 16 holds L = 4
    # exactly): the converged state is off by O(dt^2), so its (variational) energy error
    # falls as dt^4
    L, W, h = 4, 2, 3.0
    d = 2 ** W
    e0 = float(np.linalg.eigvalsh(tebd.dense_cylinder_hamiltonian(L, h, W))[0])
    terms = tebd.cylinder_bond_terms(L, h, W)
    comp = tebd.make_compressor("tsvd")
    errs = []
    for dts in (((0.2, 40), (0.08, 200)), ((0.2, 40), (0.04, 400))):
        B, lam = tebd.product_state(np.ones((L, d)) + 0.1 * np.arange(L * d).reshape(L, d), tebd.bond_dims(L, d, 16))
        step = 0
        for dt, n in dts:
            for _ in range(n):
                tebd.trotter_step_product(B, lam, L, h, W, dt, comp, step)
                step += 1
        errs.append(tebd.mps_energy(B, L, h, terms) - e0)
    assert 0 < errs[1] < errs[0] < 1e-2 * abs(e0)
    assert 12.0 < errs[0] / errs[1] < 20.0
