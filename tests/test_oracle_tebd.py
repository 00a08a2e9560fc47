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
