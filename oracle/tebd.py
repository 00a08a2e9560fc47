"""Oracle: imaginary-time TEBD of the open transverse-field Ising chain.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Models (Sec. III.B): the spin-S chain of Eq. ising_chain and the 2D cylinder of
Eq. ising_cylinder mapped onto a chain of rings (d = 2^W).  The paper writes the
couplings in x and the field in z; this module uses the unitarily equivalent form
with the axes exchanged (rotate x <-> z, then by pi about x to flip the field's
sign), which has the same spectrum: at S = 1/2, H = -sum Z_j Z_{j+1} - h sum X_j.
Open boundaries; the spin-1/2 chain is critical at h = 1.

TEBD (Sec. III.A "block update (B)", Sec. III.C protocol), readings where the
paper is silent:

* MPS in right-canonical "B" form (Hastings' variant of Vidal's form): tensors
  B[i] of shape (D[i], d, D[i+1]), Schmidt values lam[j] on virtual bond j
  (lam[0] = lam[L] = [1]).  No division by Schmidt values is ever needed.
* Bond dimensions are fixed at the caps D[j] = min(d^j, d^(L-j), chi) from the
  first step on (zero-padded), so every bond update keeps rank k = D[i+1].
* Field split: an interior site gives h/2 to each of its two bonds; an edge
  site gives its full field to its only bond.
* Second-order Trotter step: exp(-dt/2 H_A) exp(-dt H_B) exp(-dt/2 H_A), where
  layer A holds the bonds (0,1), (2,3), ... and layer B the bonds (1,2), (3,4), ...
* Bond update on sites (i, i+1) with gate G (d^2 x d^2):
    theta_B[a,s1,s2,c] = sum G[(s1 s2),(t1 t2)] B[i][a,t1,b] B[i+1][b,t2,c]
    theta = lam[i][a] * theta_B, reshaped (D[i] d) x (d D[i+2])
    (U, S, V^T) = rank-D[i+1] truncated factorization of theta
    B[i+1] <- V^T,  B[i] <- theta_B V / ||S||,  lam[i+1] <- S / ||S||
* Product update (Sec. III.A, "product update (P)"): the gate as a sum of K
  Kronecker products of single-site operators, theta = X Y with X of K D[i+1]
  columns; the cylinder's bonds as W gates of K = 2 (its commuting couplings),
  the rings' own terms folded into the first and last (see
  cylinder_product_gates).
* Philox stream of a bond update: (3 * step + layer) * L + i, layer in {0,1,2}.
* Energy: exact contraction <psi|H|psi> / <psi|psi> (no canonical-form
  assumption).
"""
import numpy as np

from .rsvd import rsvd, tsvd

PAULI_X = np.array([[0.0, 1.0], [1.0, 0.0]])
PAULI_Z = np.array([[1.0, 0.0], [0.0, -1.0]])
EYE2 = np.eye(2)


def spin_ops(S):
    """Spin-S operators (S^x, S^z), d = 2S + 1, basis m = S, S-1, ..., -S (Sec. III.B).

    <m|S^z|m> = m and <m+1|S^x|m> = <m|S^x|m+1> = sqrt(S(S+1) - m(m+1)) / 2, the
    standard ladder-operator elements (the paper's printed X element is garbled:
    its radicand is negative at S = 1/2; for S = 1/2 these are Pauli / 2, as
    the paper states they must be).
    """
    d = int(round(2 * S)) + 1
    m = S - np.arange(d)
    sz = np.diag(m)
    sx = np.zeros((d, d))
    for a in range(d - 1):  # rows a (m = S - a) and a + 1 (m - 1)
        mm = m[a + 1]
        v = 0.5 * np.sqrt(S * (S + 1) - mm * (mm + 1))
        sx[a, a + 1] = sx[a + 1, a] = v
    return sx, sz


def bond_dims(L, d, chi):
    """D[j] = min(d^j, d^(L-j), chi), j = 0..L."""
    return [int(min(d ** min(j, L - j), chi)) for j in range(L + 1)]


def bond_hamiltonian(i, L, h, S=0.5):
    """Two-site term of bond (i, i+1), d^2 x d^2 on (s_i, s_{i+1}), of the spin-S chain
    H = -(1/S^2) sum S^z_j S^z_{j+1} - (h/S) sum S^x_j (Eq. ising_chain with x and z
    exchanged, a unitary change of basis); S = 1/2 is -sum Z Z - h sum X (Pauli)."""
    sx, sz = spin_ops(S)
    one = np.eye(sx.shape[0])
    fl = 1.0 if i == 0 else 0.5
    fr = 1.0 if i + 1 == L - 1 else 0.5
    return -np.kron(sz, sz) / S ** 2 - (h / S) * (fl * np.kron(sx, one) + fr * np.kron(one, sx))


def ring_ops(W):
    """One ring of the W-site circumference of the 2D cylinder (Eq. ising_cylinder) as a
    site of dimension d = 2^W: Z_j, X_j (Pauli on spin j of the ring), the ring's own
    coupling sum_j Z_j Z_{j+1 mod W} and sum_j X_j (x and z exchanged as for the chain)."""
    def on(op, j):
        out = np.ones((1, 1))
        for t in range(W):
            out = np.kron(out, op if t == j else EYE2)
        return out
    Z = [on(PAULI_Z, j) for j in range(W)]
    X = [on(PAULI_X, j) for j in range(W)]
    ring = sum(Z[j] @ Z[(j + 1) % W] for j in range(W))
    return Z, X, ring, sum(X)


def cylinder_bond_hamiltonian(i, L, h, W):
    """Two-site term of rings (i, i+1) of the cylinder mapped onto a chain of L rings:
    -sum_j Z_{i,j} Z_{i+1,j}, plus each ring's own terms -ring - h sum_j X_j shared between
    its bonds like the chain's field (interior rings half to each bond, edge rings all)."""
    Z, X, ring, xsum = ring_ops(W)
    one = np.eye(2 ** W)
    fl = 1.0 if i == 0 else 0.5
    fr = 1.0 if i + 1 == L - 1 else 0.5
    onsite = -ring - h * xsum
    inter = -sum(np.kron(Z[j], Z[j]) for j in range(W))
    return inter + fl * np.kron(onsite, one) + fr * np.kron(one, onsite)


def gate(hb, tau):
    """exp(-tau h_b) of a symmetric bond Hamiltonian, through its eigenbasis."""
    w, V = np.linalg.eigh(hb)
    return (V * np.exp(-tau * w)[None, :]) @ V.T


def product_state(vectors, D):
    """Zero-padded MPS of a product state: B[i][0, :, 0] = vectors[i]."""
    L, d = vectors.shape
    B = []
    for i in range(L):
        t = np.zeros((D[i], d, D[i + 1]))
        t[0, :, 0] = vectors[i] / np.linalg.norm(vectors[i])
        B.append(t)
    lam = []
    for j in range(L + 1):
        v = np.zeros(D[j])
        v[0] = 1.0
        lam.append(v)
    return B, lam


def bond_update(B, lam, i, G, compress, stream):
    """One TEBD block update on sites (i, i+1); returns the discarded weight."""
    Dl, d, _ = B[i].shape
    Dr = B[i + 1].shape[2]
    k = B[i].shape[2]
    two = np.einsum("atb,buc->atuc", B[i], B[i + 1])
    G4 = G.reshape(d, d, d, d)
    thetaB = np.einsum("stxy,axyc->astc", G4, two)
    theta = lam[i][:, None, None, None] * thetaB
    M = theta.reshape(Dl * d, d * Dr)
    MB = thetaB.reshape(Dl * d, d * Dr)
    U, S, Vt = compress(M, k, stream)
    nrm = float(np.linalg.norm(S))
    B[i + 1] = Vt.reshape(k, d, Dr).copy()
    B[i] = (MB @ Vt.T / nrm).reshape(Dl, d, k)
    lam[i + 1] = S / nrm
    tot = float(np.sum(M * M))
    return max(0.0, 1.0 - nrm * nrm / tot) if tot > 0 else 0.0


def product_update(B, lam, i, uL, uR, compress, stream):
    """One TEBD product update (Sec. III.A, "product update (P)") on sites (i, i+1)
    with the two-site gate sum_k uL[k] (x) uR[k] (K terms of d x d operators);
    returns the discarded weight.

    Each side takes its K single-site operators, which widens the bond to K D[i+1]:
      XB[(a,s1),(k,b)] = sum_t uL[k][s1,t] B[i][a,t,b],   X = lam[i][a] XB
      Y[(k,b),(s2,c)]  = sum_t uR[k][s2,t] B[i+1][b,t,c]
    so theta = X Y and theta_B = XB Y, (D[i] d) x (d D[i+2]) of rank <= K D[i+1].
    The bond is compressed from theta = X Y exactly as in the block update.  With
    X = Q_X R (thin QR), theta and the (K D[i+1]) x (d D[i+2]) matrix R Y of the
    paper's P update have the same singular values and right singular vectors,
    and Alg. RSVD with the same Omega gives the same B = Q^T A for both (their
    samples differ by the isometry Q_X)."""
    Dl, d, k = B[i].shape
    Dr = B[i + 1].shape[2]
    K = len(uL)
    XB = np.einsum("kst,atb->askb", np.asarray(uL), B[i]).reshape(Dl * d, K * k)
    Y = np.einsum("kst,btc->kbsc", np.asarray(uR), B[i + 1]).reshape(K * k, d * Dr)
    X = np.repeat(lam[i], d)[:, None] * XB
    M = X @ Y
    MB = XB @ Y
    U, S, Vt = compress(M, k, stream)
    nrm = float(np.linalg.norm(S))
    B[i + 1] = Vt.reshape(k, d, Dr).copy()
    B[i] = (MB @ Vt.T / nrm).reshape(Dl, d, k)
    lam[i + 1] = S / nrm
    tot = float(np.sum(M * M))
    return max(0.0, 1.0 - nrm * nrm / tot) if tot > 0 else 0.0


def product_factors(B, lam, i, uL, uR):
    """(X, Y) of the product update and the paper's (K D[i+1]) x (d D[i+2]) matrix
    R Y (X = Q_X R, thin QR), for checks of the P form."""
    Dl, d, k = B[i].shape
    Dr = B[i + 1].shape[2]
    K = len(uL)
    XB = np.einsum("kst,atb->askb", np.asarray(uL), B[i]).reshape(Dl * d, K * k)
    Y = np.einsum("kst,btc->kbsc", np.asarray(uR), B[i + 1]).reshape(K * k, d * Dr)
    X = np.repeat(lam[i], d)[:, None] * XB
    R = np.linalg.qr(X, mode="r") if X.shape[0] >= X.shape[1] else X
    return X, Y, R @ Y


def gate_terms(G, d, tol=1e-14):
    """Operator-Schmidt form of a two-site gate: G[(s1 s2),(t1 t2)] = sum_k
    uL[k][s1,t1] uR[k][s2,t2], from the SVD of G regrouped as ((s1 t1),(s2 t2));
    terms below tol times the largest are dropped.  Returns (uL, uR), K x d x d."""
    R = np.asarray(G).reshape(d, d, d, d).transpose(0, 2, 1, 3).reshape(d * d, d * d)
    U, s, Vt = np.linalg.svd(R)
    K = max(1, int(np.sum(s > tol * s[0]))) if s[0] > 0 else 1
    w = np.sqrt(s[:K])
    uL = (U[:, :K] * w).T.reshape(K, d, d)
    uR = (Vt[:K].T * w).T.reshape(K, d, d)
    return uL, uR


def cylinder_product_gates(i, L, h, W, tau):
    """The bond (i, i+1) of the W-wide cylinder as W gates of K = 2 terms each, the
    form in which the product update pays (K = 2 < d = 2^W).

    The bond term is C + A with C = -sum_j Z_{i,j} Z_{i+1,j} (W commuting couplings)
    and A its share of the two rings' own terms (a sum of single-ring operators).
    exp(-tau (A + C)) is split symmetrically as exp(-tau A / 2) prod_j exp(-tau C_j)
    exp(-tau A / 2) (error O(tau^3), the order of the layer splitting), with
    exp(-tau C_j) = cosh(tau) 1 (x) 1 + sinh(tau) Z_j (x) Z_j and exp(-tau A / 2) =
    gL (x) gR folded into the first and the last coupling.  Returns W pairs
    (uL, uR), applied in list order."""
    Z, X, ring, xsum = ring_ops(W)
    fl = 1.0 if i == 0 else 0.5
    fr = 1.0 if i + 1 == L - 1 else 0.5
    onsite = -ring - h * xsum
    gL = gate_1site(fl * onsite, tau / 2)
    gR = gate_1site(fr * onsite, tau / 2)
    one = np.eye(2 ** W)
    ch, sh = np.cosh(tau), np.sinh(tau)
    out = []
    for j in range(W):
        aL, aR = [ch * one, sh * Z[j]], [one, Z[j]]
        if j == 0:  # exp(-tau A / 2) acts first
            aL = [u @ gL for u in aL]
            aR = [u @ gR for u in aR]
        if j == W - 1:  # and last
            aL = [gL @ u for u in aL]
            aR = [gR @ u for u in aR]
        out.append((np.array(aL), np.array(aR)))
    return out


def gate_1site(h1, tau):
    """exp(-tau h1) of a symmetric single-site operator, through its eigenbasis."""
    w, V = np.linalg.eigh(h1)
    return (V * np.exp(-tau * w)[None, :]) @ V.T


def trotter_step_product(B, lam, L, h, W, dt, compress, step):
    """One second-order Trotter step of the W-wide cylinder with product updates: the
    layers of trotter_step, each bond applied as its W gates of cylinder_product_gates
    (one compression per gate).  Philox stream of gate j of bond i in layer t of the
    step: ((3 step + t) W + j) L + i.  Returns the summed discarded weight."""
    la, lb = layers(L)
    err = 0.0
    for layer, (bonds, tau) in enumerate(((la, dt / 2), (lb, dt), (la, dt / 2))):
        gates = {i: cylinder_product_gates(i, L, h, W, tau) for i in bonds}
        for j in range(W):
            for i in bonds:
                uL, uR = gates[i][j]
                err += product_update(B, lam, i, uL, uR, compress, ((3 * step + layer) * W + j) * L + i)
    return err


def make_compressor(kind, p=10, q=2, seed=0):
    """compress(M, k, stream) -> (U, S, Vt) via Alg. RSVD or Alg. TSVD."""
    if kind == "rsvd":
        return lambda M, k, stream: rsvd(M, k, p, q, seed, stream)
    if kind == "tsvd":
        return lambda M, k, stream: tsvd(M, k)
    raise ValueError(kind)


def layers(L):
    """Bonds of layer A (i even) and layer B (i odd)."""
    return list(range(0, L - 1, 2)), list(range(1, L - 1, 2))


def chain_bond_terms(L, h, S=0.5):
    """The L - 1 bond terms of the spin-S chain."""
    return [bond_hamiltonian(i, L, h, S) for i in range(L - 1)]


def cylinder_bond_terms(L, h, W):
    """The L - 1 bond terms of the W-wide cylinder mapped onto a chain of rings."""
    return [cylinder_bond_hamiltonian(i, L, h, W) for i in range(L - 1)]


def trotter_step(B, lam, L, h, dt, compress, step, terms=None):
    """One second-order Trotter step; returns the summed discarded weight.  terms: the
    bond terms (default: the spin-1/2 chain at field h)."""
    if terms is None:
        terms = chain_bond_terms(L, h)
    la, lb = layers(L)
    err = 0.0
    for layer, (bonds, tau) in enumerate(((la, dt / 2), (lb, dt), (la, dt / 2))):
        for i in bonds:
            G = gate(terms[i], tau)
            err += bond_update(B, lam, i, G, compress, (3 * step + layer) * L + i)
    return err


def mps_energy(B, L, h, terms=None):
    """<psi|H|psi> / <psi|psi> by exact contraction of psi = B[0] B[1] ... B[L-1]."""
    if terms is None:
        terms = chain_bond_terms(L, h)
    left = [np.ones((1, 1))]
    for i in range(L):
        left.append(np.einsum("ab,asc,bsd->cd", left[i], B[i], B[i], optimize=True))
    right = [None] * (L + 1)
    right[L] = np.ones((1, 1))
    for i in range(L - 1, -1, -1):
        right[i] = np.einsum("asc,bsd,cd->ab", B[i], B[i], right[i + 1], optimize=True)
    norm = float(left[L][0, 0])
    e = 0.0
    d = B[0].shape[1]
    for i in range(L - 1):
        two = np.einsum("atb,buc->atuc", B[i], B[i + 1])
        hb = terms[i].reshape(d, d, d, d)
        htwo = np.einsum("stxy,axyc->astc", hb, two)
        e += float(np.einsum("ab,astc,bstd,cd->", left[i], htwo, two, right[i + 2], optimize=True))
    return e / norm


def mps_to_dense(B):
    """Dense state vector of a (small) MPS, site 0 as the most significant index."""
    psi = B[0].reshape(B[0].shape[1], B[0].shape[2])
    for t in B[1:]:
        psi = np.einsum("xa,asb->xsb", psi, t).reshape(-1, t.shape[2])
    return psi.reshape(-1)


def dense_chain_hamiltonian(L, h, S=0.5):
    """Spin-S chain as a dense d^L x d^L matrix, built site by site (brute force)."""
    sx, sz = spin_ops(S)
    d = sx.shape[0]

    def site_op(op, j):
        out = np.ones((1, 1))
        for t in range(L):
            out = np.kron(out, op if t == j else np.eye(d))
        return out
    H = np.zeros((d ** L, d ** L))
    for j in range(L - 1):
        H -= site_op(sz, j) @ site_op(sz, j + 1) / S ** 2
    for j in range(L):
        H -= (h / S) * site_op(sx, j)
    return H


def dense_cylinder_hamiltonian(L, h, W):
    """Cylinder of L rings of W spins, dense 2^(LW) matrix, from the single-spin terms of
    Eq. ising_cylinder (x and z exchanged): -sum Z Z around and along, -h sum X."""
    n = L * W

    def op_at(op, k):
        out = np.ones((1, 1))
        for t in range(n):
            out = np.kron(out, op if t == k else EYE2)
        return out
    H = np.zeros((2 ** n, 2 ** n))
    for i in range(L):
        for j in range(W):
            k = i * W + j
            H -= op_at(PAULI_Z, k) @ op_at(PAULI_Z, i * W + (j + 1) % W)
            if i + 1 < L:
                H -= op_at(PAULI_Z, k) @ op_at(PAULI_Z, k + W)
            H -= h * op_at(PAULI_X, k)
    return H


def dense_hamiltonian(L, h):
    """H = -sum Z_j Z_{j+1} - h sum X_j as a dense 2^L x 2^L matrix (brute force)."""
    def site_op(op, j):
        out = np.ones((1, 1))
        for s in range(L):
            out = np.kron(out, op if s == j else EYE2)
        return out
    H = np.zeros((2 ** L, 2 ** L))
    for j in range(L - 1):
        H -= site_op(PAULI_Z, j) @ site_op(PAULI_Z, j + 1)
    for j in range(L):
        H -= h * site_op(PAULI_X, j)
    return H


def exact_ground_energy_ed(L, h):
    """Lowest eigenvalue of the dense Hamiltonian (exact diagonalisation)."""
    return float(np.linalg.eigvalsh(dense_hamiltonian(L, h))[0])


def free_fermion_ground_energy(L, h, J=1.0):
    """Ground energy of the open chain from its free-fermion solution.

    After the Jordan-Wigner transformation the single-particle energies are the
    singular values of the L x L upper-bidiagonal matrix with h on the diagonal
    and J on the superdiagonal; the ground energy is minus their sum.
    """
    M = np.diag(np.full(L, float(h))) + np.diag(np.full(L - 1, float(J)), 1)
    return -float(np.sum(np.linalg.svd(M, compute_uv=False)))


def critical_ground_energy(L):
    """Closed form at h = J = 1: E0 = 1 - 1 / sin(pi / (2 (2L + 1)))."""
    return 1.0 - 1.0 / np.sin(np.pi / (2.0 * (2 * L + 1)))


def entanglement_entropy(lam_j):
    """Von Neumann entropy S_N = -sum lam^2 log lam^2 of one bond (Sec. III.C)."""
    p = np.asarray(lam_j, dtype=np.float64) ** 2
    p = p[p > 0]
    return float(-np.sum(p * np.log(p)))
