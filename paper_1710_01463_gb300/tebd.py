"""Imaginary-time TEBD driver on a device-resident MPS (Sec. III.A, III.C).

Models (Sec. III.B), with the coupling and field axes exchanged (a unitary change of
basis, same spectrum):
  * the spin-S chain of Eq. ising_chain, H = -(1/S^2) sum S^z_j S^z_{j+1} - (h/S) sum S^x_j,
    d = 2S + 1 (S = 1/2: H = -sum Z Z - h sum X with Pauli matrices);
  * the 2D cylinder of Eq. ising_cylinder with circumference W mapped onto a chain of
    rings, d = 2^W: -sum Z Z around each ring and between neighbouring rings, -h sum X.
Evolution by second-order Trotter steps exp(-dt/2 H_A) exp(-dt H_B) exp(-dt/2 H_A), layer A
holding the bonds (0,1), (2,3), ... and layer B the bonds (1,2), (3,4), ...  Each layer is
ONE call of tebd_bond_update over all of its bonds, which are independent.  Bond dimensions
are fixed at min(d^j, d^(L-j), chi); an interior site (ring) gives half of its on-site terms
to each of its two bonds, an edge site all of them.

The gates (d^2 x d^2 matrix exponentials of the bond Hamiltonians) are inputs of the bond
update and are formed once on the host.
"""
import ctypes

import numpy as np
import torch

from . import _lib
from .api import _params, _stream_handle

_X = np.array([[0.0, 1.0], [1.0, 0.0]])
_Z = np.array([[1.0, 0.0], [0.0, -1.0]])
_I = np.eye(2)


def spin_matrices(S):
    """(S^x, S^z) of spin S in the basis m = S, S-1, ..., -S: <m|S^z|m> = m and
    <m+1|S^x|m> = sqrt(S(S+1) - m(m+1)) / 2 (the standard ladder elements)."""
    d = int(round(2 * S)) + 1
    m = S - np.arange(d)
    sx = np.zeros((d, d))
    for a in range(d - 1):
        v = 0.5 * np.sqrt(S * (S + 1) - m[a + 1] * (m[a + 1] + 1))
        sx[a, a + 1] = sx[a + 1, a] = v
    return sx, np.diag(m)


def bond_hamiltonian(i, L, h, S=0.5):
    """Two-site term of bond (i, i+1) of the spin-S chain, d^2 x d^2 on (s_i, s_{i+1})."""
    sx, sz = spin_matrices(S)
    one = np.eye(sx.shape[0])
    fl = 1.0 if i == 0 else 0.5
    fr = 1.0 if i + 1 == L - 1 else 0.5
    return -np.kron(sz, sz) / S ** 2 - (h / S) * (fl * np.kron(sx, one) + fr * np.kron(one, sx))


def ring_bond_hamiltonian(i, L, h, W):
    """Two-site term of rings (i, i+1) of the W-wide cylinder, 4^W x 4^W."""
    def on(op, j):
        out = np.ones((1, 1))
        for t in range(W):
            out = np.kron(out, op if t == j else _I)
        return out
    Z = [on(_Z, j) for j in range(W)]
    X = [on(_X, j) for j in range(W)]
    onsite = -sum(Z[j] @ Z[(j + 1) % W] for j in range(W)) - h * sum(X)
    one = np.eye(2 ** W)
    fl = 1.0 if i == 0 else 0.5
    fr = 1.0 if i + 1 == L - 1 else 0.5
    inter = -sum(np.kron(Z[j], Z[j]) for j in range(W))
    return inter + fl * np.kron(onsite, one) + fr * np.kron(one, onsite)


def ring_product_gates(i, L, h, W, tau):
    """Bond (i, i+1) of the W-wide cylinder as W gates of K = 2 Kronecker terms (the
    product update, Sec. III.A P): exp(-tau A/2) prod_j exp(-tau C_j) exp(-tau A/2), where
    C_j = -Z_{i,j} Z_{i+1,j} are the bond's commuting couplings, exp(-tau C_j) =
    cosh(tau) 1 (x) 1 + sinh(tau) Z_j (x) Z_j, and A is the bond's share of the two rings'
    own terms (exp(-tau A/2) = gL (x) gR, folded into the first and last coupling).
    Returns W arrays (2, 2, d, d): [uL, uR] of K = 2 operators each, in the order applied."""
    def on(op, j):
        out = np.ones((1, 1))
        for t in range(W):
            out = np.kron(out, op if t == j else _I)
        return out
    Z = [on(_Z, j) for j in range(W)]
    X = [on(_X, j) for j in range(W)]
    onsite = -sum(Z[j] @ Z[(j + 1) % W] for j in range(W)) - h * sum(X)
    fl = 1.0 if i == 0 else 0.5
    fr = 1.0 if i + 1 == L - 1 else 0.5
    gL = bond_gate(fl * onsite, tau / 2)
    gR = bond_gate(fr * onsite, tau / 2)
    one = np.eye(2 ** W)
    out = []
    for j in range(W):
        uL = [np.cosh(tau) * one, np.sinh(tau) * Z[j]]
        uR = [one, Z[j]]
        if j == 0:
            uL, uR = [u @ gL for u in uL], [u @ gR for u in uR]
        if j == W - 1:
            uL, uR = [gL @ u for u in uL], [gR @ u for u in uR]
        out.append(np.array([uL, uR]))
    return out


# Imaginary-time schedules, as (dt, steps) stages.  EARLY: a few coarse steps from the
# product state, which leave the decaying spectra of a run in progress.  GROUND: the
# paper's protocol of reducing dt in stages (Sec. III.C); on the open critical Ising
# chain at L = 64, chi = 128 it ends within 1e-6 of the free-fermion ground energy.
SCHEDULE_EARLY = ((0.1, 20),)
SCHEDULE_GROUND = ((0.1, 700), (0.05, 500), (0.02, 250))


def bond_gate(hb, tau):
    """exp(-tau h_b) through the eigenbasis of the symmetric h_b."""
    w, V = np.linalg.eigh(hb)
    return (V * np.exp(-tau * w)[None, :]) @ V.T


class TebdChain:
    """MPS of an L-site chain with right-canonical tensors B[i] and Schmidt values lam[j]."""

    def __init__(self, L, chi, h=1.0, p=10, q=2, seed=0, device="cuda", max_sweeps=0, simt=False, S=0.5, W=None,
                 update="block", tsvd=False):
        """S: spin of the chain (d = 2S + 1); W: circumference of the 2D cylinder (d = 2^W;
        overrides S).  update: "block" (one d^2 x d^2 gate per bond, tebd_bond_update) or,
        for the cylinder, "product" (each bond as W gates of K = 2 Kronecker terms,
        tebd_product_update: W compressions of a rank <= 2 chi product per bond).
        tsvd: compress by Alg. TSVD on the same engine (RSVD_FLAG_FULL_SVD: the full Jacobi
        SVD of every two-site matrix, then truncation) instead of Alg. RSVD (block update)."""
        if L < 2:
            raise ValueError("L >= 2 required")
        if update not in ("block", "product") or (update == "product" and not W):
            raise ValueError("update is 'block', or 'product' for the cylinder")
        if tsvd and update != "block":
            raise ValueError("tsvd compresses the block update only")
        self.update = update
        self.flags = _lib.RSVD_FLAG_FULL_SVD if tsvd else 0
        self.S, self.W = S, W
        d = 2 ** W if W else int(round(2 * S)) + 1
        self.L, self.d, self.chi, self.h = L, d, chi, h
        self.p, self.q, self.seed, self.max_sweeps, self.simt = p, q, seed, max_sweeps, simt
        self.device = torch.device(device)
        d = self.d
        self.D = [int(min(d ** min(j, L - j), chi)) for j in range(L + 1)]
        self.tensor_stride = max(self.D[i] * d * self.D[i + 1] for i in range(L))
        self.lam_stride = max(self.D)
        self.B = torch.zeros((L, self.tensor_stride), dtype=torch.float64, device=self.device)
        self.lam = torch.zeros((L + 1, self.lam_stride), dtype=torch.float64, device=self.device)
        self.layers = [list(range(0, L - 1, 2)), list(range(1, L - 1, 2))]
        self.D_arr = _lib.int_array(self.D)
        nb = max(len(x) for x in self.layers)
        lib = _lib.load()
        par = _params(1, p, q, _lib.RSVD_F64, seed, 0, 0, simt, self.flags)
        sz = ctypes.c_size_t(0)
        if update == "product":
            _lib.check(lib.tebd_product_workspace_size(L, d, self.D_arr, nb, 2, ctypes.byref(par), ctypes.byref(sz)),
                       "tebd_product_workspace_size")
        else:
            _lib.check(lib.tebd_workspace_size(L, d, self.D_arr, nb, ctypes.byref(par), ctypes.byref(sz)),
                       "tebd_workspace_size")
        self.work = torch.empty(max(sz.value, 1), dtype=torch.uint8, device=self.device)
        nsub = W if update == "product" else 1  # compressions per bond and layer
        self.trunc_err = torch.zeros((3, nsub, nb), dtype=torch.float64, device=self.device)
        self.info = torch.zeros((3, nsub, nb, _lib.INFO_INTS), dtype=torch.int32, device=self.device)
        self.bond_arr = [_lib.int_array(b) for b in self.layers]
        self.dt = None

    def set_dt(self, dt):
        """Form the gates of the three layers of one Trotter step."""
        self.dt = float(dt)
        gates = []
        if self.update == "product":
            # gates[t][j]: (nb, 2, 2, d, d) -> uL = [:, 0], uR = [:, 1], each (nb, K, d, d)
            for layer, tau in ((0, dt / 2), (1, dt), (0, dt / 2)):
                per = [ring_product_gates(i, self.L, self.h, self.W, tau) for i in self.layers[layer]]
                gl = []
                for j in range(self.W):
                    g = np.stack([pb[j] for pb in per]) if per else np.zeros((0, 2, 2, self.d, self.d))
                    gl.append((torch.tensor(np.ascontiguousarray(g[:, 0]), dtype=torch.float64, device=self.device),
                               torch.tensor(np.ascontiguousarray(g[:, 1]), dtype=torch.float64, device=self.device)))
                gates.append(gl)
            self.gates = gates
            return
        for layer, tau in ((0, dt / 2), (1, dt), (0, dt / 2)):
            g = [bond_gate(self.bond_term(i), tau).ravel() for i in self.layers[layer]]
            gates.append(torch.tensor(np.stack(g), dtype=torch.float64, device=self.device))
        self.gates = gates

    def bond_term(self, i):
        """The Hamiltonian term of bond (i, i+1) of this chain's model."""
        if self.W:
            return ring_bond_hamiltonian(i, self.L, self.h, self.W)
        return bond_hamiltonian(i, self.L, self.h, self.S)

    def set_product_state(self, vectors):
        """B[i][0, :, 0] = vectors[i] / |vectors[i]|, lam[j] = (1, 0, ...)."""
        v = np.asarray(vectors, dtype=np.float64)
        self.B.zero_()
        self.lam.zero_()
        host = np.zeros((self.L, self.tensor_stride))
        for i in range(self.L):
            t = np.zeros((self.D[i], self.d, self.D[i + 1]))
            t[0, :, 0] = v[i] / np.linalg.norm(v[i])
            host[i, : t.size] = t.ravel()
        self.B.copy_(torch.from_numpy(host))
        lam = np.zeros((self.L + 1, self.lam_stride))
        lam[:, 0] = 1.0
        self.lam.copy_(torch.from_numpy(lam))

    def step(self, step_index, stream=None):
        """One second-order Trotter step (three layers), asynchronous."""
        lib = _lib.load()
        sh = _stream_handle(stream)
        if self.update == "product":
            self._step_product(step_index, lib, sh)
            return
        for j, layer in enumerate((0, 1, 0)):
            bonds = self.layers[layer]
            if not bonds:
                continue
            par = _params(1, self.p, self.q, _lib.RSVD_F64, self.seed, (3 * step_index + j) * self.L,
                          self.max_sweeps, self.simt, self.flags)
            rc = lib.tebd_bond_update(self.L, self.d, self.D_arr, len(bonds), self.bond_arr[layer],
                                      ctypes.c_void_p(self.B.data_ptr()), self.tensor_stride,
                                      ctypes.c_void_p(self.lam.data_ptr()), self.lam_stride,
                                      ctypes.c_void_p(self.gates[j].data_ptr()), ctypes.byref(par),
                                      ctypes.c_void_p(self.trunc_err[j, 0].data_ptr()),
                                      ctypes.c_void_p(self.work.data_ptr()), ctypes.c_size_t(self.work.numel()),
                                      ctypes.c_void_p(self.info[j, 0].data_ptr()), sh)
            _lib.check(rc, "tebd_bond_update")

    def _step_product(self, step_index, lib, sh):
        """Product-update Trotter step: per layer, the W coupling gates one after another,
        each ONE call of tebd_product_update over the layer's bonds.  Philox stream of gate j
        of bond i in layer t: ((3 step + t) W + j) L + i."""
        for t, layer in enumerate((0, 1, 0)):
            bonds = self.layers[layer]
            if not bonds:
                continue
            for j in range(self.W):
                uL, uR = self.gates[t][j]
                par = _params(1, self.p, self.q, _lib.RSVD_F64, self.seed, ((3 * step_index + t) * self.W + j) * self.L,
                              self.max_sweeps, self.simt)
                rc = lib.tebd_product_update(self.L, self.d, self.D_arr, len(bonds), self.bond_arr[layer],
                                             ctypes.c_void_p(self.B.data_ptr()), ctypes.c_size_t(self.tensor_stride),
                                             ctypes.c_void_p(self.lam.data_ptr()), ctypes.c_size_t(self.lam_stride), 2,
                                             ctypes.c_void_p(uL.data_ptr()), ctypes.c_void_p(uR.data_ptr()),
                                             ctypes.byref(par), ctypes.c_void_p(self.trunc_err[t, j].data_ptr()),
                                             ctypes.c_void_p(self.work.data_ptr()), ctypes.c_size_t(self.work.numel()),
                                             ctypes.c_void_p(self.info[t, j].data_ptr()), sh)
                _lib.check(rc, "tebd_product_update")

    def evolve(self, schedule, first_step=0, stream=None):
        """Run the (dt, steps) stages of an imaginary-time schedule (asynchronous);
        returns the index of the next step."""
        s = first_step
        for dt, n in schedule:
            self.set_dt(dt)
            for _ in range(n):
                self.step(s, stream)
                s += 1
        return s

    def tensors(self):
        """Host copies of the B tensors, shaped (D[i], d, D[i+1])."""
        host = self.B.cpu().numpy()
        return [host[i, : self.D[i] * self.d * self.D[i + 1]].reshape(self.D[i], self.d, self.D[i + 1]).copy()
                for i in range(self.L)]

    def schmidt_values(self):
        host = self.lam.cpu().numpy()
        return [host[j, : self.D[j]].copy() for j in range(self.L + 1)]

    def state_to_host(self):
        return self.B.cpu().numpy().copy(), self.lam.cpu().numpy().copy()

    def state_from_host(self, B, lam):
        self.B.copy_(torch.from_numpy(np.asarray(B)))
        self.lam.copy_(torch.from_numpy(np.asarray(lam)))

    def save(self, path, step):
        """Checkpoint: B tensors, Schmidt values, bond dimensions, step and dt (.npz)."""
        B, lam = self.state_to_host()
        np.savez(path, B=B, lam=lam, D=np.asarray(self.D), L=self.L, chi=self.chi, h=self.h, d=self.d,
                 S=float(self.S), W=int(self.W or 0), step=int(step), dt=float(self.dt if self.dt is not None else 0.0))

    def load(self, path):
        """Restore a checkpoint written by save(); returns the step to continue from."""
        z = np.load(path)
        if int(z["L"]) != self.L or int(z["chi"]) != self.chi or list(z["D"]) != self.D:
            raise ValueError("checkpoint does not match this chain")
        if "d" in z and (int(z["d"]) != self.d or float(z["S"]) != float(self.S) or int(z["W"]) != int(self.W or 0)):
            raise ValueError("checkpoint is of another model")
        self.state_from_host(z["B"], z["lam"])
        if float(z["dt"]) > 0:
            self.set_dt(float(z["dt"]))
        return int(z["step"])
