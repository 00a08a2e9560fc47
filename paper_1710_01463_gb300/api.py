"""Python entry points of librsvd with the same names as the C ABI.

PyTorch provides device memory and the current CUDA stream; every step of the
computation runs in librsvd's kernels.  Inputs must be CUDA tensors; there is
no CPU path.
"""
import ctypes

import torch

from . import _lib

_DTYPE_PREC = {torch.float64: _lib.RSVD_F64, torch.float32: _lib.RSVD_F32, torch.bfloat16: _lib.RSVD_BF16}


def _prec_of(A, tf32=False):
    if tf32:
        if A.dtype != torch.float32:
            raise ValueError("TF32 products need a float32 A")
        return _lib.RSVD_TF32
    return _DTYPE_PREC[A.dtype]


def _out_dtype(A):
    return torch.float64 if A.dtype == torch.float64 else torch.float32


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _params(k, p, q, prec, seed, stream, max_sweeps=0, simt=False, flags=0):
    """rsvd_params; simt=True sets RSVD_FLAG_F64_SIMT (FP64 products with A on FP64 FMAs
    instead of the tensor cores by exact slicing); flags adds further RSVD_FLAG_* bits."""
    return _lib.RsvdParams(int(k), int(p), int(q), int(prec), int(seed) & ((1 << 64) - 1),
                           int(stream) & ((1 << 64) - 1), int(max_sweeps),
                           (_lib.RSVD_FLAG_F64_SIMT if simt else 0) | int(flags))


def _require_cuda(*ts):
    for t in ts:
        if not (isinstance(t, torch.Tensor) and t.is_cuda):
            raise ValueError("librsvd works on CUDA tensors only")


def info_dicts(info):
    """Decode a (batch, INFO_INTS) int32 info tensor into a list of dicts."""
    rows = info.view(-1, _lib.INFO_INTS).cpu().tolist()
    keys = ("status", "path", "chol_fallbacks", "jacobi_sweeps", "l", "rotations", "qr_columns", "qr_kflop",
            "jacobi_pairs", "cg_iterations")
    return [dict(zip(keys, r)) for r in rows]


def rsvd_gaussian(n, l, seed, stream=0, device="cuda", out=None):
    """Omega (n x l, FP64) of Alg. RSVD step 1; see include/rsvd.h."""
    lib = _lib.load()
    if out is None:
        out = torch.empty((n, l), dtype=torch.float64, device=device)
    _require_cuda(out)
    _lib.check(lib.rsvd_gaussian(int(n), int(l), int(seed), int(stream), ctypes.c_void_p(out.data_ptr()),
                                 int(out.stride(0)), _stream_handle()), "rsvd_gaussian")
    return out


def rsvd_workspace_size(m, n, k, p=8, q=2, dtype=torch.float64):
    lib = _lib.load()
    par = _params(k, p, q, _DTYPE_PREC[dtype], 0, 0)
    sz = ctypes.c_size_t(0)
    _lib.check(lib.rsvd_workspace_size(int(m), int(n), ctypes.byref(par), ctypes.byref(sz)), "rsvd_workspace_size")
    return sz.value


def rsvd_truncate(A, k, p=8, q=2, seed=0, stream=0, max_sweeps=0, work=None, tf32=False, simt=False, flags=0):
    """Rank-k RSVD of one matrix: returns (U, S, Vt, info) as CUDA tensors.

    A float64 -> FP64 products (tensor cores by exact slicing where m, n <= 1024, l <= 256,
    unless simt=True); float32 -> FP32 (tf32=True: TF32 tensor cores); bfloat16 -> BF16
    tensor cores.  U and Vt are float64 for float64 A, else float32.
    """
    lib = _lib.load()
    _require_cuda(A)
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a row-major 2-D tensor")
    prec = _prec_of(A, tf32)
    m, n = A.shape
    par = _params(k, p, q, prec, seed, stream, max_sweeps, simt, flags)
    sz = ctypes.c_size_t(0)
    _lib.check(lib.rsvd_workspace_size(m, n, ctypes.byref(par), ctypes.byref(sz)), "rsvd_workspace_size")
    if work is None or work.numel() < sz.value:
        work = torch.empty(max(sz.value, 1), dtype=torch.uint8, device=A.device)
    U = torch.empty((m, k), dtype=_out_dtype(A), device=A.device)
    S = torch.empty((k,), dtype=torch.float64, device=A.device)
    Vt = torch.empty((k, n), dtype=_out_dtype(A), device=A.device)
    info = torch.zeros((1, _lib.INFO_INTS), dtype=torch.int32, device=A.device)
    rc = lib.rsvd_truncate(m, n, ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.byref(par),
                           ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(U.data_ptr()), U.stride(0),
                           ctypes.c_void_p(Vt.data_ptr()), Vt.stride(0), ctypes.c_void_p(work.data_ptr()),
                           work.numel(), ctypes.c_void_p(info.data_ptr()), _stream_handle())
    _lib.check(rc, "rsvd_truncate")
    return U, S, Vt, info


def rsvd_truncate_complex(A, k, p=8, q=2, seed=0, stream=0, max_sweeps=0, work=None, flags=0):
    """Rank-k RSVD of a complex matrix (rsvd_truncate_complex): A a complex128 (FP64) or
    complex64 (FP32) CUDA tensor, row-major.  Returns (U, S, Vh, info): U m x k and Vh
    k x n complex (Vh = V^H), S float64."""
    lib = _lib.load()
    _require_cuda(A)
    if A.dim() != 2 or A.stride(1) != 1 or A.dtype not in (torch.complex128, torch.complex64):
        raise ValueError("A must be a row-major complex128 or complex64 2-D tensor")
    prec = _lib.RSVD_F64 if A.dtype == torch.complex128 else _lib.RSVD_F32
    m, n = A.shape
    par = _params(k, p, q, prec, seed, stream, max_sweeps, False, flags)
    sz = ctypes.c_size_t(0)
    _lib.check(lib.rsvd_complex_workspace_size(m, n, ctypes.byref(par), ctypes.byref(sz)),
               "rsvd_complex_workspace_size")
    if work is None or work.numel() < sz.value:
        work = torch.empty(max(sz.value, 1), dtype=torch.uint8, device=A.device)
    U = torch.empty((m, k), dtype=A.dtype, device=A.device)
    S = torch.empty((k,), dtype=torch.float64, device=A.device)
    Vh = torch.empty((k, n), dtype=A.dtype, device=A.device)
    info = torch.zeros((1, _lib.INFO_INTS), dtype=torch.int32, device=A.device)
    rc = lib.rsvd_truncate_complex(m, n, ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.byref(par),
                                   ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(U.data_ptr()), U.stride(0),
                                   ctypes.c_void_p(Vh.data_ptr()), Vh.stride(0), ctypes.c_void_p(work.data_ptr()),
                                   ctypes.c_size_t(work.numel()), ctypes.c_void_p(info.data_ptr()), _stream_handle())
    _lib.check(rc, "rsvd_truncate_complex")
    return U, S, Vh, info


def rsvd_truncate_factored(X, Y, k, p=8, q=2, seed=0, stream=0, max_sweeps=0, work=None):
    """Rank-k RSVD of A = X Y without forming A (rsvd_truncate_factored): X (m x r) and Y
    (r x n) float64 or float32 CUDA tensors.  Returns (U, S, Vt, info)."""
    lib = _lib.load()
    _require_cuda(X, Y)
    if X.dim() != 2 or Y.dim() != 2 or X.stride(1) != 1 or Y.stride(1) != 1 or X.shape[1] != Y.shape[0]:
        raise ValueError("X (m x r) and Y (r x n) must be row-major with matching r")
    if X.dtype != Y.dtype or X.dtype not in (torch.float64, torch.float32):
        raise ValueError("X and Y must both be float64 or both float32")
    m, r = X.shape
    n = Y.shape[1]
    par = _params(k, p, q, _DTYPE_PREC[X.dtype], seed, stream, max_sweeps)
    sz = ctypes.c_size_t(0)
    _lib.check(lib.rsvd_factored_workspace_size(m, r, n, ctypes.byref(par), ctypes.byref(sz)),
               "rsvd_factored_workspace_size")
    if work is None or work.numel() < sz.value:
        work = torch.empty(max(sz.value, 1), dtype=torch.uint8, device=X.device)
    U = torch.empty((m, k), dtype=X.dtype, device=X.device)
    S = torch.empty((k,), dtype=torch.float64, device=X.device)
    Vt = torch.empty((k, n), dtype=X.dtype, device=X.device)
    info = torch.zeros((1, _lib.INFO_INTS), dtype=torch.int32, device=X.device)
    rc = lib.rsvd_truncate_factored(m, r, n, ctypes.c_void_p(X.data_ptr()), X.stride(0), ctypes.c_void_p(Y.data_ptr()),
                                    Y.stride(0), ctypes.byref(par), ctypes.c_void_p(S.data_ptr()),
                                    ctypes.c_void_p(U.data_ptr()), U.stride(0), ctypes.c_void_p(Vt.data_ptr()),
                                    Vt.stride(0), ctypes.c_void_p(work.data_ptr()), ctypes.c_size_t(work.numel()),
                                    ctypes.c_void_p(info.data_ptr()), _stream_handle())
    _lib.check(rc, "rsvd_truncate_factored")
    return U, S, Vt, info


def rsvd_truncate_tol(A, eps, k0, k_max, p=8, q=2, seed=0, stream=0, max_sweeps=0, work=None):
    """Fixed-error RSVD (rsvd_truncate_tol): the smallest rank k <= k_max with
    ||A - U diag(S) Vt||_F <= eps ||A||_F, trial ranks k0, 2 k0, ...; A a float64 CUDA
    tensor.  Returns (U, S, Vt, err, info) cut to the chosen rank."""
    lib = _lib.load()
    _require_cuda(A)
    if A.dim() != 2 or A.stride(1) != 1 or A.dtype != torch.float64:
        raise ValueError("A must be a row-major float64 2-D tensor")
    m, n = A.shape
    cap = min(int(k_max), m, n)
    par = _params(k0, p, q, _lib.RSVD_F64, seed, stream, max_sweeps)
    sz = ctypes.c_size_t(0)
    _lib.check(lib.rsvd_tol_workspace_size(m, n, int(k_max), ctypes.byref(par), ctypes.byref(sz)),
               "rsvd_tol_workspace_size")
    if work is None or work.numel() < sz.value:
        work = torch.empty(max(sz.value, 1), dtype=torch.uint8, device=A.device)
    U = torch.empty((m, cap), dtype=torch.float64, device=A.device)
    S = torch.empty((cap,), dtype=torch.float64, device=A.device)
    Vt = torch.empty((cap, n), dtype=torch.float64, device=A.device)
    info = torch.zeros((1, _lib.INFO_INTS), dtype=torch.int32, device=A.device)
    k = ctypes.c_int(0)
    err = ctypes.c_double(0.0)
    rc = lib.rsvd_truncate_tol(m, n, ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_double(eps), int(k_max),
                               ctypes.byref(par), ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(U.data_ptr()),
                               U.stride(0), ctypes.c_void_p(Vt.data_ptr()), Vt.stride(0), ctypes.byref(k),
                               ctypes.byref(err), ctypes.c_void_p(work.data_ptr()), ctypes.c_size_t(work.numel()),
                               ctypes.c_void_p(info.data_ptr()), _stream_handle())
    _lib.check(rc, "rsvd_truncate_tol")
    kk = k.value
    return U[:, :kk], S[:kk], Vt[:kk], err.value, info


class BatchedPlan:
    """Preallocated outputs and workspace of rsvd_truncate_batched for fixed shapes."""

    def __init__(self, shapes, ks, p=8, q=2, seed=0, stream=0, dtype=torch.float64, device="cuda",
                 max_sweeps=0, chi_global=0, tf32=False, simt=False, flags=0):
        lib = _lib.load()
        self.shapes = [(int(m), int(n)) for m, n in shapes]
        self.ks = [int(k) for k in ks]
        self.dtype = dtype
        self.chi_global = int(chi_global)
        prec = _lib.RSVD_TF32 if tf32 else _DTYPE_PREC[dtype]
        out = torch.float64 if dtype == torch.float64 else torch.float32
        self.par = _params(self.ks[0], p, q, prec, seed, stream, max_sweeps, simt, flags)
        B = len(self.shapes)
        self.m_arr = _lib.int_array([s[0] for s in self.shapes])
        self.n_arr = _lib.int_array([s[1] for s in self.shapes])
        self.k_arr = _lib.int_array(self.ks)
        sz = ctypes.c_size_t(0)
        _lib.check(lib.rsvd_batched_workspace_size(B, self.m_arr, self.n_arr, self.k_arr, ctypes.byref(self.par),
                                                   ctypes.byref(sz)), "rsvd_batched_workspace_size")
        self.work = torch.empty(max(sz.value, 1), dtype=torch.uint8, device=device)
        self.U = [torch.empty((m, k), dtype=out, device=device) for (m, _), k in zip(self.shapes, self.ks)]
        self.S = [torch.empty((k,), dtype=torch.float64, device=device) for k in self.ks]
        self.Vt = [torch.empty((k, n), dtype=out, device=device) for (_, n), k in zip(self.shapes, self.ks)]
        self.info = torch.zeros((B, _lib.INFO_INTS), dtype=torch.int32, device=device)
        self.k_out = torch.zeros((B,), dtype=torch.int32, device=device)
        self.S_ptr = _lib.ptr_array([t.data_ptr() for t in self.S])
        self.U_ptr = _lib.ptr_array([t.data_ptr() for t in self.U])
        self.V_ptr = _lib.ptr_array([t.data_ptr() for t in self.Vt])
        self.ldu = _lib.int_array([t.stride(0) for t in self.U])
        self.ldv = _lib.int_array([t.stride(0) for t in self.Vt])

    def run(self, As, stream=None):
        lib = _lib.load()
        if len(As) != len(self.shapes):
            raise ValueError("batch size mismatch")
        for A, (m, n) in zip(As, self.shapes):
            _require_cuda(A)
            if tuple(A.shape) != (m, n) or A.dtype != self.dtype or A.stride(1) != 1:
                raise ValueError("matrix shape / dtype / layout mismatch")
        A_ptr = _lib.ptr_array([A.data_ptr() for A in As])
        lda = _lib.int_array([A.stride(0) for A in As])
        rc = lib.rsvd_truncate_batched(len(As), self.m_arr, self.n_arr, A_ptr, lda, self.k_arr, ctypes.byref(self.par),
                                       self.S_ptr, self.U_ptr, self.ldu, self.V_ptr, self.ldv, self.chi_global,
                                       ctypes.c_void_p(self.k_out.data_ptr()), ctypes.c_void_p(self.work.data_ptr()),
                                       self.work.numel(), ctypes.c_void_p(self.info.data_ptr()),
                                       _stream_handle(stream))
        _lib.check(rc, "rsvd_truncate_batched")
        return self.U, self.S, self.Vt


def rsvd_truncate_batched(As, ks, p=8, q=2, seed=0, stream=0, chi_global=0, max_sweeps=0, tf32=False, flags=0):
    """Alg. RSVD on a list of matrices; returns (U list, S list, Vt list, k_out, info)."""
    plan = BatchedPlan([tuple(A.shape) for A in As], ks, p, q, seed, stream, As[0].dtype, As[0].device,
                       max_sweeps, chi_global, tf32, flags=flags)
    U, S, Vt = plan.run(As)
    return U, S, Vt, plan.k_out, plan.info


class AdaptiveSectorsPlan:
    """Preallocated outputs and workspace of rsvd_truncate_sectors_adaptive for fixed block
    shapes: block-wise RSVD with the global top-chi cut and per-block trial ranks grown
    until no block is saturated.  `ranks` carries the last trial ranks into the next run
    (estimates from the previous iteration)."""

    def __init__(self, shapes, chi, ranks0, p=8, q=2, seed=0, stream=0, dtype=torch.float64, device="cuda",
                 max_sweeps=0, device_rounds=False):
        """device_rounds=True: rsvd_truncate_sectors_adaptive_device - the rounds are decided on
        the device (no host synchronisation: the run can be captured in a CUDA graph), every
        run starts from ranks0, and the final ranks and the rounds stay on the device
        (k_final, rounds_dev)."""
        lib = _lib.load()
        self.device_rounds = bool(device_rounds)
        self.ranks0 = [int(k) for k in ranks0]
        self.shapes = [(int(m), int(n)) for m, n in shapes]
        self.chi = int(chi)
        self.dtype = dtype
        B = len(self.shapes)
        caps = [min(self.chi, m, n) for m, n in self.shapes]
        self.ranks = [max(1, min(int(k), c)) for k, c in zip(ranks0, caps)]
        self.par = _params(1, p, q, _DTYPE_PREC[dtype], seed, stream, max_sweeps)
        self.m_arr = _lib.int_array([s[0] for s in self.shapes])
        self.n_arr = _lib.int_array([s[1] for s in self.shapes])
        sz = ctypes.c_size_t(0)
        _lib.check(lib.rsvd_sectors_adaptive_workspace_size(B, self.m_arr, self.n_arr, self.chi, ctypes.byref(self.par),
                                                            ctypes.byref(sz)), "rsvd_sectors_adaptive_workspace_size")
        self.work = torch.empty(max(sz.value, 1), dtype=torch.uint8, device=device)
        out = torch.float64 if dtype == torch.float64 else torch.float32
        self.U = [torch.empty((m, c), dtype=out, device=device) for (m, _), c in zip(self.shapes, caps)]
        self.S = [torch.empty((c,), dtype=torch.float64, device=device) for c in caps]
        self.Vt = [torch.empty((c, n), dtype=out, device=device) for (_, n), c in zip(self.shapes, caps)]
        self.info = torch.zeros((B, _lib.INFO_INTS), dtype=torch.int32, device=device)
        self.k_out = torch.zeros((B,), dtype=torch.int32, device=device)
        self.S_ptr = _lib.ptr_array([t.data_ptr() for t in self.S])
        self.U_ptr = _lib.ptr_array([t.data_ptr() for t in self.U])
        self.V_ptr = _lib.ptr_array([t.data_ptr() for t in self.Vt])
        self.ldu = _lib.int_array([t.stride(0) for t in self.U])
        self.ldv = _lib.int_array([t.stride(0) for t in self.Vt])
        self.rounds = 0
        self.k_final = torch.zeros((B,), dtype=torch.int32, device=device)
        self.rounds_dev = torch.zeros((1,), dtype=torch.int32, device=device)

    def run(self, As, stream=None):
        lib = _lib.load()
        for A, (m, n) in zip(As, self.shapes):
            _require_cuda(A)
            if tuple(A.shape) != (m, n) or A.dtype != self.dtype or A.stride(1) != 1:
                raise ValueError("block shape / dtype / layout mismatch")
        A_ptr = _lib.ptr_array([A.data_ptr() for A in As])
        lda = _lib.int_array([A.stride(0) for A in As])
        if self.device_rounds:
            caps = [min(self.chi, m, n) for m, n in self.shapes]
            k0 = _lib.int_array([max(1, min(k, c)) for k, c in zip(self.ranks0, caps)])
            rc = lib.rsvd_truncate_sectors_adaptive_device(
                len(As), self.m_arr, self.n_arr, A_ptr, lda, k0, ctypes.byref(self.par), self.chi, self.S_ptr,
                self.U_ptr, self.ldu, self.V_ptr, self.ldv, ctypes.c_void_p(self.k_out.data_ptr()),
                ctypes.c_void_p(self.k_final.data_ptr()), ctypes.c_void_p(self.rounds_dev.data_ptr()),
                ctypes.c_void_p(self.work.data_ptr()), ctypes.c_size_t(self.work.numel()),
                ctypes.c_void_p(self.info.data_ptr()), _stream_handle(stream))
            _lib.check(rc, "rsvd_truncate_sectors_adaptive_device")
            return self.U, self.S, self.Vt, self.k_out
        kt = _lib.int_array(self.ranks)
        rounds = ctypes.c_int(0)
        rc = lib.rsvd_truncate_sectors_adaptive(len(As), self.m_arr, self.n_arr, A_ptr, lda, kt, ctypes.byref(self.par),
                                                self.chi, self.S_ptr, self.U_ptr, self.ldu, self.V_ptr, self.ldv,
                                                ctypes.c_void_p(self.k_out.data_ptr()), ctypes.byref(rounds),
                                                ctypes.c_void_p(self.work.data_ptr()), ctypes.c_size_t(self.work.numel()),
                                                ctypes.c_void_p(self.info.data_ptr()), _stream_handle(stream))
        _lib.check(rc, "rsvd_truncate_sectors_adaptive")
        self.ranks = [int(kt[i]) for i in range(len(As))]
        self.rounds = rounds.value
        return self.U, self.S, self.Vt, self.k_out


def rsvd_truncate_backward_batched(As, Us, Ss, Vts, Ubars=None, Sbars=None, Vtbars=None, max_iter=300, tol=None):
    """Abar for each matrix from its factors and the cotangents (see include/rsvd.h)."""
    lib = _lib.load()
    B = len(As)
    dtype = As[0].dtype
    prec = _DTYPE_PREC[dtype]
    if tol is None:
        tol = 1e-12 if dtype == torch.float64 else 1e-6
    ms = [A.shape[0] for A in As]
    ns = [A.shape[1] for A in As]
    ks = [S.numel() for S in Ss]
    m_a, n_a, k_a = _lib.int_array(ms), _lib.int_array(ns), _lib.int_array(ks)
    sz = ctypes.c_size_t(0)
    _lib.check(lib.rsvd_backward_workspace_size(B, m_a, n_a, k_a, prec, ctypes.byref(sz)), "rsvd_backward_workspace_size")
    dev = As[0].device
    work = torch.empty(max(sz.value, 1), dtype=torch.uint8, device=dev)
    Abars = [torch.empty_like(A) for A in As]
    info = torch.zeros((B, _lib.INFO_INTS), dtype=torch.int32, device=dev)
    for t in list(As) + list(Us) + list(Vts):
        _require_cuda(t)
        if t.dtype != dtype or t.stride(1) != 1:
            raise ValueError("factors must share the dtype of A and be row-major")

    def arr(ts):
        return None if ts is None else _lib.ptr_array([t.data_ptr() for t in ts])

    def lds(ts):
        return None if ts is None else _lib.int_array([t.stride(0) for t in ts])

    rc = lib.rsvd_truncate_backward_batched(
        B, m_a, n_a, k_a, prec, arr(As), lds(As), arr(Ss), arr(Us), lds(Us), arr(Vts), lds(Vts),
        arr(Ubars), lds(Ubars), arr(Sbars), arr(Vtbars), lds(Vtbars), arr(Abars), lds(Abars),
        int(max_iter), float(tol), ctypes.c_void_p(work.data_ptr()), work.numel(),
        ctypes.c_void_p(info.data_ptr()), _stream_handle())
    _lib.check(rc, "rsvd_truncate_backward_batched")
    return Abars, info


def check_info(info, what):
    """Read the device status records of a call (synchronises the stream): raise on an
    error status (negative: non-finite input, a timed-out device wait), warn on a warning
    (the Jacobi sweep cap, an unconverged conjugate-gradient column)."""
    import warnings
    for d in info_dicts(info):
        st = d["status"]
        if st < 0:
            raise RuntimeError(f"{what}: device status {st} ({_lib.status_string(st)})")
        if st > 0:
            warnings.warn(f"{what}: device status {st} ({_lib.status_string(st)})", RuntimeWarning, stacklevel=3)


class RSVDTrunc(torch.autograd.Function):
    """(U, S, Vt) = rank-k RSVD of A (forward: rsvd_truncate), with the
    derivative of the truncated factorization (backward: the library's
    rsvd_truncate_backward_batched).  Both passes read their device status
    records: an error status raises, a warning (Jacobi sweep cap, unconverged
    conjugate gradients; max_iter caps the latter) is issued as a RuntimeWarning."""

    @staticmethod
    def forward(ctx, A, k, p=8, q=2, seed=0, stream=0, max_iter=300):
        U, S, Vt, info = rsvd_truncate(A.contiguous(), k, p, q, seed, stream)
        check_info(info, "rsvd_truncate")
        ctx.save_for_backward(A.contiguous(), U, S, Vt)
        ctx.max_iter = int(max_iter)
        return U, S, Vt

    @staticmethod
    def backward(ctx, gU, gS, gVt):
        A, U, S, Vt = ctx.saved_tensors
        Ub = None if gU is None else [gU.contiguous().to(A.dtype)]
        Sb = None if gS is None else [gS.contiguous().to(torch.float64)]
        Vb = None if gVt is None else [gVt.contiguous().to(A.dtype)]
        Abar, info = rsvd_truncate_backward_batched([A], [U], [S], [Vt], Ub, Sb, Vb, max_iter=ctx.max_iter)
        check_info(info, "rsvd_truncate_backward_batched")
        return Abar[0], None, None, None, None, None, None
