"""Benchmark: RSVD bond truncations/s of imaginary-time TEBD on one GB300.

Workload (one "step" = one second-order Trotter step = every bond update of the
chain once per layer, 95 truncations): open transverse-field Ising chain,
L = 64, h = 1, d = 2, chi = 128, dt = 0.01, FP64; each bond update is an RSVD
of the (chi d) x (chi d) = 256 x 256 two-site matrix truncated to chi
(p = 10, q = 2).  The state is first evolved from a seeded product state (20
untimed steps at dt = 0.1) so that the timed bond matrices carry the decaying
spectra of a converging TEBD run.

Prints ONE JSON line (rank 0).  Under torchrun every rank evolves its own chain
(replicas; the chain is not sharded) and the value is the total over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RSVD truncations/s & TFLOP/s vs full-SVD-truncate, 1 GB300, at stated error"
UNIT = "truncations/s"
L_SITES, CHI, D_LOC, H_FIELD, DT, P_OVER, Q_POW, SEED = 64, 128, 2, 1.0, 0.01, 10, 2, 5
SPIN, WIDTH = 0.5, 0  # model: spin-S chain (d = 2S + 1), or the 2D cylinder of circumference WIDTH (d = 2^WIDTH)
UPDATE, K_TERMS = "block", 2  # TEBD update form; "product": each cylinder bond as WIDTH gates of K_TERMS = 2 terms
PREP_STEPS, PREP_DT = 20, 0.1
WORKLOAD = "tebd_tfim_L64_chi128_d2_dt0.01_p10_q2_fp64"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
OZ_SLICE_PRODUCTS = 53  # BF16 slice products per FP64 product on the tensor cores (levels i + j <= 11 of 9 slices)

# DRAM bytes (read + write) per launch of a workload's dominant kernel, from one
# ncu capture of that kernel as it stands (summaries under profiles/); a kernel
# changed since its capture has no entry (traffic null).
TRAFFIC_PER_LAUNCH = {
    ("tebd", "householder"): (7.989504e6, "profiles/householder_panel_tebd_L64_chi128.md"),
    ("mixed", "gram"): (20.98e6, "profiles/gram_and_tc_gemm_mixed_bf16_16x4096.md"),
    ("mixed", "tcgemm"): (561.69e6 + 16.31e6, "profiles/gram_and_tc_gemm_mixed_bf16_16x4096.md"),
}


def traffic_of(workload, kernel):
    t = TRAFFIC_PER_LAUNCH.get((workload, kernel))
    return (t[0], t[1]) if t else (None, None)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz


def base_config():
    return {"workload": WORKLOAD, "model": model_name(), "L": L_SITES, "chi": CHI, "d": D_LOC, "h": H_FIELD, "dt": DT,
            "p": P_OVER, "q": Q_POW, "update": UPDATE,
            "bond_matrix": (f"{CHI * D_LOC}x{CHI * D_LOC}" if UPDATE == "block" else
                            f"X Y, X {CHI * D_LOC}x{K_TERMS * CHI}, Y {K_TERMS * CHI}x{CHI * D_LOC} (never formed)"),
            "fp64_products_with_A": "tcgen05 tensor cores, exact 9-slice BF16 split, FP64-class error",
            "truncations_per_step": truncations_per_step(), "l2": "flushed (512 MB write) before every timed step"}


def model_name():
    return f"cyl{WIDTH}" if WIDTH else ("tfim" if SPIN == 0.5 else f"spin{SPIN:g}")


def bond_term_oracle(otebd, i):
    """The bond term of the bench's model, from the oracle (CPU legs only)."""
    if WIDTH:
        return otebd.cylinder_bond_hamiltonian(i, L_SITES, H_FIELD, WIDTH)
    return otebd.bond_hamiltonian(i, L_SITES, H_FIELD, SPIN)


def truncations_per_step():
    """Bond compressions per Trotter step (product updates: one per coupling gate)."""
    a = len(range(0, L_SITES - 1, 2))
    b = len(range(1, L_SITES - 1, 2))
    return (2 * a + b) * (WIDTH if UPDATE == "product" else 1)


def job_ms(local_ms):
    """Timed-region duration of the whole job: the maximum over ranks (any
    torch.distributed backend; the local value when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_ms)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 7:
                continue
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
            except ValueError:
                continue
            for nme, v in zip(names, r[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nme)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ flop model
def bond_shapes():
    """(m, n, k, l) of every bond update of one Trotter step, per layer (A, B, A)."""
    D = [int(min(D_LOC ** min(j, L_SITES - j), CHI)) for j in range(L_SITES + 1)]
    out = []
    for layer in (0, 1, 0):
        lay = []
        for i in range(layer, L_SITES - 1, 2):
            m, n, k = D[i] * D_LOC, D_LOC * D[i + 2], D[i + 1]
            lay.append((m, n, k, min(k + P_OVER, m, n)))
        out.append(lay)
    return out


def hh_flops(rows, l, r):
    """Householder QR of a rows x l sample stopped after r reflectors (r = l when it
    runs to the end), and the accumulation of the explicit Q (rows x l) from them:
    2 (4 rows l r - 2 (rows + l) r^2 + 4 r^3 / 3)."""
    r = min(r, l)
    return 2.0 * (4.0 * rows * l * r - 2.0 * (rows + l) * r * r + 4.0 * r ** 3 / 3.0)


def step_flops(info):
    """Algorithmic FP64 flops of one Trotter step, split by kernel class.

    Follows the library's path decisions: Q = I, B = A only for m <= 16 (and
    m <= l); otherwise GEMMs for the sketch / power / projection (2q+2) 2mnl,
    plus the two-site contraction 2mnk and the B update 2mnk.  Each of the
    2q+1 orthonormalisations of a rows x l sample: CholeskyQR2 (two passes of
    Gram rows l^2, Cholesky + triangular inverse 2 l^3 / 3, Y R^-1 rows l^2)
    or, for nearly square samples (3l > rows), Householder QR stopped after the
    device-reported number of reflectors (rsvd_info.qr_columns of the last
    orthonormalisation, taken for all of them) with its explicit Q.  Jacobi
    (from the device counts): every sweep forms the row norms (2nl) and the
    inner products of all l(l-1)/2 pairs (2n each); each applied rotation
    costs 6n (the TEBD update does not accumulate the rotations of U).
    """
    flops = {"gemm": 0.0, "gram": 0.0, "cholesky": 0.0, "householder": 0.0, "jacobi": 0.0, "ozgemm": 0.0}
    if UPDATE == "product":
        return product_step_flops(info, flops)
    for j, lay in enumerate(bond_shapes()):
        for b, (m, n, k, l) in enumerate(lay):
            rec = info[j][0][b]  # (layer, compression, bond) records
            sweeps, rots, qr_cols, falls = int(rec[3]), int(rec[5]), int(rec[6]), int(rec[2])
            # the bond update forms no U: after the first orthonormalisation only the leading
            # r columns of Q carry the range (r = reported qr_columns, else l), and the products,
            # the later QRs, the contraction B_i B_{i+1} (over the nonzero Schmidt values,
            # at most r) and the B update (over the nonzero columns of V) work on r columns
            r = min(l, qr_cols) if qr_cols > 0 else l
            flops["gemm"] += 2.0 * m * n * min(k, r) + 2.0 * m * n * min(k, r)
            if not (m <= l and m <= 16):
                # products with A: on the tensor cores by exact slicing when m, n <= 1024 and l <= 256
                oz = m <= 1024 and n <= 1024 and l <= 256
                flops["ozgemm" if oz else "gemm"] += 2.0 * m * n * l + (2 * Q_POW + 1) * 2.0 * m * n * r
                for it in range(2 * Q_POW + 1):
                    rows = m if it % 2 == 0 else n
                    lw = l if it == 0 else r
                    if 3 * l > rows:
                        flops["householder"] += hh_flops(rows, lw, r)
                    else:
                        flops["gram"] += 2 * rows * l * l
                        flops["cholesky"] += 2 * (2.0 * l ** 3 / 3.0)
                        flops["gemm"] += 2 * rows * l * l
                # orthonormalisations whose CholeskyQR2 broke down ran Householder QR as well
                # (device count; which ones is not recorded: rows (m + n) / 2, the effective width)
                flops["householder"] += falls * hh_flops((m + n) // 2, r, r)
            svd_b_flops(flops, n, k, l, sweeps, rots)
    return flops


def svd_b_flops(flops, n, k, l, sweeps, rots):
    """The SVD of B (l x n): Jacobi on B, or for wide B (n >= 3l) the orthonormalisation of
    B^T (n x l), M = B Q_b (2 l n l), Jacobi on M (l x l) and V^T = W Q_b^T (2 k l n).
    Jacobi per sweep: row norms (2 n l) and all l (l - 1) / 2 pair products (2 n each); per
    applied rotation 6 n."""
    if 10 * n >= 30 * l:
        if 3 * l > n:
            flops["householder"] += hh_flops(n, l, l)
        else:
            flops["gram"] += 2 * n * l * l
            flops["cholesky"] += 2 * (2.0 * l ** 3 / 3.0)
            flops["gemm"] += 2 * n * l * l
        flops["gemm"] += 2.0 * l * n * l + 2.0 * k * l * n
        n = l
    flops["jacobi"] += sweeps * (l * (l - 1) / 2.0) * 2.0 * n + rots * 6.0 * n + (sweeps + 1) * 2.0 * n * l


def product_step_flops(info, flops):
    """step_flops of the product update: per compression of theta = X Y (X m x r, Y r x n,
    r = K k, never formed) every product with A is two GEMMs through r columns: the sketch
    2 (n + m) r l, then (2q + 1) more of 2 (m + n) r r_eff (r_eff = the effective rank, as in
    step_flops) and B = (X^T Q)^T Y; the Grams X^T X, Y Y^T (2 m r^2 + 2 n r^2) for
    ||theta||_F; W = Y V (2 r n k) and B_i = X_B W (2 m r k); orthonormalisations and
    Jacobi as in step_flops."""
    for j, lay in enumerate(bond_shapes()):
        for w in range(WIDTH):
            for b, (m, n, k, l) in enumerate(lay):
                rec = info[j][w][b]
                sweeps, rots, qr_cols, falls = int(rec[3]), int(rec[5]), int(rec[6]), int(rec[2])
                rr = min(l, qr_cols) if qr_cols > 0 else l
                r = K_TERMS * k
                flops["gemm"] += 2.0 * (m + n) * r * l + (2 * Q_POW + 1) * 2.0 * (m + n) * r * rr
                flops["gemm"] += 2.0 * m * r * r + 2.0 * n * r * r + 2.0 * r * n * min(k, rr) + 2.0 * m * r * min(k, rr)
                for it in range(2 * Q_POW + 1):
                    rows = m if it % 2 == 0 else n
                    lw = l if it == 0 else rr
                    if 3 * l > rows:
                        flops["householder"] += hh_flops(rows, lw, rr)
                    else:
                        flops["gram"] += 2 * rows * l * l
                        flops["cholesky"] += 2 * (2.0 * l ** 3 / 3.0)
                        flops["gemm"] += 2 * rows * l * l
                flops["householder"] += falls * hh_flops((m + n) // 2, rr, rr)
                svd_b_flops(flops, n, k, l, sweeps, rots)
    return flops


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import ctypes

    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1710_01463_gb300 import _lib, inputs
    from paper_1710_01463_gb300.tebd import TebdChain

    lib = _lib.load()
    ch = TebdChain(L_SITES, CHI, h=H_FIELD, p=P_OVER, q=Q_POW, seed=SEED + 1000 * rank, S=SPIN, W=WIDTH or None,
                   update=UPDATE)
    ch.set_product_state(inputs.product_state_vectors(L_SITES, D_LOC, 102 + rank))
    ch.set_dt(PREP_DT)
    for s in range(PREP_STEPS):
        ch.step(s)
    ch.set_dt(DT)
    for s in range(args.warmup):
        ch.step(PREP_STEPS + s)
    torch.cuda.synchronize()

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    clocks = ClockSampler(local)
    lib.rsvd_profile_enable(200000)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.time()
    for s in range(args.steps):
        flush.zero_()
        ev[s][0].record(stream)
        ch.step(PREP_STEPS + args.warmup + s)
        ev[s][1].record(stream)
        infos.append(ch.info.clone())
    torch.cuda.synchronize()
    wall = time.time() - t0
    clk = clocks.stop()
    nclass = 16
    ms_c = (ctypes.c_double * nclass)()
    cnt_c = (ctypes.c_int * nclass)()
    ncls = lib.rsvd_profile_collect(ms_c, cnt_c, nclass)
    lib.rsvd_profile_enable(0)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = job_ms(sum(step_ms))
    ms_per_step = tot_ms / args.steps
    value = ws * truncations_per_step() / (ms_per_step / 1e3)

    # algorithmic flops from the device-reported sweep / rotation counts
    fl = {"gemm": 0.0, "gram": 0.0, "cholesky": 0.0, "householder": 0.0, "jacobi": 0.0, "ozgemm": 0.0}
    for inf in infos:
        f = step_flops(inf.cpu().numpy())
        for key in fl:
            fl[key] += f[key]
    tflops = ws * sum(fl.values()) / (tot_ms / 1e3) / 1e12
    classes = {lib.rsvd_profile_class_name(c).decode(): (ms_c[c], cnt_c[c]) for c in range(ncls)}
    total_kernel_ms = sum(v[0] for v in classes.values())
    kernels = {}
    for name, (ms, cnt) in classes.items():
        if cnt == 0:
            continue
        entry = {"launch_groups": cnt, "ms_total": round(ms, 3), "share": round(ms / total_kernel_ms, 4)}
        if name == "ozgemm" and ms > 0:  # FP64 products on the tensor cores: FP64-equivalent rate
            entry["tflops_fp64_equivalent"] = round(fl[name] / (ms / 1e3) / 1e12, 4)
        elif name in fl and ms > 0:
            entry["tflops"] = round(fl[name] / (ms / 1e3) / 1e12, 4)
            entry["frac_fp64_peak"] = round(fl[name] / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS, 4)
        kernels[name] = entry
    dom = max(kernels, key=lambda k: kernels[k]["ms_total"])
    dom_ach = fl.get(dom, 0.0) / (classes[dom][0] / 1e3) / 1e12 if classes[dom][0] > 0 else 0.0
    launches = 0
    per_group = {"gram": 2, "select": 2}
    for name, (ms, cnt) in classes.items():
        launches += cnt * per_group.get(name, 1)
    roofline = {"bound": "alu", "kernel": dom, "achieved": round(dom_ach, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                "unit": "TFLOP/s", "frac": round(dom_ach / FP64_PEAK_TFLOPS, 4),
                # the captured traffic belongs to the default chain (its 256-row samples) only
                "traffic": traffic_of("tebd" if model_name() == "tfim" and UPDATE == "block" else WORKLOAD, dom)[0],
                "traffic_source": traffic_of("tebd" if model_name() == "tfim" and UPDATE == "block" else WORKLOAD,
                                             dom)[1],
                "peak_source": "FP64 DFMA: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s; "
                               "DFMA microbenchmark on this GB300: 1.20 TFLOP/s)"}

    result = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
              "config": dict(base_config(), parallelism=f"replicas{ws}"),
              "tflops": round(tflops, 4), "roofline": roofline, "kernels": kernels,
              "gpu_launches": launches, "clocks": clk, "wall_s_timed_loop": round(wall, 3)}
    trunc = torch.stack([i for i in infos]).cpu().numpy()
    result["device_status"] = {"max_jacobi_sweeps": int(trunc[..., 3].max()),
                               "mean_jacobi_sweeps": round(float(trunc[..., 3].mean()), 3),
                               "householder_fallbacks_per_step": round(float(trunc[..., 2].sum()) / args.steps, 2),
                               "nonzero_status": int((trunc[..., 0] != 0).sum())}
    if rank == 0 and not args.no_extras:
        result["e2e"] = e2e_leg(ch, args)
        result["error"] = error_leg(ch)
        result["comparator"] = comparator_leg()
        result["cpu_baseline"] = cpu_leg(ch)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


def e2e_leg(ch, args):
    """Same metric through the public API with the MPS in pinned host memory:
    every step copies the state host->device, runs the Trotter step, and copies
    the new state device->host."""
    import torch
    hB = torch.empty(ch.B.shape, dtype=torch.float64, pin_memory=True)
    hl = torch.empty(ch.lam.shape, dtype=torch.float64, pin_memory=True)
    hB.copy_(ch.B)
    hl.copy_(ch.lam)
    stream = torch.cuda.current_stream()
    steps = max(1, min(args.steps, 10))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    for s in range(steps):
        flush.zero_()  # L2 flushed between steps, outside the timing, as in the device-timed loop
        ev[s][0].record(stream)
        ch.B.copy_(hB, non_blocking=True)
        ch.lam.copy_(hl, non_blocking=True)
        ch.step(10_000 + s)
        hB.copy_(ch.B, non_blocking=True)
        hl.copy_(ch.lam, non_blocking=True)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    nbytes = hB.numel() * 8 + hl.numel() * 8
    return {"value": round(truncations_per_step() / (ms / 1e3), 3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "ms_per_step": round(ms, 4), "steps": steps}


def center_theta(ch):
    """Host copy of the center bond's two-site matrix theta = lam . (B_i B_{i+1}) (no gate)."""
    import numpy as np
    B = ch.tensors()
    lam = ch.schmidt_values()
    i = L_SITES // 2 - 1
    two = np.einsum("atb,buc->atuc", B[i], B[i + 1])
    th = lam[i][:, None, None, None] * two
    return th.reshape(B[i].shape[0] * D_LOC, D_LOC * B[i + 1].shape[2])


def error_leg(ch):
    """RSVD error on a live bond matrix: GPU RSVD vs the exact truncated SVD."""
    import numpy as np
    import torch
    from paper_1710_01463_gb300 import api
    A = center_theta(ch)
    U, S, Vt, info = api.rsvd_truncate(torch.from_numpy(A).cuda(), CHI, P_OVER, Q_POW, SEED, 0)
    torch.cuda.synchronize()
    s_full = np.linalg.svd(A, compute_uv=False)
    u, s, vt = U.cpu().numpy(), S.cpu().numpy(), Vt.cpu().numpy()
    err = np.linalg.norm(A - (u * s) @ vt)
    dtr = np.sqrt(np.sum(s_full[CHI:] ** 2))
    big = s_full[:CHI] > 1e-8 * s_full[0]
    nrm = float(np.linalg.norm(A))
    # the ratio to the optimal (Eckart-Young) error means something only when that error is
    # above rounding; otherwise the error is reported relative to ||A||_F
    meaningful = dtr > 1e-12 * nrm
    return {"bond": "center", "fro_err_over_delta_trunc": float(err / dtr) if meaningful else None,
            "fro_err_over_norm_a": float(err / nrm),
            "delta_trunc_fro": float(dtr), "sigma_chi_over_sigma_1": float(s_full[CHI - 1] / s_full[0]),
            "max_rel_sigma_err_above_1e-8": float(np.max(np.abs(s[big] - s_full[:CHI][big]) / s_full[:CHI][big]))}


def comparator_leg():
    """Full SVD + truncate with torch.linalg.svd (cuSOLVER) FP64 on 32 bond-sized matrices
    (product update: the paper's TSVD of the P form, QR of X then the SVD of the
    (K chi) x (chi d) matrix R Y)."""
    import torch
    from paper_1710_01463_gb300 import inputs
    if UPDATE == "product":
        return product_comparator_leg()
    A = torch.stack([torch.from_numpy(inputs.dense_case(CHI * D_LOC, CHI * D_LOC, seed=300 + j)) for j in range(32)]).cuda()
    torch.linalg.svd(A[:2], full_matrices=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    U, S, Vh = torch.linalg.svd(A, full_matrices=False)
    Uk, Sk, Vk = U[..., :CHI].contiguous(), S[..., :CHI].contiguous(), Vh[..., :CHI, :].contiguous()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"kind": f"torch.linalg.svd (cuSOLVER) FP64 + slice to chi, batch of 32 {CHI * D_LOC}x{CHI * D_LOC} matrices",
            "truncations_per_s": round(32 / (ms / 1e3), 3), "ms_per_truncation": round(ms / 32, 4)}


def product_comparator_leg():
    import torch
    from paper_1710_01463_gb300 import inputs
    m = n = CHI * D_LOC
    r = K_TERMS * CHI
    X = torch.stack([torch.from_numpy(inputs.random_dense(m, r, 400 + j)) for j in range(32)]).cuda()
    Y = torch.stack([torch.from_numpy(inputs.random_dense(r, n, 500 + j)) for j in range(32)]).cuda()
    torch.linalg.svd(torch.linalg.qr(X[:2])[1] @ Y[:2], full_matrices=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    Qx, R = torch.linalg.qr(X)
    U, S, Vh = torch.linalg.svd(R @ Y, full_matrices=False)
    Uk, Sk, Vk = (Qx @ U[..., :CHI]).contiguous(), S[..., :CHI].contiguous(), Vh[..., :CHI, :].contiguous()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"kind": f"torch.linalg.qr of X ({m}x{r}) + torch.linalg.svd (cuSOLVER) of R Y ({r}x{n}) FP64 + slice "
                    f"to chi, batch of 32",
            "truncations_per_s": round(32 / (ms / 1e3), 3), "ms_per_truncation": round(ms / 32, 4)}


def cpu_leg(ch):
    """The oracle (numpy FP64, as it stands) on the host: a bounded sample of the
    same workload - the bond updates of one layer-A sweep over the 8 central
    bonds, from the current GPU state."""
    import numpy as np
    from oracle import tebd as otebd
    B = ch.tensors()
    lam = ch.schmidt_values()
    comp = otebd.make_compressor("rsvd", p=P_OVER, q=Q_POW, seed=SEED)
    bonds = [i for i in range(0, L_SITES - 1, 2)][12:20]
    t0 = time.time()
    n = 0
    while True:
        for i in bonds:
            if UPDATE == "product":
                for j, (uL, uR) in enumerate(otebd.cylinder_product_gates(i, L_SITES, H_FIELD, WIDTH, DT / 2)):
                    otebd.product_update(B, lam, i, uL, uR, comp, (7 * WIDTH + j) * L_SITES + i)
                    n += 1
            else:
                G = otebd.gate(bond_term_oracle(otebd, i), DT / 2)
                otebd.bond_update(B, lam, i, G, comp, 7 * L_SITES + i)
                n += 1
        if time.time() - t0 > 10.0:
            break
    el = time.time() - t0
    return {"value": round(n / el, 4), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} central {CHI * D_LOC}x{CHI * D_LOC} bond compressions ({UPDATE} update; RSVD k={CHI}, "
                      f"p={P_OVER}, q={Q_POW}) "
                      f"of the L={L_SITES} {model_name()} chain, numpy FP64, "
                      f"BLAS threads = all host cores, Philox in pure Python"}


# ------------------------------------------------------------------ other workloads
# `--workload dense|mixed|sectors|grad`: the other configurations of the path,
# each as its own JSON line (same contract; the default run is the TEBD one).
HBM_PEAK_GBS = None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


def profile_classes(lib):
    import ctypes
    nclass = 16
    ms_c = (ctypes.c_double * nclass)()
    cnt_c = (ctypes.c_int * nclass)()
    ncls = lib.rsvd_profile_collect(ms_c, cnt_c, nclass)
    lib.rsvd_profile_enable(0)
    return {lib.rsvd_profile_class_name(c).decode(): (ms_c[c], cnt_c[c]) for c in range(ncls)}


def rsvd_flops(m, n, k, l, q, sweeps, rots, prec, qr_cols=0, want_u=True):
    """Algorithmic flops of one RSVD by kernel class (see step_flops), plus the
    tensor-core products of the BF16 / TF32 forms.  Wide B (n >= 3l): the SVD
    of B runs on the l x l factor of an orthonormalisation of B^T."""
    f = {"gemm": 0.0, "gram": 0.0, "cholesky": 0.0, "householder": 0.0, "jacobi": 0.0, "tcgemm": 0.0, "ozgemm": 0.0}
    exact = m <= l and m <= 16
    oz = prec == "f64" and m <= 1024 and n <= 1024 and l <= 256  # FP64 products with A on the tensor cores

    def orth(rows):
        if 3 * l > rows:
            f["householder"] += hh_flops(rows, l, qr_cols if qr_cols > 0 else l)
        else:
            f["gram"] += 2 * rows * l * l
            f["cholesky"] += 2 * (2.0 * l ** 3 / 3.0)
            f["gemm"] += 2 * rows * l * l

    if not exact:
        f["tcgemm" if prec in ("bf16", "tf32") else "ozgemm" if oz else "gemm"] += (2 * q + 2) * 2.0 * m * n * l
        for it in range(2 * q + 1):
            orth(m if it % 2 == 0 else n)
    if want_u:
        f["gemm"] += 2.0 * m * l * k  # lift
    jn = n
    if 10 * n >= 30 * l:  # B^T = Q_b R, M = B Q_b, V^T = W Q_b^T
        orth(n)
        f["gemm"] += 2.0 * l * n * l + 2.0 * k * l * n
        jn = l
    f["jacobi"] += (sweeps * (l * (l - 1) / 2.0) * 2.0 * jn + rots * (6.0 * jn + (6.0 * l if want_u else 0.0))
                    + (sweeps + 1) * 2.0 * jn * l)
    return f


def tc_bytes(m, n, l, q, eb):
    """HBM bytes of the tensor-core products of one RSVD: every product reads A
    (or A^T) once, the split thin operand (2 lp rows) and writes the FP32 sample."""
    lp = (l + 15) // 16 * 16
    npad = 2 * lp if 2 * lp <= 256 else lp
    tot = 0.0
    for it in range(2 * q + 2):
        rows, K = (m, n) if it % 2 == 0 else (n, m)
        tot += rows * K * eb + npad * K * eb + rows * l * 4
    return tot


def run_workload(args):
    import numpy as np
    import torch
    from paper_1710_01463_gb300 import _lib, api, inputs
    from oracle import rsvd as orsvd

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib = _lib.load()
    peaks = measured_peaks()
    dev = torch.device("cuda", local)
    wl = args.workload
    q = 2
    g = torch.Generator(device="cpu").manual_seed(1234 + rank)

    def ortho(nn, seed):
        # seeded orthogonal factor, formed on the host (no solver library on the device side)
        return torch.from_numpy(inputs.haar_like_orthogonal(nn, seed)).to(dev)

    if wl == "dense":
        m = n = 256
        k, p, B = 32, 8, 1024
        s = torch.from_numpy(inputs.exp_spectrum(256)).to(dev)
        U0, V0 = ortho(256, 202), ortho(256, 203)
        As = []
        for j in range(B):
            rp, cp = torch.randperm(256, generator=g).to(dev), torch.randperm(256, generator=g).to(dev)
            As.append(((U0[rp] * s[None, :]) @ V0[cp].T).contiguous())
        dtype = torch.float64
        ks = [k] * B
        prec = "f64"
        config = {"workload": "dense_fp64_256x256_k32_p8_q2_batch1024", "m": 256, "n": 256, "k": k, "p": p, "q": q,
                  "batch": B, "spectrum": "s_i = exp(-i/16)", "l2": "inputs (512 MB) larger than L2"}
    elif wl == "mixed":
        m = n = 4096
        k, p, B = 64, 16, 16
        s = torch.from_numpy(inputs.power_spectrum(n, 1.5)).to(dev)
        U0, V0 = ortho(n, 206), ortho(n, 207)
        As = []
        for j in range(B):
            rp, cp = torch.randperm(n, generator=g).to(dev), torch.randperm(n, generator=g).to(dev)
            As.append(((U0[rp] * s[None, :]) @ V0[cp].T).to(torch.bfloat16 if args.precision == "bf16" else torch.float32).contiguous())
        del U0, V0
        dtype = As[0].dtype
        ks = [k] * B
        prec = args.precision
        config = {"workload": f"ttn_{prec}_4096x4096_k64_p16_q2_batch16", "m": m, "n": n, "k": k, "p": p, "q": q,
                  "batch": B, "spectrum": "s_i = i^-1.5", "l2": "inputs (16 x 4096^2) larger than L2"}
    elif wl == "sectors":
        shapes, f = inputs.sector_shapes(N=32, lo=64, hi=2048, seed=104)
        k, p, B = 512, 16, 32
        As = []
        for b, ((mb, nb), fb) in enumerate(zip(shapes, f)):
            r = min(mb, nb)
            s = torch.from_numpy(inputs.power_spectrum(r, 1.2, fb)).to(dev)
            Ub = ortho(mb, 3000 + 2 * b)[:, :r]
            Vb = ortho(nb, 3001 + 2 * b)[:, :r]
            As.append(((Ub * s[None, :]) @ Vb.T).float().contiguous())
        dtype = torch.float32
        ks = [min(k, *A.shape) for A in As]
        prec = "f32"
        config = {"workload": "sectors32_64to2048_chi512_fp32_p16_q2", "blocks": 32, "chi_global": 512, "p": p,
                  "q": q, "policy": "maximal k_b = min(chi, m_b, n_b)", "spectrum": "s_i = f_b i^-1.2",
                  "elements": int(sum(A.numel() for A in As)), "l2": "flushed (512 MB write) before every timed step"}
    elif wl == "grad":
        m = n = 1024
        k, p, B = 128, 16, 64
        s = torch.from_numpy(inputs.harmonic_spectrum(n)).to(dev)
        U0, V0 = ortho(n, 208), ortho(n, 209)
        As = []
        for j in range(B):
            rp, cp = torch.randperm(n, generator=g).to(dev), torch.randperm(n, generator=g).to(dev)
            As.append(((U0[rp] * s[None, :]) @ V0[cp].T).float().contiguous())
        rng = np.random.default_rng(105)
        w = torch.from_numpy(rng.uniform(0, 1, size=k)).to(dev)
        W = torch.from_numpy(rng.standard_normal((n, 8))).float().to(dev)
        dtype = torch.float32
        ks = [k] * B
        prec = "f32"
        config = {"workload": "grad_fp32_1024x1024_k128_p16_q2_batch64", "m": m, "n": n, "k": k, "p": p, "q": q,
                  "batch": B, "spectrum": "s_i = 1/(1+0.05 i)", "loss": "sum w_i s_i + ||W^T U_k||_F^2, W 1024x8",
                  "l2": "inputs (256 MB) larger than L2"}
    else:
        raise ValueError(wl)

    plan = api.BatchedPlan([tuple(A.shape) for A in As], ks, p, q, 103 + 1000 * rank, 0, dtype, dev,
                           chi_global=(512 if wl == "sectors" else 0), tf32=(prec == "tf32"))
    if wl == "sectors" and args.policy == "estimate":
        # trial ranks from the previous step's selection plus a margin of 16
        # (the paper: estimates from previous iterations plus oversampling)
        plan.run(As)
        torch.cuda.synchronize()
        kprev = plan.k_out.cpu().tolist()
        ks = [min(min(A.shape), kp + 16) for A, kp in zip(As, kprev)]
        config["policy"] = "previous step's kept count + 16 (first step: maximal)"
        plan = api.BatchedPlan([tuple(A.shape) for A in As], ks, p, q, 103 + 1000 * rank, 0, dtype, dev,
                               chi_global=512)
    adaptive = wl == "sectors" and args.policy == "adaptive"
    if adaptive:
        # the paper's chi / N (c = 0) as the first guess of every step; saturated blocks grow
        r0 = [max(1, 512 // len(As))] * len(As)
        plan = api.AdaptiveSectorsPlan([tuple(A.shape) for A in As], 512, r0, p, q, 103 + 1000 * rank, 0, dtype, dev)
        config["policy"] = ("adaptive: first guess chi / N = 16 every step, the ranks of saturated blocks doubled "
                            "until none is (flops counted for the final round only)")

    def step():
        if adaptive:
            plan.ranks = list(r0)
        plan.run(As)
        if wl == "grad":
            Ub = [2.0 * (W @ (W.T @ U)) for U in plan.U]
            Sb = [w.clone() for _ in plan.S]
            api.rsvd_truncate_backward_batched(As, plan.U, plan.S, plan.Vt, Ub, Sb, None, max_iter=120, tol=1e-6)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    lib.rsvd_profile_enable(400000)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    infos = []
    for i in range(args.steps):
        if wl == "sectors":
            flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        infos.append(plan.info.clone())
    torch.cuda.synchronize()
    clk = clocks.stop()
    classes = profile_classes(lib)
    tot_ms = job_ms(sum(a.elapsed_time(b) for a, b in ev))
    ms_per_step = tot_ms / args.steps
    units_per_step = 1 if wl == "sectors" else B
    value = ws * units_per_step / (ms_per_step / 1e3)
    if adaptive:
        ks = list(plan.ranks)

    # algorithmic work
    fl = {"gemm": 0.0, "gram": 0.0, "cholesky": 0.0, "householder": 0.0, "jacobi": 0.0, "tcgemm": 0.0, "ozgemm": 0.0}
    tcb = 0.0
    for inf in infos:
        rec = inf.cpu().numpy()
        for j, A in enumerate(As):
            mm, nn = A.shape
            kk = ks[j]
            ll = min(kk + p, mm, nn)
            f = rsvd_flops(mm, nn, kk, ll, q, int(rec[j][3]), int(rec[j][5]), prec, int(rec[j][6]))
            for key in fl:
                fl[key] += f[key]
            if prec in ("bf16", "tf32"):
                tcb += tc_bytes(mm, nn, ll, q, 2 if prec == "bf16" else 4)
            if wl == "grad":  # backward: retained block + 120 CG iterations + the coupling terms (GEMMs)
                fl["gemm"] += 2.0 * mm * kk * kk * 2 + 2.0 * mm * nn * kk
                fl["gemm"] += 120 * (2 * 2.0 * mm * nn * kk + 4 * 2.0 * mm * kk * kk)
                fl["gemm"] += 3 * 2.0 * mm * nn * kk
    total_kernel_ms = sum(v[0] for v in classes.values())
    kernels = {}
    for name, (ms, cnt) in classes.items():
        if cnt == 0:
            continue
        e = {"launch_groups": cnt, "ms_total": round(ms, 3), "share": round(ms / total_kernel_ms, 4)}
        if name == "tcgemm" and ms > 0:
            e["gbs"] = round(tcb / (ms / 1e3) / 1e9, 1)
            e["frac_hbm_peak"] = round(tcb / (ms / 1e3) / 1e9 / peaks["hbm_gbs"], 4)
            e["tflops"] = round(fl["tcgemm"] / (ms / 1e3) / 1e12, 3)
        elif name == "ozgemm" and ms > 0:
            e["tflops_fp64_equivalent"] = round(fl[name] / (ms / 1e3) / 1e12, 4)
        elif name in fl and ms > 0 and fl[name] > 0:
            e["tflops"] = round(fl[name] / (ms / 1e3) / 1e12, 4)
            if prec == "f64" or name in ("gram", "cholesky", "householder", "jacobi"):
                e["frac_fp64_peak"] = round(fl[name] / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS, 4)
            else:
                e["frac_fp32_peak"] = round(fl[name] / (ms / 1e3) / 1e12 / FP32_PEAK_TFLOPS, 4)
        kernels[name] = e
    dom = max(kernels, key=lambda x: kernels[x]["ms_total"])
    dms = classes[dom][0] / 1e3
    if dom == "ozgemm":
        # 53 exact BF16 slice products per FP64 product, against the measured BF16 tensor peak
        tfl = OZ_SLICE_PRODUCTS * fl["ozgemm"] / dms / 1e12 if dms > 0 else 0.0
        roofline = {"bound": "tensor", "kernel": dom, "achieved": round(tfl, 2), "peak": peaks["bf16_tflops"],
                    "unit": "TFLOP/s", "frac": round(tfl / peaks["bf16_tflops"], 4),
                    "traffic": traffic_of(wl, dom)[0], "traffic_source": traffic_of(wl, dom)[1],
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops (of measured)",
                    "note": "BF16 flops executed = 53 slice products x the FP64 product's 2 m n l"}
    elif dom == "tcgemm":
        roofline = {"bound": "hbm", "kernel": dom, "achieved": round(tcb / dms / 1e9, 1), "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": round(tcb / dms / 1e9 / peaks["hbm_gbs"], 4),
                    "traffic": traffic_of(wl, dom)[0], "traffic_source": traffic_of(wl, dom)[1],
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    else:
        fp64 = prec == "f64" or dom in ("gram", "cholesky", "householder", "jacobi")
        pk = FP64_PEAK_TFLOPS if fp64 else FP32_PEAK_TFLOPS
        ach = fl.get(dom, 0.0) / dms / 1e12 if dms > 0 else 0.0
        roofline = {"bound": "alu", "kernel": dom, "achieved": round(ach, 4), "peak": round(pk, 3), "unit": "TFLOP/s",
                    "frac": round(ach / pk, 4), "traffic": traffic_of(wl, dom)[0],
                    "traffic_source": traffic_of(wl, dom)[1],
                    "peak_source": ("FP64 DFMA 152 SMs x 2/clk x 2 flop x 2.07 GHz" if fp64 else
                                    "FP32 FFMA 152 SMs x 128/clk x 2 flop x 2.07 GHz") + " (derived)"}
    launches = sum(cnt * {"gram": 2, "select": 2}.get(name, 1) for name, (ms, cnt) in classes.items())
    stat = torch.stack(infos).cpu().numpy()
    result = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": {"f64": "f64", "f32": "f32", "bf16": "bf16",
                                                                "tf32": "tf32"}[prec],
              "data": "synthetic", "config": dict(config, parallelism=f"replicas{ws}"),
              "tflops": round(ws * sum(fl.values()) / (tot_ms / 1e3) / 1e12, 4), "roofline": roofline,
              "kernels": kernels, "gpu_launches": launches, "clocks": clk,
              "device_status": {"max_jacobi_sweeps": int(stat[..., 3].max()),
                                "mean_jacobi_sweeps": round(float(stat[..., 3].mean()), 3),
                                "nonzero_status": int((stat[..., 0] != 0).sum())}}
    if adaptive:
        result["device_status"]["adaptive_rounds"] = plan.rounds
        result["device_status"]["final_trial_ranks"] = list(plan.ranks)
    if rank == 0 and not args.no_extras:
        # e2e: inputs from pinned host memory, results back to the host, every step
        hA = [A.cpu().pin_memory() for A in As]
        hS = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in plan.S]
        nst = max(1, min(args.steps, 5))
        eev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nst)]
        torch.cuda.synchronize()
        for i in range(nst):
            flush.zero_()  # L2 flushed between steps, outside the timing
            eev[i][0].record(stream)
            for A, h in zip(As, hA):
                A.copy_(h, non_blocking=True)
            step()
            for h, t in zip(hS, plan.S):
                h.copy_(t, non_blocking=True)
            eev[i][1].record(stream)
        torch.cuda.synchronize()
        ems = sum(a.elapsed_time(b) for a, b in eev) / nst
        result["e2e"] = {"value": round(units_per_step / (ems / 1e3), 3), "unit": UNIT,
                         "h2d_bytes_per_step": int(sum(h.numel() * h.element_size() for h in hA)),
                         "d2h_bytes_per_step": int(sum(t.numel() * 8 for t in plan.S)), "ms_per_step": round(ems, 3)}
        # error against the exact truncated SVD on matrix 0
        A0 = As[0].double().cpu().numpy()
        k0 = ks[0]
        sv = np.linalg.svd(A0, compute_uv=False)
        s_gpu = plan.S[0].cpu().numpy()
        big = sv[:k0] > 1e-8 * sv[0]
        s_gpu = s_gpu[:k0]
        u0, v0 = plan.U[0][:, :k0].double().cpu().numpy(), plan.Vt[0][:k0].double().cpu().numpy()
        err = np.linalg.norm(A0 - (u0 * s_gpu) @ v0)
        dtr = np.sqrt(np.sum(sv[k0:] ** 2))
        _, so, _ = orsvd.rsvd(A0, k0, p, q, 103, 0)
        result["error"] = {"matrix": 0, "fro_err_over_delta_trunc": float(err / dtr) if dtr > 0 else None,
                           "max_rel_sigma_err_vs_exact": float(np.max(np.abs(s_gpu[big] - sv[:k0][big]) / sv[:k0][big])),
                           "max_abs_sigma_err_vs_fp64_oracle_rsvd_over_sigma1": float(np.max(np.abs(s_gpu - so)) / so[0])}
        if wl == "sectors":
            ko = plan.k_out.cpu().tolist()
            result["error"]["k_out"] = ko
            # a trial rank is adequate when the block's last trial value was not selected
            result["error"]["trial_ranks_adequate"] = bool(all(kk < kt or kt == min(A.shape)
                                                               for kk, kt, A in zip(ko, ks, As)))
        # comparator: full SVD + truncate (cuSOLVER via torch) on matrix 0..3
        cd = torch.float64 if prec == "f64" else torch.float32
        Ac = [A.to(cd) for A in As[:(1 if wl == "mixed" else 4)]]
        torch.linalg.svd(Ac[0], full_matrices=False)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        for A in Ac:
            Uf, Sf, Vf = torch.linalg.svd(A, full_matrices=False)
        c1.record()
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1) / len(Ac)
        result["comparator"] = {"kind": f"torch.linalg.svd (cuSOLVER) {cd} + slice, per matrix",
                                "ms_per_matrix": round(cms, 3),
                                "matrices_per_s": round(1e3 / cms, 3)}
        # CPU oracle on a bounded sample: oracle RSVD of matrix 0 (and more while under ~10 s)
        t0 = time.time()
        nrun = 0
        while True:
            orsvd.rsvd(As[nrun % len(As)].double().cpu().numpy(), ks[nrun % len(As)], p, q, 103, nrun)
            nrun += 1
            if time.time() - t0 > 10.0:
                break
        el = time.time() - t0
        per = el / nrun
        cpu_value = (1.0 / (per * len(As))) if wl == "sectors" else 1.0 / per
        result["cpu_baseline"] = {"value": round(cpu_value, 5), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                  "sample": f"{nrun} oracle RSVD(s) of the workload's matrices (numpy FP64, BLAS threads = all host cores)"
                                            + ("; sectors: per-block time x 32" if wl == "sectors" else "")}
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


# ------------------------------------------------------------------ reference arm (the oracle)
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from oracle import tebd as otebd
    from paper_1710_01463_gb300 import inputs
    D = otebd.bond_dims(L_SITES, D_LOC, CHI)
    B, lam = otebd.product_state(inputs.product_state_vectors(L_SITES, D_LOC, 102), D)
    comp = otebd.make_compressor("rsvd", p=P_OVER, q=Q_POW, seed=SEED)
    # a step of the reference arm: 4 central bond updates (a bounded sample of one Trotter step)
    bonds = [i for i in range(0, L_SITES - 1, 2)][14:18]

    per = WIDTH if UPDATE == "product" else 1  # compressions per bond update

    def one(step):
        for i in bonds:
            if UPDATE == "product":
                for j, (uL, uR) in enumerate(otebd.cylinder_product_gates(i, L_SITES, H_FIELD, WIDTH, DT / 2)):
                    otebd.product_update(B, lam, i, uL, uR, comp, (3 * step * WIDTH + j) * L_SITES + i)
            else:
                G = otebd.gate(bond_term_oracle(otebd, i), DT / 2)
                otebd.bond_update(B, lam, i, G, comp, (3 * step) * L_SITES + i)

    for s in range(args.warmup):
        one(s)
    t0 = time.time()
    for s in range(args.steps):
        one(args.warmup + s)
    el = time.time() - t0
    value = len(bonds) * per * args.steps / el
    sample = (f"{len(bonds) * per} central {CHI * D_LOC}x{CHI * D_LOC} bond compressions per step ({UPDATE} update; "
              f"RSVD k={CHI}, p={P_OVER}, q={Q_POW}), numpy FP64 oracle, bond matrices from a product state")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": dict(base_config(), parallelism=f"replicas{ws}"),
           "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the e2e / error / comparator / CPU legs")
    ap.add_argument("--workload", default="tebd", choices=["tebd", "dense", "mixed", "sectors", "grad"],
                    help="tebd (default): the TEBD bond-update workload; the others time the remaining configurations")
    ap.add_argument("--precision", default="bf16", choices=["bf16", "tf32"], help="mixed workload: operand precision")
    ap.add_argument("--policy", default="estimate", choices=["estimate", "maximal", "adaptive"],
                    help="sectors workload: per-block trial ranks")
    ap.add_argument("--chain-length", type=int, default=64,
                    help="L (default 64); a shorter chain keeps the 256 x 256 central bonds (profiling case)")
    ap.add_argument("--spin", type=float, default=0.5, help="TEBD: spin S of the chain (d = 2S + 1; Sec. III.B)")
    ap.add_argument("--cylinder-width", type=int, default=0,
                    help="TEBD: circumference W of the 2D cylinder mapped onto a chain of rings (d = 2^W)")
    ap.add_argument("--update", default="block", choices=["block", "product"],
                    help="TEBD: block update (one d^2 x d^2 gate per bond) or, for the cylinder, product update "
                         "(each bond as W gates of K = 2 Kronecker terms; Sec. III.A)")
    ap.add_argument("--field", type=float, default=None,
                    help="TEBD: field h (default 1 for S = 1/2, 1.5 for S > 1/2, 3.044 for the cylinder)")
    args = ap.parse_args()
    global L_SITES, WORKLOAD, SPIN, WIDTH, D_LOC, H_FIELD, UPDATE
    if args.chain_length != L_SITES:
        L_SITES = args.chain_length
    SPIN, WIDTH = args.spin, args.cylinder_width
    if args.update == "product" and not WIDTH:
        ap.error("--update product needs --cylinder-width")
    UPDATE = args.update
    D_LOC = 2 ** WIDTH if WIDTH else int(round(2 * SPIN)) + 1
    H_FIELD = args.field if args.field is not None else (3.044 if WIDTH else (1.0 if SPIN == 0.5 else 1.5))
    WORKLOAD = (f"tebd_{model_name()}{'_product' if UPDATE == 'product' else ''}_L{L_SITES}_chi{CHI}_d{D_LOC}"
                f"_dt{DT:g}_p{P_OVER}_q{Q_POW}_fp64"
                + (f"_h{H_FIELD:g}" if args.field is not None else ""))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "tebd":
        run_workload(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
