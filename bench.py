"""Benchmark: RSVD bond truncations/s of imaginary-time TEBD on one GB300.

Workload (one "step" = one second-order Trotter step = every bond update of the
chain once per layer, 95 truncations): open transverse-field Ising chain,
L = 64, h = 1, d = 2, chi = 128, dt = 0.01, FP64; each bond update is an RSVD
of the (chi d) x (chi d) = 256 x 256 two-site matrix truncated to chi
(p = 10, q = 2).  The timed steps start from the converged ground state: the
chain is first evolved from a seeded product state by the imaginary-time
schedule dt = 0.1, 0.05, 0.02 (1450 untimed steps; `--state early` times the
state after 20 coarse steps instead).

The line also carries: the end-to-end rate through the public API with the MPS
in pinned host memory; the error of the compression on a live bond matrix; the
same steps with Alg. TSVD on the library's own engine (the speedup tau of the
paper); torch.linalg.svd (cuSOLVER) as a black-box comparator; the oracle on the
host cores; and short legs of the other configurations (`other_configs`).

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
STATE = "ground"
WORKLOAD = "tebd_tfim_L64_chi128_d2_dt0.01_p10_q2_fp64"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # 152 SMs x 128 FFMA/clk x 2 flop x 2.07 GHz
OZ_SLICE_PRODUCTS = 53  # BF16 slice products per FP64 product on the tensor cores (levels i + j <= 11 of 9 slices)
FP64_PEAK_SOURCE = ("FP64 DFMA: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived from unit counts and clocks; "
                    "nominal 1.25 TFLOP/s; a DFMA microbenchmark on this GB300 reached 1.20 TFLOP/s)")
FP32_PEAK_SOURCE = "FP32 FFMA: 152 SMs x 128/clk x 2 flop x 2.07 GHz (derived from unit counts and clocks)"

# rsvd_info fields (int32 each, in order)
I_STATUS, I_PATH, I_FALLS, I_SWEEPS, I_L, I_ROTS, I_QRCOLS, I_QRKFLOP, I_PAIRS, I_CGIT = range(10)

# DRAM bytes (read + write) per launch of a workload's dominant kernel, from one
# ncu capture of that kernel as it stands (summaries under profiles/); a kernel
# changed since its capture has no entry (traffic null).
# DRAM bytes (read + write) per launch from one ncu capture of the kernel in the named
# workload: the evidence that the kernel reads its operands once (for the Jacobi SVD: the
# central group's launch, 25 bond matrices B of 138 x 256 FP64 = 7.07 MB)
TRAFFIC_PER_LAUNCH = {
    ("mixed", "tcgemm"): (561.69e6 + 16.31e6, "profiles/gram_and_tc_gemm_mixed_bf16_16x4096.md"),
    ("tebd_tfim_L64_chi128_d2_dt0.01_p10_q2_fp64", "jacobi"):
        (7.145e6, "profiles/jacobi_tebd_L64_chi128_ground.md (central group's launch, 25 matrices)"),
}


def traffic_of(workload, kernel):
    t = TRAFFIC_PER_LAUNCH.get((workload, kernel))
    return (t[0], t[1]) if t else (None, None)


def model_name():
    return f"cyl{WIDTH}" if WIDTH else ("tfim" if SPIN == 0.5 else f"spin{SPIN:g}")


def base_config():
    return {"workload": WORKLOAD, "model": model_name(), "L": L_SITES, "chi": CHI, "d": D_LOC, "h": H_FIELD, "dt": DT,
            "p": P_OVER, "q": Q_POW, "update": UPDATE,
            "state": ("ground state: product state evolved by dt = 0.1 x 700, 0.05 x 500, 0.02 x 250 steps"
                      if STATE == "ground" else "early: product state evolved by 20 steps at dt = 0.1"),
            "bond_matrix": (f"{CHI * D_LOC}x{CHI * D_LOC}" if UPDATE == "block" else
                            f"X Y, X {CHI * D_LOC}x{K_TERMS * CHI}, Y {K_TERMS * CHI}x{CHI * D_LOC} (never formed)"),
            "fp64_products_with_A": "tcgen05 tensor cores, exact 9-slice BF16 split, FP64-class error",
            "truncations_per_step": truncations_per_step(), "l2": "flushed (512 MB write) before every timed step"}


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


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


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
# Algorithmic work of one compression, by kernel class, from its device record:
# the Householder QRs' work is reported by the kernels themselves (qr_kflop: the
# standard factorization and explicit-Q counts over the reflectors applied and the
# columns formed), the Jacobi SVD's from its pair, rotation and sweep counts; the
# products with A, the CholeskyQR2 passes and the small GEMMs from the shapes and
# the effective rank the library works on.
def new_flops():
    return {"gemm": 0.0, "gram": 0.0, "cholesky": 0.0, "householder": 0.0, "jacobi": 0.0, "tcgemm": 0.0,
            "ozgemm": 0.0}


def cholqr2_flops(f, rows, l):
    """Two CholeskyQR passes on a rows x l sample: Gram (rows l^2 each, symmetric), Cholesky
    and triangular inverse (2 l^3 / 3 each), Y R^-1 (rows l^2 each)."""
    f["gram"] += 2.0 * rows * l * l
    f["cholesky"] += 2.0 * (2.0 * l ** 3 / 3.0)
    f["gemm"] += 2.0 * rows * l * l


def jacobi_flops(rec, jn, l, want_p):
    """One-sided Jacobi on an l x jn matrix: every sweep's exact row norms (2 jn l, and once
    more at the end), each pair's inner product (2 jn), each rotation (6 jn, and 6 l when the
    rotations are accumulated for U)."""
    sweeps, rots, pairs = int(rec[I_SWEEPS]), int(rec[I_ROTS]), int(rec[I_PAIRS])
    return pairs * 2.0 * jn + rots * (6.0 * jn + (6.0 * l if want_p else 0.0)) + (sweeps + 1) * 2.0 * jn * l


def compression_flops(f, rec, m, n, k, l, q, prec, want_u, full_svd=False, factored_r=0):
    """Add the algorithmic flops of one compression of an m x n matrix (sample width l)
    to f.  prec: "f64" (FP64 products with A on the tensor cores by exact slicing for
    m, n <= 1024, l <= 256), "f32", "bf16", "tf32".  full_svd: Alg. TSVD on the same
    engine (B = A, l = m).  factored_r: A = X Y with inner dimension r (never formed)."""
    f["householder"] += 1e3 * float(rec[I_QRKFLOP])
    exact = full_svd or (m <= l and m <= 16)
    qr_cols = int(rec[I_QRCOLS])
    r = l if want_u or qr_cols <= 0 else min(l, qr_cols)  # columns later products work on
    if not exact:
        if factored_r:
            f["gemm"] += 2.0 * (m + n) * factored_r * l + (2 * q + 1) * 2.0 * (m + n) * factored_r * r
        else:
            cls = "tcgemm" if prec in ("bf16", "tf32") else (
                "ozgemm" if prec == "f64" and m <= 1024 and n <= 1024 and l <= 256 else "gemm")
            f[cls] += 2.0 * m * n * l + (2 * q + 1) * 2.0 * m * n * r
        for it in range(2 * q + 1):
            rows = m if it % 2 == 0 else n
            if not 3 * l > rows:  # CholeskyQR2 (its Householder fallbacks are in qr_kflop)
                cholqr2_flops(f, rows, l)
    jn = n
    if 10 * n >= 30 * l:  # wide B: B^T = Q_b R, M = B Q_b, V^T = W Q_b^T
        if not 3 * l > n:
            cholqr2_flops(f, n, l)
        f["gemm"] += 2.0 * l * n * l + 2.0 * k * l * n
        jn = l
    f["jacobi"] += jacobi_flops(rec, jn, l, want_u)
    if want_u:
        f["gemm"] += 2.0 * m * l * k  # lift U = Q U~


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


def step_flops(info, full_svd=False):
    """Algorithmic FP64 flops of one Trotter step by kernel class, from the device records
    (layer, compression, bond, fields).  Per bond besides the compression: the two-site
    contraction B_i B_{i+1} and the B-tensor update, 2 m n k' each (k' = the columns they
    run over: the nonzero Schmidt values, at most the effective rank)."""
    f = new_flops()
    for j, lay in enumerate(bond_shapes()):
        for w in range(WIDTH if UPDATE == "product" else 1):
            for b, (m, n, k, l) in enumerate(lay):
                rec = info[j][w][b]
                if full_svd:
                    l = m
                qr_cols = int(rec[I_QRCOLS])
                kk = min(k, qr_cols) if qr_cols > 0 else k
                if UPDATE == "product":
                    r = K_TERMS * k
                    f["gemm"] += 2.0 * m * r * r + 2.0 * n * r * r + 2.0 * r * n * kk + 2.0 * m * r * kk
                    compression_flops(f, rec, m, n, k, l, Q_POW, "f64", False, factored_r=r)
                else:
                    f["gemm"] += 4.0 * m * n * kk
                    compression_flops(f, rec, m, n, k, l, Q_POW, "f64", False, full_svd=full_svd)
    return f


def add_flops(a, b):
    for key in a:
        a[key] += b.get(key, 0.0)


# ------------------------------------------------------------------ kernel classes and roofline
def profile_classes(lib):
    import ctypes
    nclass = 16
    ms_c = (ctypes.c_double * nclass)()
    cnt_c = (ctypes.c_int * nclass)()
    ncls = lib.rsvd_profile_collect(ms_c, cnt_c, nclass)
    lib.rsvd_profile_enable(0)
    return {lib.rsvd_profile_class_name(c).decode(): (ms_c[c], cnt_c[c]) for c in range(ncls)}


FP64_CLASSES = ("gram", "cholesky", "householder", "jacobi")


def kernel_table(classes, fl, prec, tcb=0.0, peaks=None):
    """Per kernel class: launch groups, device time, share, and the achieved rate against
    the class's roofline."""
    total = sum(v[0] for v in classes.values()) or 1.0
    out = {}
    for name, (ms, cnt) in classes.items():
        if cnt == 0:
            continue
        e = {"launch_groups": cnt, "ms_total": round(ms, 3), "share": round(ms / total, 4)}
        if ms > 0 and name == "tcgemm" and peaks:
            e["gbs"] = round(tcb / (ms / 1e3) / 1e9, 1)
            e["frac_hbm_peak"] = round(tcb / (ms / 1e3) / 1e9 / peaks["hbm_gbs"], 4)
        elif ms > 0 and name == "ozgemm":
            e["tflops_fp64_equivalent"] = round(fl[name] / (ms / 1e3) / 1e12, 4)
        elif ms > 0 and fl.get(name, 0.0) > 0:
            t = fl[name] / (ms / 1e3) / 1e12
            e["tflops"] = round(t, 4)
            if prec == "f64" or name in FP64_CLASSES:
                e["frac_fp64_peak"] = round(t / FP64_PEAK_TFLOPS, 4)
            else:
                e["frac_fp32_peak"] = round(t / FP32_PEAK_TFLOPS, 4)
        out[name] = e
    return out


def roofline_of(dom, classes, fl, prec, workload, peaks, tcb=0.0):
    """Roofline record of the dominant kernel class: algorithmic work over its measured
    device time (the sum of its launches' CUDA-event durations)."""
    dms = classes[dom][0] / 1e3
    trf, src = traffic_of(workload, dom)
    if dom == "ozgemm":
        tfl = OZ_SLICE_PRODUCTS * fl["ozgemm"] / dms / 1e12 if dms > 0 else 0.0
        return {"bound": "tensor", "kernel": dom, "achieved": round(tfl, 2), "peak": peaks["bf16_tflops"],
                "unit": "TFLOP/s", "frac": round(tfl / peaks["bf16_tflops"], 4), "traffic": trf,
                "traffic_source": src, "peak_source": "MEASURED_PEAKS.json bf16_tflops (of measured)",
                "note": "BF16 flops executed = 53 slice products x the FP64 product's 2 m n l"}
    if dom == "tcgemm":
        return {"bound": "hbm", "kernel": dom, "achieved": round(tcb / dms / 1e9, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(tcb / dms / 1e9 / peaks["hbm_gbs"], 4), "traffic": trf,
                "traffic_source": src, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    fp64 = prec == "f64" or dom in FP64_CLASSES
    pk = FP64_PEAK_TFLOPS if fp64 else FP32_PEAK_TFLOPS
    ach = fl.get(dom, 0.0) / dms / 1e12 if dms > 0 else 0.0
    return {"bound": "alu", "kernel": dom, "achieved": round(ach, 4), "peak": round(pk, 4), "unit": "TFLOP/s",
            "frac": round(ach / pk, 4), "traffic": trf, "traffic_source": src,
            "work": round(fl.get(dom, 0.0), 1), "device_ms": round(classes[dom][0], 4),
            "peak_source": FP64_PEAK_SOURCE if fp64 else FP32_PEAK_SOURCE}


def launches_of(classes):
    # gram and select classes time two launches per recorded group
    return sum(cnt * {"gram": 2, "select": 2}.get(name, 1) for name, (ms, cnt) in classes.items())


# ------------------------------------------------------------------ TEBD (the default line)
def make_chain(tsvd=False, rank=0):
    from paper_1710_01463_gb300.tebd import TebdChain
    return TebdChain(L_SITES, CHI, h=H_FIELD, p=P_OVER, q=Q_POW, seed=SEED + 1000 * rank, S=SPIN, W=WIDTH or None,
                     update=UPDATE, tsvd=tsvd)


def timed_steps(ch, first, steps, flush, stream, infos=None):
    """Run `steps` Trotter steps from step index `first`, each bracketed by CUDA events on
    the launching stream with the L2 flushed before it; returns the per-step durations (ms)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for s in range(steps):
        flush.zero_()
        ev[s][0].record(stream)
        ch.step(first + s)
        ev[s][1].record(stream)
        if infos is not None:
            infos.append(ch.info.clone())
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def run_ours(args):
    import numpy as np
    import torch

    from paper_1710_01463_gb300 import _lib, inputs
    from paper_1710_01463_gb300 import tebd as tebd_mod

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib = _lib.load()
    peaks = measured_peaks()
    t_prep = time.time()
    ch = make_chain(rank=rank)
    state_file = args.state_file + (f".rank{rank}" if ws > 1 else "") if args.state_file else None
    if state_file and os.path.exists(state_file):
        # the prepared state of an earlier run of the same workload (profiling runs)
        z = np.load(state_file)
        if str(z["workload"]) != WORKLOAD:
            raise SystemExit(f"{state_file} holds a state of {z['workload']}, not {WORKLOAD}")
        ch.state_from_host(z["B"], z["lam"])
        nxt = int(z["step"])
    else:
        ch.set_product_state(inputs.product_state_vectors(L_SITES, D_LOC, 102 + rank))
        nxt = ch.evolve(tebd_mod.SCHEDULE_GROUND if STATE == "ground" else tebd_mod.SCHEDULE_EARLY)
        if state_file:
            B_h, lam_h = ch.state_to_host()
            np.savez(state_file, B=B_h, lam=lam_h, step=nxt, workload=WORKLOAD)
    ch.set_dt(DT)
    if args.autotune:  # the first warm-up step times the candidate tiles of every new shape class
        lib.rsvd_autotune_enable(1)
    for s in range(args.warmup):
        ch.step(nxt + s)
        if args.autotune:
            lib.rsvd_autotune_enable(0)
    first = nxt + args.warmup
    torch.cuda.synchronize()
    prep_s = time.time() - t_prep
    state0 = (ch.B.clone(), ch.lam.clone())  # the timed steps' initial state (the TSVD arm starts here too)

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    infos = []
    clocks = ClockSampler(local)
    lib.rsvd_profile_enable(200000)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.time()
    step_ms = timed_steps(ch, first, args.steps, flush, stream, infos)
    wall = time.time() - t0
    clk = clocks.stop()
    classes = profile_classes(lib)
    tot_ms = job_ms(sum(step_ms))
    ms_per_step = tot_ms / args.steps
    value = ws * truncations_per_step() / (ms_per_step / 1e3)
    final_rsvd = (ch.B.clone(), ch.lam.clone())

    fl = new_flops()
    for inf in infos:
        add_flops(fl, step_flops(inf.cpu().numpy()))
    tflops = ws * sum(fl.values()) / (tot_ms / 1e3) / 1e12
    kernels = kernel_table(classes, fl, "f64")
    dom = max(kernels, key=lambda x: kernels[x]["ms_total"])
    roofline = roofline_of(dom, classes, fl, "f64", WORKLOAD, peaks)
    roofline["timing"] = ("sum of the class's launch durations, CUDA events on the launching streams inside the "
                          "timed region (the library's side streams overlap groups of a call)")

    result = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
              "config": dict(base_config(), parallelism=f"replicas{ws}"),
              "tflops": round(tflops, 4), "roofline": roofline, "kernels": kernels,
              "gpu_launches": launches_of(classes), "clocks": clk, "wall_s_timed_loop": round(wall, 3),
              "prep_s": round(prep_s, 1)}
    st = torch.stack(infos).cpu().numpy()
    result["device_status"] = {"max_jacobi_sweeps": int(st[..., I_SWEEPS].max()),
                               "mean_jacobi_sweeps": round(float(st[..., I_SWEEPS].mean()), 3),
                               "householder_fallbacks_per_step": round(float(st[..., I_FALLS].sum()) / args.steps, 2),
                               "mean_qr_columns_256_bonds": round(float(st[..., I_QRCOLS][st[..., I_L] == 138].mean()), 2)
                               if (st[..., I_L] == 138).any() else None,
                               "nonzero_status": int((st[..., I_STATUS] != 0).sum())}
    if rank == 0 and not args.no_extras:
        result["roofline_serial"] = serial_leg(ch, lib, first + args.steps, flush, stream, peaks)
        if UPDATE == "block":  # the engine's TSVD form compresses the formed two-site matrix
            result["tsvd_same_engine"] = tsvd_leg(ch, state0, first, args, flush, stream, ms_per_step)
        ch.B.copy_(final_rsvd[0])
        ch.lam.copy_(final_rsvd[1])
        result["e2e"] = e2e_leg(ch, args)
        result["error"] = error_leg(ch) if UPDATE == "block" else {
            "note": "the product update compresses factored matrices X Y per gate; its factors are checked "
                    "against the oracle in the tests (test_gpu_tebd.py, test_gpu_factored.py)"}
        result["comparator"] = comparator_leg()
        result["cpu_baseline"] = cpu_leg(ch)
        if not args.no_other_configs and UPDATE == "block" and WIDTH == 0 and SPIN == 0.5:
            result["other_configs"] = other_configs(args)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


def serial_leg(ch, lib, first, flush, stream, peaks, steps=2):
    """The same steps with the call's independent groups serialised on one stream
    (RSVD_FLAG_SERIAL, bit-identical results): the kernel classes' device times then add
    up to the step time, and the dominant class's rate is free of overlap."""
    import torch

    from paper_1710_01463_gb300 import _lib
    ch.flags |= _lib.RSVD_FLAG_SERIAL
    infos = []
    lib.rsvd_profile_enable(200000)
    step_ms = timed_steps(ch, first, steps, flush, stream, infos)
    classes = profile_classes(lib)
    ch.flags &= ~_lib.RSVD_FLAG_SERIAL
    fl = new_flops()
    for inf in infos:
        add_flops(fl, step_flops(inf.cpu().numpy()))
    kt = kernel_table(classes, fl, "f64")
    dom = max(kt, key=lambda x: kt[x]["ms_total"])
    r = roofline_of(dom, classes, fl, "f64", WORKLOAD, peaks)
    r["ms_per_step"] = round(sum(step_ms) / steps, 4)
    r["kernel_ms_per_step"] = round(sum(v[0] for v in classes.values()) / steps, 4)
    r["shares"] = {k: v["share"] for k, v in kt.items()}
    r["steps"] = steps
    return r


def tsvd_leg(ch, state0, first, args, flush, stream, rsvd_ms):
    """The timed steps' first few again from the same initial state with Alg. TSVD on the
    same engine (RSVD_FLAG_FULL_SVD: the full Jacobi SVD of each two-site matrix, then
    truncation): the paper's speedup tau = T_TSVD / T_RSVD (Sec. IV) at equal truncation
    (both keep chi values per bond).  The same steps with RSVD (untimed) give the
    comparison of the two arms' Schmidt values and discarded weights."""
    import numpy as np
    import torch
    steps = max(1, min(args.steps, 3))
    ch.B.copy_(state0[0])
    ch.lam.copy_(state0[1])
    for s in range(steps):
        ch.step(first + s)
    torch.cuda.synchronize()
    lam_r = ch.lam.cpu().numpy()
    trunc_r = float(ch.trunc_err.mean())
    tch = make_chain(tsvd=True)
    tch.set_dt(DT)
    # one untimed step warms the TSVD path; then the same step indices from the same state
    tch.B.copy_(state0[0])
    tch.lam.copy_(state0[1])
    tch.step(first)
    torch.cuda.synchronize()
    tch.B.copy_(state0[0])
    tch.lam.copy_(state0[1])
    infos = []
    ms = timed_steps(tch, first, steps, flush, stream, infos)
    t_ms = sum(ms) / steps
    fl = new_flops()
    for inf in infos:
        add_flops(fl, step_flops(inf.cpu().numpy(), full_svd=True))
    st = torch.stack(infos).cpu().numpy()
    return {"kind": "Alg. TSVD on this library's engine (RSVD_FLAG_FULL_SVD): full one-sided Jacobi SVD of "
                    "every two-site matrix, then truncation to chi",
            "value": round(truncations_per_step() / (t_ms / 1e3), 3), "unit": UNIT, "ms_per_step": round(t_ms, 4),
            "steps": steps, "tau_T_tsvd_over_T_rsvd": round(t_ms / rsvd_ms, 3),
            "tflops": round(sum(fl.values()) / (t_ms / 1e3) / 1e12, 4),
            "max_abs_schmidt_diff_rsvd_vs_tsvd": float(np.max(np.abs(lam_r - tch.lam.cpu().numpy()))),
            "mean_discarded_weight_rsvd": trunc_r, "mean_discarded_weight_tsvd": float(tch.trunc_err.mean()),
            "nonzero_status": int((st[..., I_STATUS] != 0).sum()),
            "mean_jacobi_sweeps": round(float(st[..., I_SWEEPS].mean()), 3)}


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
    """Host copy of the center bond's two-site matrix as the layer-A update compresses it:
    theta = lam (row scaling) . gate . (B_i B_{i+1})."""
    import numpy as np
    B = ch.tensors()
    lam = ch.schmidt_values()
    i = (L_SITES // 2 - 1) // 2 * 2  # the layer-A (even) bond at the center
    d = D_LOC
    G = ch.gates[0].cpu().numpy()[ch.layers[0].index(i)].reshape(d, d, d, d)
    two = np.einsum("atb,buc->atuc", B[i], B[i + 1])
    th = np.einsum("stxy,axyc->astc", G, two)
    th = lam[i][:, None, None, None] * th
    return th.reshape(B[i].shape[0] * d, d * B[i + 1].shape[2]), i


def error_leg(ch):
    """Error of the compression on a live bond matrix of the timed state: the GPU RSVD
    (the bond update's parameters) against the exact truncated SVD (numpy LAPACK)."""
    import numpy as np
    import torch
    from paper_1710_01463_gb300 import api
    A, i = center_theta(ch)
    U, S, Vt, info = api.rsvd_truncate(torch.from_numpy(A).cuda(), CHI, P_OVER, Q_POW, SEED, 0)
    torch.cuda.synchronize()
    s_full = np.linalg.svd(A, compute_uv=False)
    u, s, vt = U.cpu().numpy(), S.cpu().numpy(), Vt.cpu().numpy()
    # the residual A - U S V^T in extended precision: the truncation error of this state is
    # near 1e-14 ||A||, within a factor of ten of an FP64 evaluation's own rounding
    xl = np.longdouble
    err = float(np.sqrt(np.sum((A.astype(xl) - (u.astype(xl) * s.astype(xl)) @ vt.astype(xl)) ** 2)))
    dtr = np.sqrt(np.sum(s_full[CHI:] ** 2))
    big = s_full[:CHI] > 1e-8 * s_full[0]
    nrm = float(np.linalg.norm(A))
    # the ratio to the optimal (Eckart-Young) error is reported when that error is above the
    # rounding of the factors themselves (about 1e-15 ||A||)
    meaningful = dtr > 1e-15 * nrm
    return {"bond": f"({i}, {i + 1}), layer A, gate applied", "matrix": f"{A.shape[0]}x{A.shape[1]}",
            "fro_err_over_delta_trunc": float(err / dtr) if meaningful else None,
            "residual_precision": f"numpy longdouble ({np.finfo(xl).precision} digits)",
            "fro_err_over_norm_a": float(err / nrm), "delta_trunc_over_norm_a": float(dtr / nrm),
            "sigma_chi_over_sigma_1": float(s_full[CHI - 1] / s_full[0]),
            "max_rel_sigma_err_above_1e-8": float(np.max(np.abs(s[big] - s_full[:CHI][big]) / s_full[:CHI][big])),
            "max_abs_sigma_err_over_sigma_1": float(np.max(np.abs(s - s_full[:CHI])) / s_full[0])}


def comparator_leg():
    """Full SVD + truncate with torch.linalg.svd (cuSOLVER) FP64 on 32 bond-sized matrices
    (product update: the paper's TSVD of the P form, QR of X then the SVD of the
    (K chi) x (chi d) matrix R Y)."""
    import torch
    from paper_1710_01463_gb300 import inputs
    if UPDATE == "product":
        return product_comparator_leg()
    A = torch.stack([torch.from_numpy(inputs.dense_case(CHI * D_LOC, CHI * D_LOC, seed=300 + j))
                     for j in range(32)]).cuda()
    torch.linalg.svd(A[:2], full_matrices=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    U, S, Vh = torch.linalg.svd(A, full_matrices=False)
    Uk, Sk, Vk = U[..., :CHI].contiguous(), S[..., :CHI].contiguous(), Vh[..., :CHI, :].contiguous()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"kind": f"torch.linalg.svd (cuSOLVER) FP64 + slice to chi, batch of 32 {CHI * D_LOC}x{CHI * D_LOC} "
                    f"matrices", "truncations_per_s": round(32 / (ms / 1e3), 3), "ms_per_truncation": round(ms / 32, 4)}


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
    same workload - layer-A bond updates of the central bonds, from the current GPU
    state, for about 10 s."""
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
# `--workload dense|mixed|sectors|grad`: the other configurations of the path, each as
# its own JSON line (same contract); the default TEBD line carries a short leg of each
# under "other_configs".
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


def build_workload(wl, args, dev, rank=0, batch=None):
    """Seeded synthetic inputs of a configuration, assembled on the device from
    host-seeded orthogonal factors.  Returns (As, ks, p, q, prec, config, extra)."""
    import numpy as np
    import torch
    from paper_1710_01463_gb300 import inputs
    q = 2
    g = torch.Generator(device="cpu").manual_seed(1234 + rank)

    def ortho(nn, seed):
        return torch.from_numpy(inputs.haar_like_orthogonal(nn, seed)).to(dev)

    extra = {}
    if wl == "dense":
        m = n = 256
        k, p, B = 32, 8, batch or 1024
        s = torch.from_numpy(inputs.exp_spectrum(256)).to(dev)
        U0, V0 = ortho(256, 202), ortho(256, 203)
        As = []
        for j in range(B):
            rp, cp = torch.randperm(256, generator=g).to(dev), torch.randperm(256, generator=g).to(dev)
            As.append(((U0[rp] * s[None, :]) @ V0[cp].T).contiguous())
        prec = "f64"
        ks = [k] * B
        config = {"workload": f"dense_fp64_256x256_k32_p8_q2_batch{B}", "m": 256, "n": 256, "k": k, "p": p, "q": q,
                  "batch": B, "spectrum": "s_i = exp(-i/16)",
                  "l2": f"inputs ({B * 0.5:.0f} MB) larger than L2" if B >= 512 else "L2 flushed before every step"}
    elif wl == "mixed":
        m = n = 4096
        k, p, B = 64, 16, batch or 16
        s = torch.from_numpy(inputs.power_spectrum(n, 1.5)).to(dev)
        U0, V0 = ortho(n, 206), ortho(n, 207)
        As = []
        for j in range(B):
            rp, cp = torch.randperm(n, generator=g).to(dev), torch.randperm(n, generator=g).to(dev)
            As.append(((U0[rp] * s[None, :]) @ V0[cp].T).to(
                torch.bfloat16 if args.precision == "bf16" else torch.float32).contiguous())
        del U0, V0
        prec = args.precision
        ks = [k] * B
        config = {"workload": f"ttn_{prec}_4096x4096_k64_p16_q2_batch{B}", "m": m, "n": n, "k": k, "p": p, "q": q,
                  "batch": B, "spectrum": "s_i = i^-1.5", "l2": f"inputs ({B} x 4096^2) larger than L2"}
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
        prec = "f32"
        ks = [min(k, *A.shape) for A in As]
        config = {"workload": "sectors32_64to2048_chi512_fp32_p16_q2", "blocks": 32, "chi_global": 512, "p": p,
                  "q": q, "policy": "maximal k_b = min(chi, m_b, n_b)", "spectrum": "s_i = f_b i^-1.2",
                  "elements": int(sum(A.numel() for A in As)), "l2": "flushed (512 MB write) before every timed step"}
    elif wl == "grad":
        m = n = 1024
        k, p, B = 128, 16, batch or 64
        s = torch.from_numpy(inputs.harmonic_spectrum(n)).to(dev)
        U0, V0 = ortho(n, 208), ortho(n, 209)
        As = []
        for j in range(B):
            rp, cp = torch.randperm(n, generator=g).to(dev), torch.randperm(n, generator=g).to(dev)
            As.append(((U0[rp] * s[None, :]) @ V0[cp].T).float().contiguous())
        rng = np.random.default_rng(105)
        extra["w"] = torch.from_numpy(rng.uniform(0, 1, size=k)).to(dev)
        extra["W"] = torch.from_numpy(rng.standard_normal((n, 8))).float().to(dev)
        prec = "f32"
        ks = [k] * B
        config = {"workload": f"grad_fp32_1024x1024_k128_p16_q2_batch{B}", "m": m, "n": n, "k": k, "p": p, "q": q,
                  "batch": B, "spectrum": "s_i = 1/(1+0.05 i)", "loss": "sum w_i s_i + ||W^T U_k||_F^2, W 1024x8",
                  "l2": f"inputs ({B * 4} MB) larger than L2" if B >= 32 else "L2 flushed before every step"}
    else:
        raise ValueError(wl)
    return As, ks, p, q, prec, config, extra


def workload_leg(wl, args, steps, warmup, extras=True, batch=None):
    """One configuration: timed steps (CUDA events, L2 flushed or inputs above L2), the
    kernel classes and roofline, and (extras) e2e, error, comparator and CPU legs.
    Returns the result dict."""
    import numpy as np
    import torch
    from paper_1710_01463_gb300 import _lib, api
    from oracle import rsvd as orsvd

    ws, rank, local = dist_env()
    lib = _lib.load()
    peaks = measured_peaks()
    dev = torch.device("cuda", local)
    As, ks, p, q, prec, config, extra = build_workload(wl, args, dev, rank, batch)
    dtype = As[0].dtype
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
    adaptive = wl == "sectors" and args.policy in ("adaptive", "adaptive-device")
    devr = args.policy == "adaptive-device"
    if adaptive:
        r0 = [max(1, 512 // len(As))] * len(As)
        plan = api.AdaptiveSectorsPlan([tuple(A.shape) for A in As], 512, r0, p, q, 103 + 1000 * rank, 0, dtype, dev,
                                       device_rounds=devr)
        config["policy"] = ("adaptive: first guess chi / N = 16 every step, the ranks of saturated blocks doubled "
                            "until none is (flops counted for the final round only)"
                            + ("; rounds decided on the device, one launch sequence per step" if devr else
                               "; rounds decided on the host"))
    bw_info = []

    def step():
        if adaptive and not devr:
            plan.ranks = list(r0)
        plan.run(As)
        if wl == "grad":
            Ub = [2.0 * (extra["W"] @ (extra["W"].T @ U)) for U in plan.U]
            Sb = [extra["w"].clone() for _ in plan.S]
            _, binfo = api.rsvd_truncate_backward_batched(As, plan.U, plan.S, plan.Vt, Ub, Sb, None, max_iter=120,
                                                          tol=1e-6)
            bw_info.append(binfo)

    tuned = getattr(args, "autotune", False)
    if tuned:  # the first warm-up step times the candidate tiles of every new shape class
        lib.rsvd_autotune_enable(1)
    for _ in range(warmup):
        step()
        if tuned:
            lib.rsvd_autotune_enable(0)
    torch.cuda.synchronize()
    bw_info.clear()
    if tuned:
        config["gemm_tiles"] = f"measured autotuner ({lib.rsvd_autotune_entries()} shape classes cached in warm-up)"
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    clocks = ClockSampler(local)
    lib.rsvd_profile_enable(400000)
    torch.cuda.synchronize()
    clocks.start()
    infos = []
    above_l2 = sum(A.numel() * A.element_size() for A in As) > 256e6
    for i in range(steps):
        if not above_l2:
            flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        infos.append(plan.info.clone())
    torch.cuda.synchronize()
    clk = clocks.stop()
    classes = profile_classes(lib)
    tot_ms = job_ms(sum(a.elapsed_time(b) for a, b in ev))
    ms_per_step = tot_ms / steps
    units_per_step = 1 if wl == "sectors" else len(As)
    value = ws * units_per_step / (ms_per_step / 1e3)
    if adaptive:
        ks = plan.k_final.cpu().tolist() if devr else list(plan.ranks)

    fl = new_flops()
    tcb = 0.0
    for inf in infos:
        rec = inf.cpu().numpy()
        for j, A in enumerate(As):
            mm, nn = A.shape
            kk = ks[j]
            ll = min(kk + p, mm, nn)
            compression_flops(fl, rec[j], mm, nn, kk, ll, q, prec, True)
            if prec in ("bf16", "tf32"):
                tcb += tc_bytes(mm, nn, ll, q, 2 if prec == "bf16" else 4)
    cg_iters = None
    if wl == "grad":  # backward: retained block, the device-reported CG iterations, the coupling terms (GEMMs)
        cg_iters = []
        for binfo in bw_info:
            rec = binfo.cpu().numpy()
            for j, A in enumerate(As):
                mm, nn = A.shape
                kk = ks[j]
                it = int(rec[j][I_CGIT])
                cg_iters.append(it)
                fl["gemm"] += 2.0 * mm * kk * kk * 2 + 2.0 * mm * nn * kk
                fl["gemm"] += it * (2 * 2.0 * mm * nn * kk + 4 * 2.0 * mm * kk * kk)
                fl["gemm"] += 3 * 2.0 * mm * nn * kk
    kernels = kernel_table(classes, fl, prec, tcb, peaks)
    dom = max(kernels, key=lambda x: kernels[x]["ms_total"])
    roofline = roofline_of(dom, classes, fl, prec, wl, peaks, tcb)
    stat = torch.stack(infos).cpu().numpy()
    result = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": steps,
              "warmup": warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": {"f64": "f64", "f32": "f32", "bf16": "bf16",
                                                                "tf32": "tf32"}[prec],
              "data": "synthetic", "config": dict(config, parallelism=f"replicas{ws}"),
              "tflops": round(ws * sum(fl.values()) / (tot_ms / 1e3) / 1e12, 4), "roofline": roofline,
              "kernels": kernels, "gpu_launches": launches_of(classes), "clocks": clk,
              "device_status": {"max_jacobi_sweeps": int(stat[..., I_SWEEPS].max()),
                                "mean_jacobi_sweeps": round(float(stat[..., I_SWEEPS].mean()), 3),
                                "nonzero_status": int((stat[..., I_STATUS] != 0).sum())}}
    if cg_iters:
        result["device_status"]["cg_iterations_mean"] = round(float(np.mean(cg_iters)), 1)
        result["device_status"]["cg_iterations_max"] = int(np.max(cg_iters))
    if adaptive:
        result["device_status"]["adaptive_rounds"] = int(plan.rounds_dev.item()) if devr else plan.rounds
        result["device_status"]["final_trial_ranks"] = list(ks)
    if rank != 0 or not extras:
        result["error"] = workload_error(wl, As, ks, p, q, plan, extra, orsvd)
        return result
    # e2e: inputs from pinned host memory, results back to the host, every step
    hA = [A.cpu().pin_memory() for A in As]
    hS = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in plan.S]
    nst = max(1, min(steps, 5))
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
    result["error"] = workload_error(wl, As, ks, p, q, plan, extra, orsvd)
    # comparator: full SVD + truncate (cuSOLVER via torch) on matrices 0..3
    cd = torch.float64 if prec == "f64" else torch.float32
    Ac = [A.to(cd) for A in As[:(1 if wl == "mixed" else 4)]]
    torch.linalg.svd(Ac[0], full_matrices=False)
    torch.cuda.synchronize()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record()
    for A in Ac:
        torch.linalg.svd(A, full_matrices=False)
    c1.record()
    torch.cuda.synchronize()
    cms = c0.elapsed_time(c1) / len(Ac)
    result["comparator"] = {"kind": f"torch.linalg.svd (cuSOLVER) {cd} + slice, per matrix",
                            "ms_per_matrix": round(cms, 3), "matrices_per_s": round(1e3 / cms, 3)}
    # CPU oracle on a bounded sample: oracle RSVD of the workload's matrices for about 10 s
    t0 = time.time()
    nrun = 0
    while True:
        orsvd.rsvd(As[nrun % len(As)].double().cpu().numpy(), ks[nrun % len(As)], p, q, 103, nrun)
        nrun += 1
        if time.time() - t0 > 10.0:
            break
    per = (time.time() - t0) / nrun
    cpu_value = (1.0 / (per * len(As))) if wl == "sectors" else 1.0 / per
    result["cpu_baseline"] = {"value": round(cpu_value, 5), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                              "sample": f"{nrun} oracle RSVD(s) of the workload's matrices (numpy FP64, BLAS threads "
                                        f"= all host cores)" + ("; sectors: per-block time x 32" if wl == "sectors"
                                                                else "")}
    return result


def workload_error(wl, As, ks, p, q, plan, extra, orsvd):
    """Error of the timed results: matrix 0 against its exact truncated SVD and against the
    FP64 oracle's Alg. RSVD (same Omega); sectors: the kept counts; grad: the end-to-end
    gradient of the loss against the exact FP64 gradient (full-SVD adjoint) and against
    FP64 central differences along 8 seeded directions, per matrix (two matrices)."""
    import numpy as np
    A0 = As[0].double().cpu().numpy()
    k0 = ks[0]
    sv = np.linalg.svd(A0, compute_uv=False)
    s_gpu = plan.S[0].cpu().numpy()[:k0]
    big = sv[:k0] > 1e-8 * sv[0]
    u0, v0 = plan.U[0][:, :k0].double().cpu().numpy(), plan.Vt[0][:k0].double().cpu().numpy()
    err = np.linalg.norm(A0 - (u0 * s_gpu) @ v0)
    dtr = np.sqrt(np.sum(sv[k0:] ** 2))
    _, so, _ = orsvd.rsvd(A0, k0, p, q, 103, 0)
    out = {"matrix": 0, "fro_err_over_delta_trunc": float(err / dtr) if dtr > 0 else None,
           "max_rel_sigma_err_vs_exact": float(np.max(np.abs(s_gpu[big] - sv[:k0][big]) / sv[:k0][big])),
           "max_abs_sigma_err_vs_fp64_oracle_rsvd_over_sigma1": float(np.max(np.abs(s_gpu - so)) / so[0])}
    if wl == "sectors":
        ko = plan.k_out.cpu().tolist()
        out["k_out"] = ko
        # a trial rank is adequate when the block's last trial value was not selected
        out["trial_ranks_adequate"] = bool(all(kk < kt or kt == min(A.shape) for kk, kt, A in zip(ko, ks, As)))
    if wl == "grad":
        out["gradient"] = grad_error(As, ks, p, q, extra)
    return out


def grad_error(As, ks, p, q, extra, nmat=2, ndir=8):
    """End-to-end FP32 gradient (RSVD forward + the library's backward) of the loss
    sum w_i s_i + ||W^T U_k||^2 against the exact FP64 gradient of the truncated SVD
    (the oracle's full-SVD adjoint) and against FP64 central differences (h = 1e-6) of the
    oracle's loss along `ndir` seeded random directions, per matrix."""
    import numpy as np
    import torch
    from oracle import grad as ograd
    from paper_1710_01463_gb300 import api
    w = extra["w"].cpu().numpy()
    W = extra["W"].double().cpu().numpy()
    rows = []
    for j in range(nmat):
        A = As[j]
        k = ks[j]
        At = A.clone().requires_grad_(True)
        U, S, Vt = api.RSVDTrunc.apply(At, k, p, q, 103, j, 120)
        loss = (extra["w"] * S).sum() + ((extra["W"].T @ U) ** 2).sum()
        loss.backward()
        g = At.grad.double().cpu().numpy()
        Ad = A.double().cpu().numpy()
        ref = ograd.loss_grad(Ad, k, w, W)
        rng = np.random.default_rng(7_000 + j)
        fd_rel = []
        for _ in range(ndir):
            D = rng.standard_normal(Ad.shape)
            D /= np.linalg.norm(D)
            fd = ograd.fd_directional(Ad, k, w, W, D)
            fd_rel.append(abs(float(np.sum(g * D)) - fd) / max(abs(fd), 1e-300))
        row = {"matrix": j, "forward": f"RSVD p={p} q={q}",
               "max_abs_err_over_max_abs_exact": float(np.max(np.abs(g - ref)) / np.max(np.abs(ref))),
               "fro_err_over_fro_exact": float(np.linalg.norm(g - ref) / np.linalg.norm(ref)),
               "fd_directional_rel_err_max": float(max(fd_rel)),
               "fd_directional_rel_err_median": float(np.median(fd_rel))}
        # the same backward behind an exact forward (Alg. TSVD on the library's engine): the
        # deviation above is then that of the RSVD factors, whose retained subspace at this
        # slowly decaying spectrum differs from the exact one, not of the backward
        gt = tsvd_forward_gradient(A, k, extra)
        row["tsvd_forward_fro_err_over_fro_exact"] = float(np.linalg.norm(gt - ref) / np.linalg.norm(ref))
        row["tsvd_forward_max_abs_err_over_max_abs_exact"] = float(np.max(np.abs(gt - ref)) / np.max(np.abs(ref)))
        rows.append(row)
    return rows


def tsvd_forward_gradient(A, k, extra):
    """d loss / d A (FP32) with the exact truncated SVD from the library's engine
    (RSVD_FLAG_FULL_SVD) as the forward and the library's backward."""
    import torch
    from paper_1710_01463_gb300 import _lib, api
    U, S, Vt, info = api.rsvd_truncate(A, k, 0, 0, 0, 0, flags=_lib.RSVD_FLAG_FULL_SVD)
    api.check_info(info, "rsvd_truncate (TSVD)")
    Ub = [2.0 * (extra["W"] @ (extra["W"].T @ U))]
    Sb = [extra["w"].clone()]
    Abar, binfo = api.rsvd_truncate_backward_batched([A], [U], [S], [Vt], Ub, Sb, None, max_iter=300, tol=1e-6)
    api.check_info(binfo, "rsvd_truncate_backward_batched")
    torch.cuda.synchronize()
    return Abar[0].double().cpu().numpy()


def other_configs(args):
    """Short legs of the other configurations, in the same run: value, roofline and error
    each (cfg1 dense FP64, cfg3 mixed BF16, cfg4 sectors FP32, cfg5 FP32 forward + backward
    with its gradient deviation)."""
    import torch
    out = {}
    for wl, steps, batch in (("dense", 5, None), ("mixed", 3, None), ("sectors", 3, None), ("grad", 2, 16)):
        try:
            r = workload_leg(wl, args, steps, 3, extras=False, batch=batch)
            keep = ("value", "unit", "ms_per_step", "steps", "dtype", "config", "tflops", "roofline", "error",
                    "device_status", "gpu_launches", "clocks")
            out[wl] = {k: r[k] for k in keep if k in r}
        except Exception as e:  # a failing leg is reported, not hidden
            out[wl] = {"failed": f"{type(e).__name__}: {e}"}
        torch.cuda.empty_cache()
    return out


def run_workload(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    result = workload_leg(args.workload, args, args.steps, args.warmup, extras=not args.no_extras)
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
    ap.add_argument("--no-other-configs", action="store_true", help="TEBD line without the other configurations")
    ap.add_argument("--workload", default="tebd", choices=["tebd", "dense", "mixed", "sectors", "grad"],
                    help="tebd (default): the TEBD bond-update workload; the others time the remaining configurations")
    ap.add_argument("--state", default="ground", choices=["ground", "early"],
                    help="TEBD: time from the converged ground state (default) or the early state")
    ap.add_argument("--autotune", action="store_true",
                    help="choose the SIMT products' tiles with the library's measured autotuner in the first "
                         "warm-up step (cached choices are used in the timed steps)")
    ap.add_argument("--state-file", default=None,
                    help="TEBD: .npz of the prepared state - loaded if it exists, else written after the "
                         "preparation (lets a profiler run skip the ground-state preparation)")
    ap.add_argument("--precision", default="bf16", choices=["bf16", "tf32"], help="mixed workload: operand precision")
    ap.add_argument("--policy", default="estimate", choices=["estimate", "maximal", "adaptive", "adaptive-device"],
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
    global L_SITES, WORKLOAD, SPIN, WIDTH, D_LOC, H_FIELD, UPDATE, STATE
    if args.chain_length != L_SITES:
        L_SITES = args.chain_length
    SPIN, WIDTH = args.spin, args.cylinder_width
    if args.update == "product" and not WIDTH:
        ap.error("--update product needs --cylinder-width")
    UPDATE = args.update
    STATE = args.state
    D_LOC = 2 ** WIDTH if WIDTH else int(round(2 * SPIN)) + 1
    H_FIELD = args.field if args.field is not None else (3.044 if WIDTH else (1.0 if SPIN == 0.5 else 1.5))
    WORKLOAD = (f"tebd_{model_name()}{'_product' if UPDATE == 'product' else ''}_L{L_SITES}_chi{CHI}_d{D_LOC}"
                f"_dt{DT:g}_p{P_OVER}_q{Q_POW}_fp64" + (f"_h{H_FIELD:g}" if args.field is not None else "")
                + ("_early" if STATE == "early" else ""))
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
