"""Benchmark of the BlockBP message update on one GB300 (or N independent replicas).

One step = one synchronous BlockBP iteration: every message update of the
network (Alg. 1).  Workloads: the translation-periodic Kagome super-cell of
6 x 2 unit cells cut into 3 parallelogram blocks of 12 sites (L = 2), d = 2,
dimer-singlet tensors plus 1e-2 complex Gaussian noise; 12 message updates
per iteration.  Default: D = 6, chi = 64 in TF32 mixed precision
(``--workload kagome-6x2-L2-D6-chi64``); ``--workload kagome-6x2-L2-D4-chi32
--precision fp64`` is the FP64 form at D = 4, chi = 32.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.  `--peaks` measures the
chip's FP64 / FP32 ALU and TF32 / BF16 tensor rates and exits.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "kagome-6x2-L2-D6-chi64": {
        "workload": "kagome-6x2-L2-D6-chi64",
        "lattice": "kagome", "Lx": 6, "Ly": 2, "L": 2, "d": 2, "D": 6, "chi": 64,
        "tensor_seed": 2, "noise": 1e-2, "noise_seed": 3, "message_seed": 7,
        "golden": "kagome_D6_chi64_2it.json",
    },
    "kagome-6x2-L2-D4-chi32": {
        "workload": "kagome-6x2-L2-D4-chi32",
        "lattice": "kagome", "Lx": 6, "Ly": 2, "L": 2, "d": 2, "D": 4, "chi": 32,
        "tensor_seed": 2, "noise": 1e-2, "noise_seed": 3, "message_seed": 7,
        "golden": "kagome_D4_chi32_fixed_point.json",
    },
}
WORKLOAD = WORKLOADS["kagome-6x2-L2-D6-chi64"]


def make_inputs(w):
    import synthetic as syn
    nb = syn.kagome_neighbours(w["Lx"], w["Ly"])
    t = syn.dimer_singlet_peps(nb, w["d"], w["D"], seed=w["tensor_seed"], noise=w["noise"], noise_seed=w["noise_seed"])
    em = syn.initial_edge_matrices(len(nb), w["D"], seed=w["message_seed"])
    return t, em


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- our engine

# Roofline of the dominant kernel class, timed live inside the timed region
# with CUDA events on the streams its launches run on (library-side timer).
KERNELS = {
    "jacobi": (1, "one-sided Jacobi SVD of the reduced matrix (k_jacobi_smem / k_jacobi)"),
    "orth": (2, "Householder panel QR of the range finder and canonical moves (k_panel_qr cluster / k_tsqr_reg)"),
    "qr": (3, "Householder QR of the canonical moves and distances (k_tsqr_reg / k_tsqr_smem)"),
    "tc": (4, "tcgen05 split-precision GEMM: the absorb contraction and the segment merges (k_tc_gemm)"),
    "absorb": (5, "SIMT complex absorb GEMM (k_gemm)"),
    "gemm": (6, "every SIMT complex GEMM (k_gemm)"),
}

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# ncu captures of the kernel cases below, keyed by (kernel class, workload,
# precision); an entry is removed when its kernel changes.
TRAFFIC = {
    ("orth", "kagome-6x2-L2-D6-chi64", "tf32"): {
        "bytes": 1.84e6,
        "note": "one 2304 x 96 complex64 panel with Q (bench.py --kernel-case panel): DRAM read 1.84 MB, write 0 "
                "(the 1.8 MB of Q stays in L2)"},
    ("tc", "kagome-6x2-L2-D6-chi64", "tf32"): {
        "bytes": 588.3e6,
        "note": "one absorb GEMM at P = Q = 1296, l = r = 64 (bench.py --kernel-case absorb): DRAM read 549.5 MB + "
                "write 38.9 MB against 250.5 MB of operands and output"},
}

# TF32 / BF16 dense tensor rates of the part, nominal (for the ratio only)
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25


def peaks():
    """Roofline denominators: the measured BF16 burst rate (MEASURED_PEAKS.json), TF32 at the
    nominal TF32 / BF16 ratio of the part; the FP32 and FP64 ALU rates from
    unit counts and the maximum clock (152 SMs x 128 FP32 lanes, x 2 FP64
    FMA per clock, 2.07 GHz), which the FMA microbenchmark of `--peaks`
    reproduces (77.7 and 1.25 TFLOP/s measured)."""
    bf16 = 1911.2
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f).get("bf16_tflops", bf16))
    except (OSError, ValueError):
        pass
    return {"fp32": 152 * 128 * 2 * 2.07e9 / 1e12, "fp64": 152 * 2 * 2 * 2.07e9 / 1e12, "bf16": bf16,
            "tf32": bf16 * NOMINAL_TF32_OVER_BF16, "fp32_kind": "unit counts x 2.07 GHz",
            "fp64_kind": "unit counts x 2.07 GHz"}


def max_over_ranks(x: float, world: int) -> float:
    """The largest x over all ranks (a replicated job takes as long as its
    slowest rank); works on whichever backend the process group uses."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def accuracy_vs_oracle(P, w, prec):
    """Observables of a fresh context against the FP64 oracle's stored values
    (tests/golden, written from oracle/ alone): every <S^z_i> and the stored
    bonds' <S_i . S_j>, after the same iterations the oracle ran (two from the
    initial messages, or its fixed point)."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", w["golden"])
    if not os.path.exists(path):
        return None
    with open(path) as f:
        g = json.load(f)
    t, em = make_inputs(w)
    ctx = P.bbp_create_peps(P.KAGOME, w["Lx"], w["Ly"], 1, w["d"], w["D"], t)
    try:
        P.bbp_partition_blocks(ctx, w["L"], w["L"])
        P.bbp_set_options(ctx, w["chi"], prec)
        P.bbp_init_messages(ctx, em)
        if "tol" in g:
            tol = g["tol"] if prec == P.FP64 else 1e-5
            it, err, _ = P.bbp_iterate(ctx, tol, 30)
        else:
            it, err, _ = P.bbp_iterate(ctx, 0.0, g["iterations"])
        sz = np.diag([0.5, -0.5]).astype(np.complex128)
        dsz = max(abs(P.bbp_expect_local(ctx, sz, [i]).real - g["sz"][i][0]) for i in range(len(g["sz"])))
        be = P.bbp_bond_energies(ctx, [(b[0], b[1]) for b in g["bonds"]])
        dss = max(abs(x - v[0]) for x, v in zip(be, g["bond_energy"]))
        out = {"iterations": it, "oracle_iterations": g["iterations"], "max_abs_d_sz": dsz, "n_sites": len(g["sz"]),
               "max_abs_d_bond_energy": dss, "n_bonds": len(g["bonds"]), "oracle": "FP64 oracle, " + w["golden"]}
        if "energy_per_site" in g:
            out["abs_d_energy_per_site"] = abs(P.bbp_energy_per_site(ctx) - g["energy_per_site"])
        return out
    finally:
        P.bbp_destroy(ctx)


def run_ours(args, rank, world):
    import numpy as np
    import torch
    import paper_2603_13304_gb300 as P

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    P.build()
    P.use_torch_allocator()
    w = WORKLOADS[args.workload]
    t, em = make_inputs(w)
    stream = torch.cuda.current_stream()
    prec = {"tf32": P.TF32, "bf16": P.BF16, "fp32": P.FP32, "fp64": P.FP64}[args.precision]

    def setup():
        ctx = P.bbp_create_peps(P.KAGOME, w["Lx"], w["Ly"], 1, w["d"], w["D"], t)
        P.bbp_partition_blocks(ctx, w["L"], w["L"])
        P.bbp_set_options(ctx, w["chi"], prec)
        P.bbp_set_execution(ctx, not args.no_graphs, 16)
        P.bbp_init_messages(ctx, em)
        return ctx

    cls, kdesc = KERNELS[args.roofline_kernel]
    ctx = setup()
    _, n_updates, n_sites = P.bbp_info(ctx)
    # settle: from the bond-1 initial messages the bond dimensions grow for a
    # few iterations; iterate until the work per iteration stops changing
    prev = None
    for _ in range(12):
        P.bbp_iterate(ctx, 0.0, 1)
        cur = P.bbp_stats(ctx)
        if cur == prev:
            break
        prev = cur
    for _ in range(args.warmup):
        P.bbp_iterate(ctx, 0.0, 1)
    # L2 flush buffer (larger than the 126 MB L2), rewritten between timed steps
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    flush.zero_()                         # loads the fill kernel before the timed region
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0 = time.perf_counter()
        torch.cuda.nvtx.range_push("timed")     # lets a profiler select the timed launches
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        e0.record(stream)
        for i in range(args.steps):
            flush.zero_()
            marks[i].record(stream)
            P.bbp_iterate(ctx, 0.0, 1)
        marks[args.steps].record(stream)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        host_secs = time.perf_counter() - h0
    secs = e0.elapsed_time(e1) * 1e-3
    step_ms = [marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps)]
    launches, flops_iter = P.bbp_stats(ctx)
    # second pass, same steps, with the dominant kernel class bracketed by
    # CUDA events on its own streams (events in the graph perturb the step,
    # so the headline value above is taken without them)
    def timer_pass(c):
        P.bbp_ktimer_select(c)
        P.bbp_set_execution(ctx, not args.no_graphs, 16)   # recapture with the event nodes
        P.bbp_iterate(ctx, 0.0, 1)
        P.bbp_ktimer_read()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            P.bbp_iterate(ctx, 0.0, 1)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t1
        out = P.bbp_ktimer_read() + (dt,)
        P.bbp_ktimer_select(0)
        return out

    k_n, k_ms, k_flops, timer_pass_secs = timer_pass(cls)
    # the tensor-core GEMM beside the dominant kernel, in the tensor modes
    tc_pass = timer_pass(KERNELS["tc"][0]) if (args.precision in ("tf32", "bf16") and args.roofline_kernel != "tc") \
        else None
    secs = max_over_ranks(secs, world)
    value = world * n_updates * args.steps / secs
    energy = P.bbp_energy_per_site(ctx) if rank == 0 else None
    P.bbp_destroy(ctx)

    # end to end through the C ABI with host buffers: upload, iterate, read back
    tp = torch.from_numpy(np.ascontiguousarray(t)).pin_memory()
    ep = torch.from_numpy(np.ascontiguousarray(em)).pin_memory()
    n_e2e = args.warmup + args.steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = P.bbp_create_peps(P.KAGOME, w["Lx"], w["Ly"], 1, w["d"], w["D"], tp.numpy())
    P.bbp_partition_blocks(ctx, w["L"], w["L"])
    P.bbp_set_options(ctx, w["chi"], prec)
    P.bbp_init_messages(ctx, ep.numpy())
    P.bbp_iterate(ctx, 0.0, n_e2e)
    d2h = 0
    for b in range(3):
        for f in range(4):
            msg = P.bbp_get_message(ctx, b, f)
            d2h += sum(x.nbytes for x in msg)
    torch.cuda.synchronize()
    e2e_secs = time.perf_counter() - t0
    P.bbp_destroy(ctx)
    e2e = {"value": n_updates * n_e2e / e2e_secs, "unit": "message updates/s",
           "h2d_bytes_per_step": (t.nbytes + em.nbytes) / n_e2e, "d2h_bytes_per_step": d2h / n_e2e,
           "iterations": n_e2e, "note": "create, upload, init, all iterations from the initial messages, read back"}

    acc = accuracy_vs_oracle(P, w, prec) if rank == 0 else None

    def roofline(kname, k_n, k_ms, k_flops, pass_secs):
        pk = peaks()
        tensor = kname == "tc"
        bound, unit = ("tensor", "TFLOP/s") if tensor else ("alu", "TFLOP/s")
        key = (args.precision if args.precision in ("tf32", "bf16") else "tf32") if tensor else (
            "fp64" if args.precision == "fp64" else "fp32")
        per_launch_s = k_ms * 1e-3 / k_n
        # the library credits each launch with its algorithmic complex flops;
        # the split tensor-core operands execute three real products per
        # complex product in TF32 (six in BF16)
        split = (6.0 if args.precision == "bf16" else 3.0) if tensor else 1.0
        achieved = k_flops / k_n / per_launch_s / 1e12
        tr = TRAFFIC.get((kname, args.workload, args.precision))
        r = {"bound": bound, "achieved": achieved, "peak": pk[key], "unit": unit, "frac": achieved / pk[key],
             "traffic": tr["bytes"] if tr else None, "kernel": KERNELS[kname][1],
             "peak_kind": (key + " dense, of measured (bf16 burst x nominal tf32/bf16 ratio)" if key == "tf32"
                           else "bf16 dense burst, of measured") if tensor else key + ", " + pk[key + "_kind"],
             "flops_kind": "algorithmic complex flops (8 per complex multiply-add)",
             "executed_tensor_frac": achieved * split / pk[key] if tensor else None,
             "launches_per_step": k_n / args.steps, "launch_us": per_launch_s * 1e6,
             "kernel_ms_per_step_all_streams": k_ms / args.steps,
             "timer_pass_ms_per_step": 1e3 * pass_secs / args.steps}
        if tr:
            r["traffic_note"] = tr["note"]
        if not tensor:
            r["frac_of_one_sm"] = achieved / (pk[key] / 152)
        return r

    roof = roofline(args.roofline_kernel, k_n, k_ms, k_flops, timer_pass_secs) if rank == 0 and k_n > 0 else None
    roof_tc = roofline("tc", *tc_pass) if rank == 0 and tc_pass and tc_pass[0] > 0 else None
    return {
        "value": value, "secs": secs, "host_secs": host_secs, "step_ms": step_ms, "n_updates": n_updates, "n_sites": n_sites, "energy": energy,
        "clocks": clk.summary(), "launches": launches, "flops_iter": flops_iter, "e2e": e2e, "roofline": roof,
        "roofline_tc": roof_tc, "accuracy": acc,
    }


def run_core(workload: str, precision: int, reps: int = 3):
    """Core extraction (Sec. 2.3) at a Kagome workload: once the messages have
    settled, the pMPS around the unit cell (up-triangle A, B, C of the
    block's first cell) of every block, each timed over `reps` calls of
    bbp_core_pmps (two bubbles, the zipper, the copy of the pMPS to the host)
    with CUDA events on the context's stream."""
    import torch
    import paper_2603_13304_gb300 as P
    w = WORKLOADS[workload]
    t, em = make_inputs(w)
    ctx = P.bbp_create_peps(P.KAGOME, w["Lx"], w["Ly"], 1, w["d"], w["D"], t)
    P.bbp_partition_blocks(ctx, w["L"], w["L"])
    P.bbp_set_options(ctx, w["chi"], precision)
    P.bbp_init_messages(ctx, em)
    prev = None
    for _ in range(12):                # until the work per iteration stops changing
        P.bbp_iterate(ctx, 0.0, 1)
        cur = P.bbp_stats(ctx)
        if cur == prev:
            break
        prev = cur
    n_blocks = P.bbp_info(ctx)[0]
    cells = [[3 * (b * w["L"]) + k for k in range(3)] for b in range(n_blocks)]   # cell (b L, 0): A, B, C
    for b, c in enumerate(cells):      # warm-up (first use of the raw plans and scratch)
        P.bbp_core_pmps(ctx, b, c)
    stream = torch.cuda.current_stream()
    ms, ring_len, bonds = [], 0, 0
    for b, c in enumerate(cells):
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ring, legs, _ = P.bbp_core_pmps(ctx, b, c)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        ring_len = len(ring)
        bonds = max(bonds, max(x.shape[0] for x in ring))
    # local quantities from the core: <S^z> of site A (one-site core) and
    # <S_A . S_B> (the A-B bond's Edge TN, three product insertions)
    import numpy as np
    sz = np.diag([0.5, -0.5]).astype(np.complex128)
    sx = np.array([[0, 0.5], [0.5, 0]], dtype=np.complex128)
    sy = np.array([[0, -0.5j], [0.5j, 0]], dtype=np.complex128)
    site_ms, bond_ms, bond_e = [], [], []
    for b, c in enumerate(cells):
        for _ in range(reps):
            torch.cuda.synchronize()
            a0 = time.perf_counter()
            P.bbp_core_expect(ctx, b, c[:1], [[sz]])
            torch.cuda.synchronize()
            site_ms.append(1e3 * (time.perf_counter() - a0))
            a0 = time.perf_counter()
            e = P.bbp_core_expect(ctx, b, c[:2], [[s, s] for s in (sx, sy, sz)])
            torch.cuda.synchronize()
            bond_ms.append(1e3 * (time.perf_counter() - a0))
        bond_e.append(float(np.sum(e).real))
    P.bbp_destroy(ctx)
    ms.sort()
    site_ms.sort()
    bond_ms.sort()
    return {"workload": workload, "core": "unit cell (up-triangle A, B, C) of each block",
            "cores_timed": len(cells), "calls": len(ms), "ms_per_core_median": ms[len(ms) // 2],
            "ms_per_core_min": ms[0], "pmps_tensors": ring_len, "pmps_bond_max": bonds,
            "note": "two bubbles from the bottom and top faces, zipper into the pMPS, copy to host memory",
            "site_expect_ms_median": site_ms[len(site_ms) // 2],
            "bond_energy_ms_median": bond_ms[len(bond_ms) // 2],
            "bond_energy_AB": bond_e,
            "expect_note": "bbp_core_expect: pMPS of a one-site core or of the A-B bond (Edge TN) and its exact "
                           "contraction with the fused core tensors, host time per call"}


def run_ite(workload: str = "kagome-6x2-L2-D4-chi32", settle: int = 4, dt: float = 0.05, sweeps: int = 10,
            max_updates: int = 0):
    """ITE with ALS (Ch. 3) at a Kagome workload in the FP64 mode: after
    `settle` BlockBP iterations, one ITE update of the A-B bond of each
    block's first unit cell (the bond's Edge TN, its dense environment, the
    gate exp(-dt S.S), ALS of at most `sweeps` sweeps, the tensors replaced),
    host time per update."""
    import numpy as np
    import torch
    import paper_2603_13304_gb300 as P
    w = WORKLOADS[workload]
    t, em = make_inputs(w)
    ctx = P.bbp_create_peps(P.KAGOME, w["Lx"], w["Ly"], 1, w["d"], w["D"], t)
    P.bbp_partition_blocks(ctx, w["L"], w["L"])
    P.bbp_set_options(ctx, w["chi"], P.FP64)
    P.bbp_init_messages(ctx, em)
    P.bbp_iterate(ctx, 0.0, settle)
    s = [np.array([[0, 0.5], [0.5, 0]]), np.array([[0, -0.5j], [0.5j, 0]]), np.diag([0.5, -0.5])]
    h = sum(np.kron(a, a) for a in s)
    ev, V = np.linalg.eigh(h)
    gate = (V * np.exp(-dt * ev)) @ V.conj().T          # the input gate exp(-dt h)
    n_blocks = P.bbp_info(ctx)[0]
    if max_updates:
        n_blocks = min(n_blocks, max_updates)
    ms, phis = [], []
    for b in range(n_blocks):
        site = 3 * (b * w["L"])                          # A of cell (b L, 0); slot 0 joins B of the same cell
        torch.cuda.synchronize()
        a0 = time.perf_counter()
        phi = P.bbp_ite_bond(ctx, site, 0, gate, max_sweeps=sweeps)
        torch.cuda.synchronize()
        ms.append(1e3 * (time.perf_counter() - a0))
        phis.append([float(phi[0]), float(phi[-1]), len(phi)])
    P.bbp_destroy(ctx)
    ms.sort()
    return {"workload": workload, "precision": "fp64", "settle_iterations": settle, "dt": dt,
            "bond": "A-B of each block's first unit cell", "updates": len(ms), "ms_per_update_median": ms[len(ms) // 2],
            "ms_per_update_min": ms[0], "phi_start_end_halfsteps": phis,
            "note": "Edge TN (two bubbles + zipper), dense environment over the six outer legs (4^12 entries), "
                    "gate, SVD start, ALS half-steps, tensors replaced; host time per bbp_ite_bond"}


# -------------------------------------------------- many networks, serving

def network_mix(n, seed):
    """The batched mix: n independent networks, each square (open 2b x 2b
    lattice cut into four b x b blocks, b uniform in 2..4) or Kagome (the
    periodic 3L x L super-cell cut into three L x L blocks of 3 L^2 sites, L
    uniform in 2..4) with equal odds; D uniform in 2..6, chi uniform in
    {8, 16, 32, 64}; complex64 site tensors, i.i.d. complex Gaussian (seeded)
    normalised by their largest singular value."""
    import numpy as np
    import synthetic as syn
    import paper_2603_13304_gb300 as P
    rng = np.random.default_rng(seed)
    jobs = []
    for _ in range(n):
        kagome = bool(rng.integers(2))
        size = int(rng.integers(2, 5))
        D = int(rng.integers(2, 7))
        chi = int(rng.choice([8, 16, 32, 64]))
        s = int(rng.integers(1 << 30))
        if kagome:
            Lx, Ly, bx = 3 * size, size, size
            n_sites = 3 * Lx * Ly
            jobs.append(dict(lattice=P.KAGOME, Lx=Lx, Ly=Ly, periodic=1, bx=bx, by=bx, D=D, chi=chi,
                             kind=f"kagome L={size}"))
        else:
            Lx = Ly = 2 * size
            n_sites = Lx * Ly
            jobs.append(dict(lattice=P.SQUARE, Lx=Lx, Ly=Ly, periodic=0, bx=size, by=size, D=D, chi=chi,
                             kind=f"square {size}x{size} blocks"))
        jobs[-1]["t"] = syn.gaussian_peps(n_sites, 2, D, seed=s).astype(np.complex64)
        jobs[-1]["em"] = syn.initial_edge_matrices(n_sites, D, seed=s + 1)
    return jobs


def make_network(P, j, precision, streams, fuse_cache=None):
    c = P.bbp_create_peps(j["lattice"], j["Lx"], j["Ly"], j["periodic"], 2, j["D"], j["t"])
    P.bbp_partition_blocks(c, j["bx"], j["by"])
    if fuse_cache is not None:
        P.bbp_set_fuse_cache(c, fuse_cache)
    P.bbp_set_options(c, j["chi"], precision)
    P.bbp_set_execution(c, True, streams)
    P.bbp_init_messages(c, j["em"])
    return c


def run_batched(n_networks, steps, warmup, precision, seed=4, groups=0):
    """One synchronous iteration of every one of n_networks independent
    networks per round (bbp_batch_iterate: the replayed iterations of a round
    go out as one graph launch), with the tensor-core tiles autotuned on the
    shapes recorded while the bond dimensions settle; beside it the same
    networks one at a time (bbp_iterate on a sample of every 8th network)."""
    import torch
    import paper_2603_13304_gb300 as P
    t0 = time.perf_counter()
    jobs = network_mix(n_networks, seed)
    # every site fused right before its absorb (nothing cached), 2 worker
    # streams a network; networks are added while 24 GB of HBM stay free (the
    # worker arenas come at the first iteration: with `groups` pools they
    # take groups x the largest arena, else one arena set per network)
    ctxs = []
    for j in jobs:
        if torch.cuda.mem_get_info()[0] < 24e9:
            break
        ctxs.append(make_network(P, j, precision, 2, fuse_cache=0))
    jobs = jobs[:len(ctxs)]
    n_networks = len(ctxs)
    n_updates = sum(P.bbp_info(c)[1] for c in ctxs)
    if groups:
        P.bbp_share_workers(ctxs, groups)
    setup_s = time.perf_counter() - t0
    def note(msg):                     # progress on stderr (the JSON line goes to stdout)
        print(f"[batched] {time.perf_counter() - t0:7.1f} s  {msg}", file=sys.stderr, flush=True)

    note(f"{n_networks} networks created, {groups or n_networks} worker pools")
    P.bbp_autotune_record(True)
    prev = None
    settle = 0
    for settle in range(1, 9):         # until the work of every network stops changing
        rc, _, _, st = P.bbp_batch_iterate(ctxs, 0.0, 1)
        cur = [P.bbp_stats(c) for c in ctxs]
        note(f"settle round {settle}: status {rc}, {sum(1 for x in st if x not in (0, 6))} failed")
        if cur == prev:
            break
        prev = cur
    P.bbp_autotune_record(False)
    t1 = time.perf_counter()
    tuned = P.bbp_autotune_run()
    tune_s = time.perf_counter() - t1
    note(f"autotuned {tuned} shapes in {tune_s:.1f} s")
    for w in range(warmup):            # recapture with the tuned tiles, build the round's graph
        P.bbp_batch_iterate(ctxs, 0.0, 1)
        note(f"warm-up round {w + 1}")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0 = time.perf_counter()
    e0.record()
    for _ in range(steps):
        rc, _, _, st = P.bbp_batch_iterate(ctxs, 0.0, 1)
    e1.record()
    torch.cuda.synchronize()
    host = time.perf_counter() - h0
    secs = max(e0.elapsed_time(e1) * 1e-3, host)
    failed = int(sum(1 for x in st if x not in (0, 6)))
    note(f"{steps} timed rounds: {secs:.1f} s")
    # one network at a time, on every 8th network (each settled and captured)
    sample = list(range(0, n_networks, 8))
    seq_updates, seq_secs = 0, 0.0
    for i in sample:
        P.bbp_iterate(ctxs[i], 0.0, 1)     # (instantiates its own graph)
        torch.cuda.synchronize()
        a = time.perf_counter()
        P.bbp_iterate(ctxs[i], 0.0, 1)
        torch.cuda.synchronize()
        seq_secs += time.perf_counter() - a
        seq_updates += P.bbp_info(ctxs[i])[1]
    used = torch.cuda.mem_get_info()
    for c in ctxs:
        P.bbp_destroy(c)
    P.bbp_autotune_clear()
    kinds = {}
    for j in jobs:
        kinds[j["kind"]] = kinds.get(j["kind"], 0) + 1
    return {"networks": n_networks, "message_updates_per_round": n_updates, "rounds": steps,
            "value": n_updates * steps / secs, "unit": "message updates/s", "ms_per_round": 1e3 * secs / steps,
            "launch": "one graph launch per round (every network's iteration graph a child)",
            "worker_pools": groups or n_networks,
            "failed_networks": failed, "settle_rounds": settle, "autotuned_shapes": tuned,
            "autotune_s": round(tune_s, 2), "setup_s": round(setup_s, 2),
            "chi_below_D2_fraction": sum(1 for j in jobs if j["chi"] < j["D"] ** 2) / n_networks,
            "hbm_used_gb": round((used[1] - used[0]) / 1e9, 1),
            "one_at_a_time": {"value": seq_updates / seq_secs, "unit": "message updates/s",
                              "sample": f"bbp_iterate on {len(sample)} networks (every 8th), one iteration each"},
            "mix": ("square 2b x 2b open (b x b blocks, b 2..4) and Kagome 3L x L (L x L blocks, L 2..4); D 2..6, "
                    f"chi 8/16/32/64; complex64 Gaussian tensors; seed {seed}; 2 streams per network"),
            "kinds": kinds}


def job_mix(n, seed, precision, max_D=4, chis=(8, 16, 32)):
    """A seeded mix of small BlockBP problems: square 4x4 (2x2 blocks) and
    6x6 (3x3 blocks) open lattices with i.i.d. Gaussian tensors normalised
    by their largest singular value, and the Kagome 6x2 super-cell (L = 2)
    near a random dimer-singlet state with 1e-2 noise; D uniform in
    2..max_D, chi uniform in `chis`."""
    import numpy as np
    import synthetic as syn
    import paper_2603_13304_gb300 as P
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(n):
        kind = rng.integers(3)
        D = int(rng.integers(2, max_D + 1))
        chi = int(rng.choice(chis))
        s = int(rng.integers(1 << 30))
        if kind == 0:
            t = syn.gaussian_peps(16, 2, D, seed=s)
            jobs.append(dict(lattice=P.SQUARE, Lx=4, Ly=4, periodic=0, bx=2, by=2, D=D, chi=chi, t=t,
                             em=syn.initial_edge_matrices(16, D, seed=s + 1)))
        elif kind == 1:
            t = syn.gaussian_peps(36, 2, D, seed=s)
            jobs.append(dict(lattice=P.SQUARE, Lx=6, Ly=6, periodic=0, bx=3, by=3, D=D, chi=chi, t=t,
                             em=syn.initial_edge_matrices(36, D, seed=s + 1)))
        else:
            nb = syn.kagome_neighbours(6, 2)
            t = syn.dimer_singlet_peps(nb, 2, D, seed=s, noise=1e-2, noise_seed=s + 1)
            jobs.append(dict(lattice=P.KAGOME, Lx=6, Ly=2, periodic=1, bx=2, by=2, D=D, chi=chi, t=t,
                             em=syn.initial_edge_matrices(36, D, seed=s + 2)))
        jobs[-1]["precision"] = precision
    return jobs


def serving_pool(n, seed):
    """Job templates of the serving stream: the batched network mix plus 10 %
    Kagome D = 6, chi = 64 jobs (the 6 x 2 super-cell, L = 2, a random
    dimer-singlet state plus 1e-2 noise, complex64)."""
    import numpy as np
    import synthetic as syn
    import paper_2603_13304_gb300 as P
    rng = np.random.default_rng(seed)
    base = network_mix(n, seed)
    pool = []
    for j in base:
        if rng.random() < 0.1:
            s = int(rng.integers(1 << 30))
            nb = syn.kagome_neighbours(6, 2)
            t = syn.dimer_singlet_peps(nb, 2, 6, seed=s, noise=1e-2, noise_seed=s + 1).astype(np.complex64)
            j = dict(lattice=P.KAGOME, Lx=6, Ly=2, periodic=1, bx=2, by=2, D=6, chi=64, t=t,
                     em=syn.initial_edge_matrices(36, 6, seed=s + 2), kind="kagome L=2 D=6 chi=64")
        pool.append(j)
    return pool


def run_serving(duration_s, rate, precision, tol=1e-8, max_iter=30, warm_s=5.0, drain_s=None, pool_n=16, seed=5,
                fp64_sample=8, max_active=32, fp64_baseline=True):
    """Poisson arrivals (seed `seed`) at `rate` jobs/s for warm_s + duration_s
    seconds of job templates drawn from serving_pool; each job runs to `tol`
    or `max_iter` iterations on the continuous-batching server (messages
    resident, admission by HBM footprint).  Latency is reported for jobs
    that arrive after the warm-up and finish within drain_s of the last
    arrival; the rest are counted as unfinished.  Beside it: one job at a
    time in FP64, as a FIFO queue over the same arrival trace whose service
    times are measured per template (FP64 time per iteration x the
    iterations the template needed when served), and the energy error of
    served jobs against FP64 runs of the same template to the same stopping
    rule, on `fp64_sample` templates."""
    import numpy as np
    import torch
    import paper_2603_13304_gb300 as P
    pool = serving_pool(pool_n, seed)
    rng = np.random.default_rng(seed)
    horizon = warm_s + duration_s
    arrivals = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > horizon:
            break
        arrivals.append((t, int(rng.integers(pool_n))))
    jobs_spec = [P.make_job(j["lattice"], j["Lx"], j["Ly"], j["periodic"], 2, j["D"], j["bx"], j["by"], j["chi"],
                            precision, j["t"], j["em"], tol, max_iter, 2, 1) for j in pool]
    free, _ = torch.cuda.mem_get_info()
    srv = P.bbp_server_create(int(free * 0.8), max_active)
    lat, iters, stat, sub = {}, {}, {}, {}
    energy = {}
    t0 = time.perf_counter()
    nxt = 0
    ids = {}
    served_e = {}
    if drain_s is None:
        drain_s = min(120.0, 2.0 * duration_s + 30.0)
    deadline = horizon + drain_s
    while True:
        now = time.perf_counter() - t0
        while nxt < len(arrivals) and arrivals[nxt][0] <= now:
            ids[P.bbp_server_submit(srv, jobs_spec[arrivals[nxt][1]])] = nxt
            nxt += 1
        q, a, f = P.bbp_server_step(srv, 2.0)
        for r in P.bbp_server_poll(srv):
            k = ids[r["id"]]
            lat[k], iters[k], stat[k] = r["latency_s"], r["iters"], r["status"]
            tpl = arrivals[k][1]
            if tpl not in served_e and r["status"] in (0, 6):
                ctx = P.bbp_server_take(srv, r["id"], keep_context=True)
                served_e[tpl] = (P.bbp_energy_per_site(ctx), r["iters"], r["err"])
                P.bbp_destroy(ctx)
            else:
                P.bbp_server_take(srv, r["id"])
        if nxt >= len(arrivals) and (len(lat) == len(arrivals) or now > deadline):
            break
    wall = time.perf_counter() - t0
    P.bbp_server_destroy(srv)
    measured = [k for k in range(len(arrivals)) if arrivals[k][0] >= warm_s]
    done = [k for k in measured if k in lat]
    # unfinished jobs enter the percentiles with their age at the end of the
    # run (a lower bound of their latency)
    L = np.array([lat[k] if k in lat else wall - arrivals[k][0] for k in measured]) if measured else np.zeros(1)
    conv = sum(1 for k in done if stat[k] == 0)
    # FP64 one at a time: service time per template, FIFO over the same trace
    prec64 = 0
    svc = {}
    e64 = {}
    e64_detail = []
    tpl_iters = {}
    for k in done:
        tpl_iters.setdefault(arrivals[k][1], iters[k])
    sample = sorted(served_e)[:fp64_sample]
    for tpl in (sorted(set(a[1] for a in arrivals)) if fp64_baseline else []):
        j = pool[tpl]
        c = make_network(P, j, prec64, 16)
        per_it = float("nan")
        try:
            # iterations until the work settles (the bond dimensions grow
            # from the initial messages), the last one timed; at most 5, and
            # none after 20 s (the last time then bounds the settled one
            # from below)
            prev = None
            spent = 0.0
            for _ in range(5):
                if spent > 20.0:
                    break
                torch.cuda.synchronize()
                a0 = time.perf_counter()
                P.bbp_iterate(c, 0.0, 1)
                torch.cuda.synchronize()
                per_it = time.perf_counter() - a0
                spent += per_it
                cur = P.bbp_stats(c)
                if cur == prev:
                    break
                prev = cur
        except P.BBPError:
            pass
        P.bbp_destroy(c)
        svc[tpl] = per_it * tpl_iters.get(tpl, max_iter)
        if tpl in sample and served_e[tpl][1] <= 40 and per_it * served_e[tpl][1] < 60.0:
            c = make_network(P, j, prec64, 16)
            it64, err64 = 0, float("nan")
            try:
                it64, err64, _ = P.bbp_iterate(c, tol, served_e[tpl][1])
            except P.BBPError:
                pass
            e_fp64 = P.bbp_energy_per_site(c)
            e64[tpl] = abs(e_fp64 - served_e[tpl][0])
            e64_detail.append({"template": j["kind"] + f" D={j['D']} chi={j['chi']}", "served_iters": served_e[tpl][1],
                               "served_err": served_e[tpl][2], "fp64_iters": int(it64), "fp64_err": float(err64),
                               "abs_d_energy": e64[tpl]})
            P.bbp_destroy(c)
    clock, seq = 0.0, []
    for k, (ta, tpl) in enumerate(arrivals if fp64_baseline else []):
        start = max(clock, ta)
        clock = start + svc[tpl]
        if ta >= warm_s:
            seq.append(clock - ta)
    S = np.array(seq) if seq else np.zeros(1)
    window = [k for k in done if arrivals[k][0] <= horizon]
    return {"arrival_rate_per_s": rate, "warmup_s": warm_s, "duration_s": duration_s, "tol": tol,
            "max_iter": max_iter, "jobs_arrived": len(measured), "jobs_finished": len(done),
            "jobs_unfinished": len(measured) - len(done), "converged": conv,
            "throughput_jobs_per_s": len(done) / max(1e-9, wall - warm_s),
            "p50_ms": 1e3 * float(np.percentile(L, 50)), "p99_ms": 1e3 * float(np.percentile(L, 99)),
            "latency_note": "over every job arriving after the warm-up; unfinished ones at their age when the run ended",
            "mean_iters": float(np.mean([iters[k] for k in done])) if done else None,
            "wall_s": round(wall, 1), "drain_s": drain_s,
            "energy_err_vs_fp64": {"max": max(e64.values()) if e64 else None, "templates": len(e64),
                                   "within_1e-5": sum(1 for v in e64.values() if v <= 1e-5),
                                   "detail": e64_detail},
            "jobs_finished_all": len(lat),
            "one_at_a_time_fp64": {"p50_ms": 1e3 * float(np.percentile(S, 50)),
                                   "p99_ms": 1e3 * float(np.percentile(S, 99)),
                                   "throughput_jobs_per_s": len(arrivals) / clock if clock > 0 else None,
                                   "method": "FIFO over the same arrivals; service = FP64 s/iteration x the "
                                             "template's served iterations (measured per template)"},
            "pool": f"{pool_n} templates (network_mix + 10% Kagome D=6 chi=64), seed {seed}; 2 streams per job",
            "max_active": max_active,
            "window_finished": len(window)}


# ---------------------------------------------------------------- oracle

def oracle_fullbond(w):
    """The FP64 oracle (as it stands) on the workload, with every incoming
    message at its full bond dimension (seeded random, normalised): the state
    of every iteration after the first, whose cost depends only on shapes."""
    import numpy as np
    from oracle.blockbp import BlockBP, normalise_message
    from oracle.geometry import Geometry
    t, em = make_inputs(w)
    geom = Geometry.kagome(w["Lx"], w["Ly"], w["L"])
    bb = BlockBP(geom, t, chi=w["chi"])
    bb.init_messages(em)
    rng = np.random.default_rng(12345)
    for key in list(bb.msgs):
        dims = [a.shape[1] for a in bb.msgs[key]]
        k = len(dims)
        bonds = [1] + [min(w["chi"], math.prod(dims[:q]), math.prod(dims[q:])) for q in range(1, k)] + [1]
        mps = [rng.standard_normal((bonds[q], dims[q], bonds[q + 1]))
               + 1j * rng.standard_normal((bonds[q], dims[q], bonds[q + 1])) for q in range(k)]
        bb.msgs[key] = normalise_message(mps, bb.face_dims(*key))
    return bb, geom


def oracle_update_time(w) -> float:
    """Seconds of one complete message update (block sweep and
    normalisation) of the oracle at full bond."""
    bb, geom = oracle_fullbond(w)
    bid, d, _ = geom.updates()[0]
    t0 = time.perf_counter()
    bb.update_message(bid, d)
    return time.perf_counter() - t0


def oracle_bulk_swallow(w, rng) -> float:
    """Seconds of one bulk swallow of the oracle's sweep at full bond: merge
    of the two boundary tensors on the segment, contraction with a fused site
    tensor (two legs in, two out), the truncated SVD of the
    (chi D^2) x (D^2 chi) split and the normalisation -- the step that the
    sweeps of this workload repeat."""
    import numpy as np
    from oracle import tn
    chi, D, d = w["chi"], w["D"], w["d"]
    D2 = D * D
    c = lambda *sh: rng.standard_normal(sh) + 1j * rng.standard_normal(sh)   # noqa: E731
    A1, A2 = c(chi, D2, chi), c(chi, D2, chi)
    X = tn.fuse(c(d, D, D, D, D))
    t0 = time.perf_counter()
    S = np.tensordot(A1, A2, axes=(2, 0))                          # (l, p1, p2, r)
    R = np.tensordot(S, X, axes=([1, 2], [0, 1]))                  # (l, r, q1, q2)
    R = np.moveaxis(R, 1, R.ndim - 1)                              # (l, q1, q2, r)
    a1, rem = tn.svd_split(R, chi)
    rem = rem / np.linalg.norm(rem)
    return time.perf_counter() - t0


def blas_threads():
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    return os.cpu_count()


# ----------------------------------------------------------------- peaks

def measure_peaks():
    """FP64 and FP32 FMA rates (this library's microbenchmark kernel), TF32
    and BF16 rates of the library's tcgen05 GEMM and of cuBLAS (torch) on an
    8192^3 product; CUDA-event timing, best of five."""
    import torch
    import paper_2603_13304_gb300 as P
    torch.cuda.set_device(0)
    P.build()
    props = torch.cuda.get_device_properties(0)
    out_buf = torch.zeros(2, dtype=torch.float64, device="cuda")
    res = {"sm_count": props.multi_processor_count, "gpu": props.name}

    def best(fn, reps=5):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fl = fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append((fl, e0.elapsed_time(e1) * 1e-3))
        return max(f / t for f, t in ts) / 1e12

    blocks = props.multi_processor_count * 8
    res["fp64_tflops"] = best(lambda: P.bbp_k_fma_peak(True, blocks, 2000, out_buf.data_ptr()))
    res["fp32_tflops"] = best(lambda: P.bbp_k_fma_peak(False, blocks, 20000, out_buf.data_ptr()))
    n = 8192
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for name, dt, bf in (("tf32", torch.float32, 0), ("bf16", torch.bfloat16, 1)):
        A = torch.randn(n, n, device="cuda").to(dt)
        B = torch.randn(n, n, device="cuda").to(dt)
        C = torch.empty(n, n, dtype=torch.float32, device="cuda")

        def ours():
            P.bbp_k_tc_gemm(bf, A.data_ptr(), n, B.data_ptr(), n, C.data_ptr(), n, n, n, n, 1.0, err.data_ptr())
            return 2.0 * n ** 3
        res[name + "_tc_gemm_tflops"] = best(ours)
        torch.backends.cuda.matmul.allow_tf32 = True
        Ac, Bc = (A, B)

        def cublas():
            torch.matmul(Ac, Bc)
            return 2.0 * n ** 3
        res[name + "_cublas_tflops"] = best(cublas)
    res["tc_gemm_error_flag"] = int(err.item())
    return res


def kernel_case(which: str):
    """One kernel of the path alone, on the shapes of the D = 6, chi = 64
    workload, for a profiler capture (`ncu -k ...`): `fuse` K1 at D = 8
    (output larger than L2), `absorb` the tcgen05 split-TF32 absorb of one
    bulk swallow (P = Q = 1296, l = r = 64), `panel` the cluster panel QR of
    one 2304 x 96 range panel.  Each runs three times; prints the CUDA-event
    time of the last."""
    import torch
    import paper_2603_13304_gb300 as P
    torch.cuda.set_device(0)
    P.build()
    g = torch.Generator(device="cuda").manual_seed(0)
    if which == "fuse":
        D, d = 8, 2
        t = torch.randn(d * D ** 4, dtype=torch.complex128, device="cuda", generator=g)
        T = torch.empty(D ** 8, dtype=torch.complex128, device="cuda")
        run = lambda: P.bbp_k_fuse(t.data_ptr(), d, D, [D] * 4, None, [0, 1, 2, 3], T.data_ptr())   # noqa: E731
        work = f"{D ** 8 * 16 / 1e9:.3f} GB written"
    elif which == "absorb":
        Pd, Q, l, r = 1296, 1296, 64, 64
        X = torch.randn(Pd, Q, dtype=torch.complex64, device="cuda", generator=g)
        S = torch.randn(l, Pd, r, dtype=torch.complex64, device="cuda", generator=g)
        R = torch.empty(l, Q, r, dtype=torch.complex64, device="cuda")
        wk = torch.empty(P.bbp_k_tc_absorb_bytes(0, Pd, Q, l, r), dtype=torch.uint8, device="cuda")
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        run = lambda: P.bbp_k_tc_absorb(0, 1, X.data_ptr(), Pd, Q, S.data_ptr(), l, r, R.data_ptr(), wk.data_ptr(),   # noqa: E731
                                        err.data_ptr())
        work = f"{8.0 * l * Pd * Q * r / 1e9:.1f} GFLOP complex"
    elif which in ("panel", "panel_r"):
        m, n = 2304, 96
        A = torch.randn(m, n, dtype=torch.complex64, device="cuda", generator=g)
        Qm = torch.empty_like(A) if which == "panel" else None
        Rm = torch.empty(n, n, dtype=torch.complex64, device="cuda")
        qp = Qm.data_ptr() if Qm is not None else None
        run = lambda: P.bbp_k_panel_qr(True, A.data_ptr(), m, n, qp, Rm.data_ptr(), 1, 0)   # noqa: E731
        work = f"{m}x{n} complex64 panel ({'Q and R' if Qm is not None else 'R only'})"
    elif which == "svd":
        m = n = 2304
        chi = 64
        A = torch.randn(m, n, dtype=torch.complex64, device="cuda", generator=g)
        U = torch.empty(m, chi, dtype=torch.complex64, device="cuda")
        Rm = torch.empty(chi, n, dtype=torch.complex64, device="cuda")
        wk = torch.empty(P.bbp_k_svd_work_bytes_rand(True, m, n, chi, False), dtype=torch.uint8, device="cuda")
        st = torch.zeros(4, dtype=torch.int32, device="cuda")
        run = lambda: P.bbp_k_svd_trunc_rand(True, A.data_ptr(), m, n, chi, U.data_ptr(), Rm.data_ptr(),   # noqa: E731
                                             wk.data_ptr(), st.data_ptr(), 1, False, None)
        work = f"complex64 randomised truncation of a {m}x{n} split to chi = {chi} (b = 96, one power step)"
    else:
        raise SystemExit("kernel case: fuse, absorb, panel, panel_r or svd")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(3):
        if i == 2:
            e0.record()
        run()
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": which, "ms": e0.elapsed_time(e1), "work": work}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="kagome-6x2-L2-D6-chi64", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="tf32", choices=["tf32", "bf16", "fp32", "fp64"])
    ap.add_argument("--roofline-kernel", default=None, choices=sorted(KERNELS),
                    help="kernel class timed for the roofline (default: orth, the cluster panel QR)")
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--batch", type=int, default=16, help="networks in the batched measurement (0: skip)")
    ap.add_argument("--batch-rounds", type=int, default=2, help="timed rounds of the batched measurement")
    ap.add_argument("--batch-pools", type=int, default=0,
                    help="worker pools shared by the batched networks (0: one each)")
    ap.add_argument("--serve", type=float, default=0.0,
                    help="seconds of arrivals after the warm-up in the serving measurement (0: skip)")
    ap.add_argument("--serve-pool", type=int, default=16, help="job templates of the serving stream")
    ap.add_argument("--serve-active", type=int, default=32, help="resident jobs at most (server slots)")
    ap.add_argument("--serve-no-fp64", action="store_true", help="skip the FP64 one-at-a-time baseline")
    ap.add_argument("--only", choices=["batched", "serving", "core", "ite"],
                    help="run only the batched, serving, core-extraction or ITE measurement and print it")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the core-extraction and ITE legs of the default line")
    ap.add_argument("--peaks", action="store_true", help="measure the chip's ALU and tensor rates and exit")
    ap.add_argument("--kernel-case", choices=["fuse", "absorb", "panel", "panel_r", "svd"],
                    help="run one kernel alone and exit")
    args = ap.parse_args()
    if args.kernel_case:
        kernel_case(args.kernel_case)
        return
    if args.roofline_kernel is None:
        args.roofline_kernel = "orth"     # the cluster panel QR: the largest share of every step
    if args.peaks:
        print(json.dumps(measure_peaks()))
        return
    if args.only:
        import torch
        import paper_2603_13304_gb300 as P
        torch.cuda.set_device(0)
        P.build()
        P.use_torch_allocator()
        prec_code = {"tf32": 1, "bf16": 2, "fp32": 3, "fp64": 0}[args.precision]
        if args.only == "batched":
            out = run_batched(args.batch, args.batch_rounds, 1, prec_code, groups=args.batch_pools)
        elif args.only == "core":
            out = run_core(args.workload, prec_code)
        elif args.only == "ite":
            out = run_ite()
        else:
            out = run_serving(args.serve, args.serve_rate, prec_code, warm_s=min(5.0, args.serve / 4),
                              pool_n=args.serve_pool, max_active=args.serve_active,
                              fp64_baseline=not args.serve_no_fp64)
        print(json.dumps({args.only: out}))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    w = WORKLOADS[args.workload]
    config = {"workload": w["workload"], "lattice": "kagome periodic super-cell 6x2 unit cells, 3 blocks of 12 sites",
              "d": w["d"], "D": w["D"], "chi": w["chi"], "updates_per_step": 12,
              "l2": "flushed between timed steps (256 MB write)", "tol": 0.0}

    if args.impl == "reference":
        if rank != 0:
            return
        import numpy as np
        rng = np.random.default_rng(7)
        # warm-up: one complete update and one bulk swallow give the number
        # of swallow-equivalents per update on these cores
        t_update = oracle_update_time(w)
        t_sw0 = oracle_bulk_swallow(w, rng)
        for _ in range(max(0, args.warmup - 1)):
            oracle_bulk_swallow(w, rng)
        per_update = t_update / t_sw0
        t_all = sum(oracle_bulk_swallow(w, rng) for _ in range(args.steps))
        value = args.steps / (t_all * per_update)
        cores = blas_threads()
        sample = (f"one bulk swallow (merge, absorb, truncated SVD of the {w['chi'] * w['D'] ** 2}^2 split) per "
                  f"step at full bond; {per_update:.2f} swallows per message update, from one complete update "
                  f"({t_update:.1f} s) timed in the warm-up")
        line = {"metric": "BlockBP message updates/s", "value": value, "unit": "message updates/s", "n_gpus": 0,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all * per_update / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
                "data": "synthetic", "config": config, "impl": "reference",
                "cpu_baseline": {"value": value, "unit": "message updates/s", "cores": cores, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": value, "unit": "message updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    res = run_ours(args, rank, world)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        dt = oracle_update_time(w)
        cpu = {"value": 1.0 / dt, "unit": "message updates/s", "cores": blas_threads(), "kind": "oracle",
               "sample": f"one complete message update at full bond ({dt:.1f} s of CPU work)"}
    prec_code = {"tf32": 1, "bf16": 2, "fp32": 3, "fp64": 0}[args.precision]
    batched = (run_batched(args.batch, args.batch_rounds, 1, prec_code, groups=args.batch_pools)
               if args.batch > 0 and world == 1 else None)
    serving = (run_serving(args.serve, args.serve_rate, prec_code, warm_s=min(5.0, args.serve / 4),
                           pool_n=args.serve_pool, max_active=args.serve_active,
                           fp64_baseline=not args.serve_no_fp64)
               if args.serve > 0 and world == 1 else None)
    core = ite_leg = None
    if world == 1 and not args.no_extras:
        # the thesis' core extraction (Sec. 2.3) and ITE update (Ch. 3), each
        # timed on its own; a failure is reported in the line, not raised
        try:
            core = run_core(args.workload, prec_code)
        except Exception as e:                              # noqa: BLE001
            core = {"error": str(e)[:300]}
        try:
            ite_leg = run_ite(max_updates=1)
        except Exception as e:                              # noqa: BLE001
            ite_leg = {"error": str(e)[:300]}
    line = {
        "metric": "BlockBP message updates/s", "value": res["value"], "unit": "message updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * res["secs"] / args.steps, "host_ms_per_step": 1e3 * res["host_secs"] / args.steps,
        "step_ms": [round(x, 3) for x in res["step_ms"]],
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "c128", "fp32": "c64+f64", "tf32": "tf32x3+c64+f64", "bf16": "bf16x6+c64+f64"}[args.precision], "data": "synthetic",
        "config": dict(config, precision=args.precision,
                       execution="eager launches" if args.no_graphs else "CUDA-graph replay of each iteration",
                       streams=16),
        "clocks": res["clocks"], "e2e": res["e2e"], "gpu_launches": res["launches"] * args.steps,
        "roofline": res["roofline"], "roofline_tensor_gemm": res["roofline_tc"], "cpu_baseline": cpu,
        "accuracy_vs_oracle": res["accuracy"],
        "energy_per_site": res["energy"], "absorb_tflop_per_step": res["flops_iter"] / 1e12,
        "batched": batched, "serving": serving, "core_extraction": core, "ite": ite_leg,
    }
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
