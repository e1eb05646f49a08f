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

# TF32 / BF16 dense tensor rates of the part, nominal (for the ratio only)
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25


def peaks():
    """Roofline denominators: the measured BF16 burst rate, TF32 at the
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
    P.bbp_ktimer_select(cls)
    P.bbp_set_execution(ctx, not args.no_graphs, 16)   # recapture with the event nodes
    P.bbp_iterate(ctx, 0.0, 1)
    P.bbp_ktimer_read()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        P.bbp_iterate(ctx, 0.0, 1)
    torch.cuda.synchronize()
    timer_pass_secs = time.perf_counter() - t1
    k_n, k_ms, k_flops = P.bbp_ktimer_read()
    P.bbp_ktimer_select(0)
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

    roof = None
    if rank == 0 and k_n > 0:
        pk = peaks()
        tensor = args.roofline_kernel == "tc"
        bound, unit = ("tensor", "TFLOP/s") if tensor else ("alu", "TFLOP/s")
        key = (args.precision if args.precision in ("tf32", "bf16") else "tf32") if tensor else (
            "fp64" if args.precision == "fp64" else "fp32")
        per_launch_s = k_ms * 1e-3 / k_n
        # the library credits each tensor-core launch with its algorithmic
        # complex flops; the split operands execute three real products per
        # complex product in TF32 (six in BF16)
        split = (6.0 if args.precision == "bf16" else 3.0) if tensor else 1.0
        achieved = k_flops / k_n / per_launch_s / 1e12
        roof = {"bound": bound, "achieved": achieved, "peak": pk[key], "unit": unit, "frac": achieved / pk[key],
                "traffic": None, "kernel": kdesc,
                "peak_kind": (key + " dense, of measured (bf16 burst x nominal tf32/bf16 ratio)" if key == "tf32"
                              else "bf16 dense burst, of measured") if tensor else key + ", " + pk[key + "_kind"],
                "flops_kind": "algorithmic complex flops (8 per complex multiply-add)",
                "executed_tensor_frac": achieved * split / pk[key] if tensor else None,
                "launches_per_step": k_n / args.steps, "launch_us": per_launch_s * 1e6,
                "kernel_ms_per_step_all_streams": k_ms / args.steps,
                "timer_pass_ms_per_step": 1e3 * timer_pass_secs / args.steps}
        if not tensor:
            roof["frac_of_one_sm"] = achieved / (pk[key] / 152)
    return {
        "value": value, "secs": secs, "host_secs": host_secs, "step_ms": step_ms, "n_updates": n_updates, "n_sites": n_sites, "energy": energy,
        "clocks": clk.summary(), "launches": launches, "flops_iter": flops_iter, "e2e": e2e, "roofline": roof,
        "accuracy": acc,
    }


# -------------------------------------------------- many networks, serving

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


def run_batched(n_networks, steps, warmup, precision):
    """All message updates of n_networks independent networks, one
    synchronous iteration of every network per round (bbp_batch_iterate)."""
    import torch
    import paper_2603_13304_gb300 as P
    jobs = job_mix(n_networks, 4, precision)
    ctxs = []
    n_updates = 0
    for j in jobs:
        c = P.bbp_create_peps(j["lattice"], j["Lx"], j["Ly"], j["periodic"], 2, j["D"], j["t"])
        P.bbp_partition_blocks(c, j["bx"], j["by"])
        P.bbp_set_options(c, j["chi"], precision)
        P.bbp_set_execution(c, True, 2)
        P.bbp_init_messages(c, j["em"])
        n_updates += P.bbp_info(c)[1]
        ctxs.append(c)
    for _ in range(warmup + 4):          # settle the bond dimensions, capture the graphs
        P.bbp_batch_iterate(ctxs, 0.0, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record()
    for _ in range(steps):
        P.bbp_batch_iterate(ctxs, 0.0, 1)
    e1.record()
    torch.cuda.synchronize()
    host = time.perf_counter() - t0
    secs = e0.elapsed_time(e1) * 1e-3
    for c in ctxs:
        P.bbp_destroy(c)
    return {"networks": n_networks, "message_updates_per_round": n_updates, "rounds": steps,
            "value": n_updates * steps / max(secs, host), "unit": "message updates/s",
            "ms_per_round": 1e3 * max(secs, host) / steps,
            "mix": "square 4x4 (2x2 blocks) / 6x6 (3x3 blocks), Kagome 6x2 (L=2); D 2..4, chi 8/16/32; seed 4"}


def run_serving(n_jobs, rate, precision, tol=1e-6, max_iter=40):
    """Poisson arrivals (seed 5) of a job mix into the server; each job runs
    to tol; returns throughput and latency percentiles, and the same trace
    run one job at a time (bbp_iterate on each in arrival order)."""
    import numpy as np
    import torch
    import paper_2603_13304_gb300 as P
    jobs = job_mix(n_jobs, 5, precision, max_D=3, chis=(8, 16))
    rng = np.random.default_rng(5)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_jobs))
    srv = P.bbp_server_create(200 << 30, 64)
    lat, waits, iters, stat = {}, {}, {}, {}
    t0 = time.perf_counter()
    nxt = 0
    ids = {}
    while len(lat) < n_jobs:
        now = time.perf_counter() - t0
        while nxt < n_jobs and arrivals[nxt] <= now:
            j = jobs[nxt]
            job = P.make_job(j["lattice"], j["Lx"], j["Ly"], j["periodic"], 2, j["D"], j["bx"], j["by"], j["chi"],
                             precision, j["t"], j["em"], tol, max_iter, 2, 1)
            ids[P.bbp_server_submit(srv, job)] = nxt
            nxt += 1
        P.bbp_server_step(srv, 2.0)
        for r in P.bbp_server_poll(srv):
            k = ids[r["id"]]
            lat[k], waits[k], iters[k], stat[k] = r["latency_s"], r["wait_s"], r["iters"], r["status"]
            P.bbp_server_take(srv, r["id"])
    wall = time.perf_counter() - t0
    P.bbp_server_destroy(srv)
    # the same trace, one job at a time
    t1 = time.perf_counter()
    seq_lat = []
    clock = 0.0
    for k, j in enumerate(jobs):
        start = max(clock, arrivals[k])
        s0 = time.perf_counter()
        c = P.bbp_create_peps(j["lattice"], j["Lx"], j["Ly"], j["periodic"], 2, j["D"], j["t"])
        P.bbp_partition_blocks(c, j["bx"], j["by"])
        P.bbp_set_options(c, j["chi"], precision)
        P.bbp_init_messages(c, j["em"])
        try:
            P.bbp_iterate(c, tol, max_iter)
        except P.BBPError:
            pass
        torch.cuda.synchronize()
        P.bbp_destroy(c)
        clock = start + (time.perf_counter() - s0)
        seq_lat.append(clock - arrivals[k])
    seq_wall = time.perf_counter() - t1
    L = np.array([lat[k] for k in range(n_jobs)])
    S = np.array(seq_lat)
    return {"jobs": n_jobs, "arrival_rate_per_s": rate, "tol": tol, "max_iter": max_iter,
            "throughput_jobs_per_s": n_jobs / wall, "p50_ms": 1e3 * float(np.percentile(L, 50)),
            "p99_ms": 1e3 * float(np.percentile(L, 99)), "mean_iters": float(np.mean([iters[k] for k in iters])),
            "converged": int(sum(1 for k in stat if stat[k] == 0)),
            "one_at_a_time": {"throughput_jobs_per_s": n_jobs / seq_wall, "p50_ms": 1e3 * float(np.percentile(S, 50)),
                              "p99_ms": 1e3 * float(np.percentile(S, 99))},
            "mix": "square 4x4 / 6x6, Kagome 6x2; D 2..3, chi 8/16; seed 5; 2 streams per job"}


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
    elif which == "panel":
        m, n = 2304, 96
        A = torch.randn(m, n, dtype=torch.complex64, device="cuda", generator=g)
        Qm = torch.empty_like(A)
        Rm = torch.empty(n, n, dtype=torch.complex64, device="cuda")
        run = lambda: P.bbp_k_panel_qr(True, A.data_ptr(), m, n, Qm.data_ptr(), Rm.data_ptr(), 1, 0)   # noqa: E731
        work = f"{m}x{n} complex64 panel, cluster {P.bbp_k_panel_cluster(True, m, n)}+"
    else:
        raise SystemExit("kernel case: fuse, absorb or panel")
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
                    help="kernel class timed for the roofline (default: tc for tf32/bf16, else orth)")
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--batch", type=int, default=64, help="networks in the batched measurement (0: skip)")
    ap.add_argument("--serve", type=int, default=48, help="jobs in the serving measurement (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--peaks", action="store_true", help="measure the chip's ALU and tensor rates and exit")
    ap.add_argument("--kernel-case", choices=["fuse", "absorb", "panel"], help="run one kernel alone and exit")
    args = ap.parse_args()
    if args.kernel_case:
        kernel_case(args.kernel_case)
        return
    if args.roofline_kernel is None:
        args.roofline_kernel = "tc" if args.precision in ("tf32", "bf16") else "orth"
    if args.peaks:
        print(json.dumps(measure_peaks()))
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
    batched = run_batched(args.batch, args.steps, args.warmup, prec_code) if args.batch > 0 and world == 1 else None
    serving = run_serving(args.serve, args.serve_rate, prec_code) if args.serve > 0 and world == 1 else None
    line = {
        "metric": "BlockBP message updates/s", "value": res["value"], "unit": "message updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * res["secs"] / args.steps, "host_ms_per_step": 1e3 * res["host_secs"] / args.steps,
        "step_ms": [round(x, 3) for x in res["step_ms"]],
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "c128", "fp32": "c64+f64", "tf32": "tf32x3+c64+f64", "bf16": "bf16x3+c64+f64"}[args.precision], "data": "synthetic",
        "config": dict(config, precision=args.precision,
                       execution="eager launches" if args.no_graphs else "CUDA-graph replay of each iteration",
                       streams=16),
        "clocks": res["clocks"], "e2e": res["e2e"], "gpu_launches": res["launches"] * args.steps,
        "roofline": res["roofline"], "cpu_baseline": cpu, "accuracy_vs_oracle": res["accuracy"],
        "energy_per_site": res["energy"], "absorb_tflop_per_step": res["flops_iter"] / 1e12,
        "batched": batched, "serving": serving,
    }
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
