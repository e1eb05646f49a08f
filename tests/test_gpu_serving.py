"""Many problems on one GPU: the batched iteration and the continuous-batching
server compute, for every job, what the job computes alone.

Each context iterates on its own streams, so the only difference a mix can
make is the order in which independent kernels run; the kernels of one job
see the same inputs in the same order.  Results are compared on dense
messages (gauge-invariant) and on the energy per site.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import tn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2603_13304_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build()
    P.lib()


def spec(kind, seed, D, chi, prec):
    if kind == "square":
        Lx = Ly = 4
        t = syn.gaussian_peps(Lx * Ly, 2, D, seed=seed)
        em = syn.initial_edge_matrices(Lx * Ly, D, seed=seed + 100)
        return dict(lattice=P.SQUARE, Lx=Lx, Ly=Ly, periodic=0, d=2, D=D, bx=2, by=2, chi=chi, precision=prec,
                    tensors=t, edge_mats=em)
    nb = syn.kagome_neighbours(6, 2)
    t = syn.dimer_singlet_peps(nb, 2, D, seed=seed, noise=1e-2, noise_seed=seed + 1)
    em = syn.initial_edge_matrices(36, D, seed=seed + 100)
    return dict(lattice=P.KAGOME, Lx=6, Ly=2, periodic=1, d=2, D=D, bx=2, by=2, chi=chi, precision=prec,
                tensors=t, edge_mats=em)


def make_ctx(s):
    ctx = P.bbp_create_peps(s["lattice"], s["Lx"], s["Ly"], s["periodic"], s["d"], s["D"], s["tensors"])
    P.bbp_partition_blocks(ctx, s["bx"], s["by"])
    P.bbp_set_options(ctx, s["chi"], s["precision"])
    P.bbp_set_execution(ctx, True, 4)
    P.bbp_init_messages(ctx, s["edge_mats"])
    return ctx


def messages(ctx):
    nbk, _, _ = P.bbp_info(ctx)
    out = {}
    for b in range(nbk):
        for f in range(4):
            try:
                out[(b, f)] = tn.mps_dense(P.bbp_get_message(ctx, b, f))
            except P.BBPError:
                pass
    return out


def diff(a, b):
    return max(float(np.linalg.norm(a[k] - b[k])) for k in a)


SPECS = [("square", 1, 2, 4, P.FP64), ("square", 2, 2, 8, P.TF32), ("kagome", 3, 2, 8, P.FP32),
         ("square", 4, 3, 8, P.FP64)]


def test_batch_matches_individual():
    specs = [spec(*a) for a in SPECS]
    alone = []
    for s in specs:
        ctx = make_ctx(s)
        P.bbp_iterate(ctx, 0.0, 5)
        alone.append((messages(ctx), P.bbp_energy_per_site(ctx)))
        P.bbp_destroy(ctx)
    ctxs = [make_ctx(s) for s in specs]
    rc, iters, errs, st = P.bbp_batch_iterate(ctxs, 0.0, 5)
    try:
        assert rc in (0, 6) and list(iters) == [5] * len(specs)
        for i, ctx in enumerate(ctxs):
            m = messages(ctx)
            e = P.bbp_energy_per_site(ctx)
            tol = 1e-10 if specs[i]["precision"] == P.FP64 else 1e-6
            print(f"job {i}: message diff {diff(alone[i][0], m):.2e}, |dE| {abs(e - alone[i][1]):.2e}")
            assert diff(alone[i][0], m) < tol
            assert abs(e - alone[i][1]) < tol
    finally:
        for c in ctxs:
            P.bbp_destroy(c)


def test_batch_single_launch_matches_separate():
    """One graph launch per round (every context's replayed iteration a
    child of one graph) computes what separate per-context launches compute;
    8 rounds, so that the graphs take over once the bond dimensions settle."""
    specs = [spec(*a) for a in SPECS]
    out = {}
    for single in (False, True):
        P.bbp_batch_single_launch(single)
        ctxs = [make_ctx(s) for s in specs]
        try:
            for _ in range(8):      # one round a call, as a serving loop would
                rc, iters, errs, st = P.bbp_batch_iterate(ctxs, 0.0, 1)
                assert rc in (0, 6)
            out[single] = [(messages(c), P.bbp_energy_per_site(c)) for c in ctxs]
        finally:
            for c in ctxs:
                P.bbp_destroy(c)
    P.bbp_batch_single_launch(True)
    for i, s in enumerate(specs):
        tol = 1e-10 if s["precision"] == P.FP64 else 1e-6
        d = diff(out[False][i][0], out[True][i][0])
        de = abs(out[False][i][1] - out[True][i][1])
        print(f"job {i}: single vs separate launches: message diff {d:.2e}, |dE| {de:.2e}")
        assert d < tol and de < tol


@pytest.mark.parametrize("single,groups", [(True, 2), (False, 2), (True, 1)])
def test_shared_workers_match_private(single, groups):
    """Contexts dealt into shared worker pools (their iterations one after
    another on the pool's streams and arenas) compute what they compute with
    private pools, with the round as one graph launch or separate launches.
    With one pool, the small networks settle (and defer their replayed
    iterations to the round's launch) while the larger ones still grow the
    pool's arenas in the same round."""
    specs = [spec(*a) for a in SPECS] + [spec("kagome", 7, 3, 16, P.TF32)]
    out = {}
    P.bbp_batch_single_launch(single)
    try:
        for shared in (False, True):
            ctxs = [make_ctx(s) for s in specs]
            try:
                if shared:
                    P.bbp_share_workers(ctxs, groups)
                for _ in range(8):
                    rc, iters, errs, st = P.bbp_batch_iterate(ctxs, 0.0, 1)
                    assert rc in (0, 6)
                out[shared] = [(messages(c), P.bbp_energy_per_site(c)) for c in ctxs]
            finally:
                for c in ctxs:
                    P.bbp_destroy(c)
    finally:
        P.bbp_batch_single_launch(True)
    for i, s in enumerate(specs):
        tol = 1e-10 if s["precision"] == P.FP64 else 1e-6
        d = diff(out[False][i][0], out[True][i][0])
        de = abs(out[False][i][1] - out[True][i][1])
        print(f"job {i}: shared vs private workers ({groups} pools, single launch {single}): message diff {d:.2e}, "
              f"|dE| {de:.2e}")
        assert d < tol and de < tol


def run_server(specs, budget=1 << 36, max_active=64, iters=6, stagger=0):
    srv = P.bbp_server_create(budget, max_active)
    ids = []
    peak = 0
    try:
        pending = list(specs)
        steps = 0
        results = {}
        while pending or len(results) < len(specs):
            # submit one job per step after the first `stagger` steps, so
            # that later jobs arrive while earlier ones are on the device
            if pending and (steps >= stagger or not ids):
                s = pending.pop(0)
                job = P.make_job(s["lattice"], s["Lx"], s["Ly"], s["periodic"], s["d"], s["D"], s["bx"], s["by"],
                                 s["chi"], s["precision"], s["tensors"], s["edge_mats"], 0.0, iters)
                ids.append(P.bbp_server_submit(srv, job))
            q, a, f = P.bbp_server_step(srv, 100.0)
            peak = max(peak, a)
            for r in P.bbp_server_poll(srv):
                ctx = P.bbp_server_take(srv, r["id"], keep_context=True)
                results[r["id"]] = (r, messages(ctx), P.bbp_energy_per_site(ctx))
                P.bbp_destroy(ctx)
            steps += 1
            assert steps < 10000
        return [results[i] for i in ids], peak
    finally:
        P.bbp_server_destroy(srv)


def test_server_alone_vs_mix():
    target = spec("square", 7, 2, 8, P.FP64)
    (alone,), _ = run_server([target])
    others = [spec(*a) for a in SPECS]
    mix = others[:2] + [target] + others[2:]
    res, peak = run_server(mix, stagger=1)
    r, m, e = res[2]
    assert r["status"] in (0, 6) and r["iters"] == 6 and alone[0]["iters"] == 6
    d = diff(alone[1], m)
    print(f"alone vs mix: message diff {d:.2e}, |dE| {abs(e - alone[2]):.2e}, peak resident {peak}")
    assert peak >= 2          # the target really shared the device with others
    assert d < 1e-10 and abs(e - alone[2]) < 1e-10


def test_server_admission_by_footprint():
    specs = [spec(*a) for a in SPECS[:3]]
    fps = []
    for s in specs:
        job = P.make_job(s["lattice"], s["Lx"], s["Ly"], s["periodic"], s["d"], s["D"], s["bx"], s["by"], s["chi"],
                         s["precision"], s["tensors"], s["edge_mats"], 0.0, 3)
        fps.append(P.bbp_job_footprint_bytes(job))
    # a budget below the two smallest footprints together admits one job at
    # a time (a job larger than the budget still runs when nothing else does)
    a, b = sorted(fps)[:2]
    budget = a + b - 1
    res, peak = run_server(specs, budget=budget, iters=3)
    assert peak == 1
    assert all(r[0]["status"] in (0, 6) and r[0]["iters"] == 3 for r in res)
    lat = [r[0]["latency_s"] for r in res]
    wait = [r[0]["wait_s"] for r in res]
    print("latencies", lat, "waits", wait)
    assert wait[1] > 0 and wait[2] >= wait[1] * 0.5


def test_kernel_timer_reselect_keeps_captured_graphs_valid():
    """Selecting a timer class bakes event nodes into the captured iteration
    graph; selecting another class (or none) afterwards must leave those
    events alive, so that replaying the graph computes what a context that
    never used the timer computes."""
    s = spec("square", 31, 2, 8, P.FP64)
    ref = make_ctx(s)
    ctx = make_ctx(s)
    try:
        P.bbp_iterate(ref, 0.0, 10)
        P.bbp_iterate(ctx, 0.0, 3)
        P.bbp_ktimer_select(P.KT_JACOBI)
        P.bbp_set_execution(ctx, True, 4)        # recapture with the timer's event nodes
        P.bbp_iterate(ctx, 0.0, 4)
        n, ms, _ = P.bbp_ktimer_read()
        assert n > 0 and ms > 0.0
        P.bbp_ktimer_select(0)
        P.bbp_iterate(ctx, 0.0, 3)                # replays the graphs holding those events
        n2, _, _ = P.bbp_ktimer_read()
        assert n2 == 0
        a, b = messages(ref), messages(ctx)
        assert max(float(np.abs(a[k] - b[k]).max()) for k in a) < 1e-12
    finally:
        P.bbp_ktimer_select(0)
        P.bbp_destroy(ctx)
        P.bbp_destroy(ref)
