"""Host-side logic of the batch and server entry points, without a GPU:
argument checks, the footprint estimate that drives admission, and the job
queue (submission, polling and removal touch only host memory)."""
import numpy as np
import pytest

import synthetic as syn

P = pytest.importorskip("paper_2603_13304_gb300")


@pytest.fixture(scope="module", autouse=True)
def lib():
    P.build()
    P.lib()


def job(D=2, chi=8, precision=None, lattice="square", tol=1e-6, max_iter=10):
    precision = P.TF32 if precision is None else precision
    if lattice == "square":
        t = syn.gaussian_peps(16, 2, D, seed=1)
        em = syn.initial_edge_matrices(16, D, seed=2)
        return P.make_job(P.SQUARE, 4, 4, 0, 2, D, 2, 2, chi, precision, t, em, tol, max_iter)
    nb = syn.kagome_neighbours(6, 2)
    t = syn.dimer_singlet_peps(nb, 2, D, seed=1, noise=1e-2, noise_seed=2)
    em = syn.initial_edge_matrices(36, D, seed=3)
    return P.make_job(P.KAGOME, 6, 2, 1, 2, D, 2, 2, chi, precision, t, em, tol, max_iter)


def test_footprint_grows_with_the_problem():
    fp = P.bbp_job_footprint_bytes
    assert fp(job(D=2, chi=8)) < fp(job(D=3, chi=8)) < fp(job(D=4, chi=8))
    assert fp(job(D=2, chi=8)) < fp(job(D=2, chi=16)) < fp(job(D=2, chi=32))
    assert fp(job(precision=P.FP32)) < fp(job(precision=P.FP64))
    assert fp(job(lattice="square")) < fp(job(lattice="kagome"))


def test_server_queue_without_device_work():
    srv = P.bbp_server_create(1 << 30, 4)
    try:
        ids = [P.bbp_server_submit(srv, job()) for _ in range(3)]
        assert ids == sorted(ids) and len(set(ids)) == 3
        assert P.bbp_server_poll(srv) == []          # nothing finished
        with pytest.raises(P.BBPError):
            P.bbp_server_take(srv, 12345)            # unknown job
    finally:
        P.bbp_server_destroy(srv)                    # queued jobs are dropped


def test_argument_checks():
    L = P.lib()
    assert L.bbp_server_create(None, 1 << 20, 1) != 0
    import ctypes
    out = ctypes.c_void_p()
    assert L.bbp_server_create(ctypes.byref(out), 0, 1) != 0          # zero budget
    assert L.bbp_server_create(ctypes.byref(out), 1 << 20, 0) != 0    # no slot
    assert L.bbp_server_submit(None, None, None) != 0
    bad = job()
    bad.chi = 0
    srv = P.bbp_server_create(1 << 20, 1)
    try:
        with pytest.raises(P.BBPError):
            P.bbp_server_submit(srv, bad)
        with pytest.raises(P.BBPError):
            P.bbp_server_step(None)
    finally:
        P.bbp_server_destroy(srv)
    # an empty batch is a no-op; a missing context is reported per slot
    rc, iters, errs, st = P.bbp_batch_iterate([None], 0.0, 3)
    assert rc != 0 and st[0] != 0 and iters[0] == 0
    rc, iters, errs, st = P.bbp_batch_iterate([], 0.0, 3)
    assert rc == 0


def test_kernel_timer_off_is_inert():
    P.bbp_ktimer_select(0)
    assert P.bbp_ktimer_read() == (0, 0.0, 0.0)


def test_failed_setup_is_reported_not_raised():
    """Without a usable device the admitted job's set-up fails; the server
    reports it as a finished job with a status instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("needs a process without a GPU")
    srv = P.bbp_server_create(1 << 30, 2)
    try:
        jid = P.bbp_server_submit(srv, job())
        P.bbp_server_step(srv, 1.0)
        done = P.bbp_server_poll(srv)
        assert [r["id"] for r in done] == [jid]
        assert done[0]["status"] != 0 and done[0]["iters"] == 0
        P.bbp_server_take(srv, jid)
        assert P.bbp_server_poll(srv) == []
    finally:
        P.bbp_server_destroy(srv)
