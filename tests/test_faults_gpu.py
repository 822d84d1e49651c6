"""Failure paths, with faults injected on the host only (no device fault, trap
or hang is provoked).

* A host-set flag makes the pass's bounded device waits give up: the call
  returns DUALIP_ETIMEOUT, and the handle keeps working (the next evaluation
  equals one taken before the fault, bit for bit).  The solver reports the
  same status.
* Serving: a queued request and a running request are cancelled; the others
  finish.
"""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04621_gb300 import build

    build.build()
    import paper_2603_04621_gb300 as d

    return d


def test_injected_wait_abort_returns_timeout_and_recovers(dl):
    import torch

    inst = synth.config("c2", scale=0.02)
    P = dl.Problem.from_instance(inst)
    lam = torch.from_numpy(np.random.default_rng(3).uniform(0, 1, inst.J).astype(np.float32)).cuda()
    g0, e0 = P.dual_grad(lam, 1e-2)
    g0 = g0.clone()
    dl.dualip_debug_abort_waits(P.h, dl._stream())
    t0 = time.time()
    with pytest.raises(dl.DualipError) as ei:
        P.dual_grad(lam, 1e-2)
    assert ei.value.status == dl.DUALIP_ETIMEOUT
    assert time.time() - t0 < 1.5  # gave up at once, not after the 2 s wait limit
    g1, e1 = P.dual_grad(lam, 1e-2)
    assert torch.equal(g0, g1)
    assert e1["dual_obj"] == pytest.approx(e0["dual_obj"], rel=1e-12)

    # the solver: a fixed number of iterations is deterministic, so the run
    # after the fault repeats the run before it
    Q = dl.Problem.from_instance(synth.greedy_budgets(inst))
    kw = dict(max_iters=200, stop_on_tol=0)
    lam_a, _ = Q.solve(**kw)
    dl.dualip_debug_abort_waits(Q.h, dl._stream())
    with pytest.raises(dl.DualipError) as ei:
        Q.solve(**kw)
    assert ei.value.status == dl.DUALIP_ETIMEOUT
    lam_b, _ = Q.solve(**kw)
    assert torch.equal(lam_a, lam_b)


def test_server_cancels_queued_and_running_requests(dl):
    trace = synth.request_trace(4, seed=11, i_range=(20_000, 40_000), j_range=(200, 800))
    insts = [synth.greedy_budgets(synth.request_instance(r)) for r in trace]
    # room for one request at a time, so the later ones queue
    x = max(insts, key=lambda v: v.E)
    need = 12 * (x.E + 8) + 8 * (x.I + 4) + 16 * (x.E // 1024 + x.I // 256 + 2) + 56 * x.J
    srv = dl.Server(int(1.2 * (need + 12 * x.E)), max_slots=4)
    kw = dict(max_iters=100000, stop_on_tol=0)  # runs until cancelled
    t_run = srv.submit(insts[0], **kw)
    t_q = srv.submit(insts[1], **kw)
    t_ok = srv.submit(insts[2], max_iters=50)
    deadline = time.time() + 60
    while srv.poll(t_run)["state"] != dl.DUALIP_REQ_RUNNING and time.time() < deadline:
        time.sleep(0.005)
    assert srv.poll(t_q)["state"] == dl.DUALIP_REQ_QUEUED
    srv.cancel(t_q)
    q_info, _ = srv.wait(t_q, 10)
    assert q_info["state"] == dl.DUALIP_REQ_FAILED and q_info["status"] == dl.DUALIP_ECANCELED
    time.sleep(0.05)
    srv.cancel(t_run)
    r_info, lam = srv.wait(t_run, 60)
    assert r_info["state"] == dl.DUALIP_REQ_FAILED and r_info["status"] == dl.DUALIP_ECANCELED
    assert lam is None and r_info["t_admit"] >= 0
    ok_info, lam_ok = srv.wait(t_ok, 120)
    assert ok_info["state"] == dl.DUALIP_REQ_DONE and ok_info["iters"] == 50
    assert lam_ok is not None and np.all(lam_ok >= 0)
    st = srv.stats()
    srv.close()
    assert st["failed"] == 2 and st["done"] == 1 and st["resident_bytes"] == 0
