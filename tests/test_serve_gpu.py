"""The serving form: a request loop with continuous batching.

* A request's result is the same alone and in a mix of requests that arrive
  while it runs (lambda bit for bit at the same iteration count, the scalars
  to the order of their partial sums).
* Admission keeps the resident footprint within the HBM budget (requests
  then run one after another), and a request that can never fit fails.
* FP32 and BF16 requests run side by side, each matching the oracle on the
  values it stores.
* A request's input arrays may be overwritten once it reports RUNNING.
"""
import time

import numpy as np
import pytest

import oracle
import synth
from test_parity_gpu import decoded

pytestmark = pytest.mark.gpu

GIB = 1 << 30


@pytest.fixture(scope="module")
def dl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04621_gb300 import build

    build.build()
    import paper_2603_04621_gb300 as d

    return d


def requests(n, seed=2024, i_range=(2_000, 60_000), j_range=(50, 3_000)):
    trace = synth.request_trace(n, seed=seed, i_range=i_range, j_range=j_range)
    return [synth.greedy_budgets(synth.request_instance(r)) for r in trace], trace


def wait_running(srv, timeout=60.0):
    t0 = time.time()
    while time.time() - t0 < timeout:
        if srv.stats()["running"] >= 1:
            return
        time.sleep(0.002)
    raise AssertionError("no request started")


def test_alone_equals_in_mix(dl):
    insts, _ = requests(6)
    kw = dict(max_iters=1500)
    target = insts[2]
    srv = dl.Server(64 * GIB, max_slots=16)
    t = srv.submit(target, **kw)
    alone, lam_alone = srv.wait(t)
    srv.close()
    assert alone["state"] == dl.DUALIP_REQ_DONE

    srv = dl.Server(64 * GIB, max_slots=16)
    others = [srv.submit(x, **kw) for k, x in enumerate(insts) if k != 2]
    wait_running(srv)
    t = srv.submit(target, **kw)  # arrives while others are on the GPU
    mixed, lam_mixed = srv.wait(t)
    rest = [srv.wait(o) for o in others]
    stats = srv.stats()
    srv.close()
    assert mixed["state"] == dl.DUALIP_REQ_DONE
    assert all(r[0]["state"] == dl.DUALIP_REQ_DONE for r in rest)
    assert stats["done"] == len(insts) and stats["failed"] == 0
    # it overlapped with the others: admitted before some of them finished
    assert any(r[0]["t_done"] > mixed["t_admit"] for r in rest)
    # its step, momentum and stopping test use its own quantities only, and its
    # gradients are exact, so it stops at the same check with the same lambda
    assert mixed["converged"] == alone["converged"]
    assert mixed["iters"] == alone["iters"]
    assert np.array_equal(lam_alone, lam_mixed)
    for key in ("dual_obj", "primal_obj", "reg", "lambda_dot_grad"):
        assert abs(mixed[key] - alone[key]) <= 1e-6 * max(1.0, abs(alone[key])), key


def test_max_iters_not_a_multiple_of_the_chunk(dl):
    """A request whose max_iters is not a multiple of the server's chunk length
    stops at exactly max_iters, alone and beside a request with a longer run."""
    insts, _ = requests(2, seed=55)
    srv = dl.Server(64 * GIB, max_slots=8, check_every=10)
    t_long = srv.submit(insts[0], max_iters=200, stop_on_tol=0)
    t = srv.submit(insts[1], max_iters=55, stop_on_tol=0)
    info, _ = srv.wait(t)
    info_long, _ = srv.wait(t_long)
    srv.close()
    assert info["state"] == info_long["state"] == dl.DUALIP_REQ_DONE
    assert info["iters"] == 55
    assert info_long["iters"] == 200


def test_budget_admission_serialises(dl):
    x = requests(1, seed=77)[0][0]
    # room for one copy (with its creation transient) but never for two
    resident = 12 * (x.E + 8) + 8 * (x.I + 4) + 16 * (x.E // 1024 + x.I // 256 + 2) + 56 * x.J
    need = resident + 12 * x.E
    budget = int(1.2 * need)
    srv = dl.Server(budget, max_slots=8)
    ts = [srv.submit(x, max_iters=300) for _ in range(3)]
    infos = [srv.wait(t)[0] for t in ts]
    st = srv.stats()
    srv.close()
    assert all(i["state"] == dl.DUALIP_REQ_DONE for i in infos)
    assert st["peak_resident_bytes"] <= budget
    # FIFO admission, one at a time: each starts once the previous one is done
    for a, b in zip(infos, infos[1:]):
        assert b["t_admit"] >= a["t_done"] - 1e-3
    # and all three give the same answer
    assert infos[0]["iters"] == infos[1]["iters"] == infos[2]["iters"]


def test_request_larger_than_budget_fails(dl):
    insts, _ = requests(1, seed=5)
    srv = dl.Server(1 << 20, max_slots=4)
    t = srv.submit(insts[0])
    info, lam = srv.wait(t)
    srv.close()
    assert info["state"] == dl.DUALIP_REQ_FAILED and info["status"] == dl.DUALIP_ENOMEM
    assert lam is None


def test_mixed_storage_matches_oracle(dl):
    insts, trace = requests(4, seed=314)
    srv = dl.Server(64 * GIB, max_slots=8)
    gamma = 1e-2
    kw = dict(max_iters=20, stop_on_tol=0, gamma0=gamma, gamma_final=gamma, row_normalize=0)
    ts = [srv.submit(x, storage=r["storage"], **kw) for x, r in zip(insts, trace)]
    out = [srv.wait(t) for t in ts]
    srv.close()
    assert {r["storage"] for r in trace} == {"f32", "bf16"}
    for (info, lam), x, r in zip(out, insts, trace):
        assert info["state"] == dl.DUALIP_REQ_DONE and info["iters"] == 20
        ref = decoded(x) if r["storage"] == "bf16" else x
        eo = oracle.Problem(ref).eval(lam.astype(np.float64), gamma)
        # the returned lambda is the point of the last evaluation
        assert abs(info["dual_obj"] - eo.dual) <= 1e-6 * max(1.0, abs(eo.dual))


def test_inputs_may_change_once_running(dl):
    """A request's host arrays have been copied by the time it reports RUNNING:
    overwriting them from then on leaves its result as it was."""
    kw = dict(max_iters=200, stop_on_tol=0)
    x_ref = requests(1, seed=99)[0][0]
    x = requests(1, seed=99)[0][0]  # the same instance, in arrays of its own
    srv = dl.Server(64 * GIB, max_slots=4)
    ref_info, ref_lam = srv.wait(srv.submit(x_ref, **kw))
    t = srv.submit(x, **kw)
    assert np.shares_memory(srv._keep[t][2], x.c)  # the server reads x's own buffers
    deadline = time.time() + 60
    while srv.poll(t)["state"] == dl.DUALIP_REQ_QUEUED and time.time() < deadline:
        time.sleep(0.001)
    for arr in (x.c, x.a, x.b):
        arr[:] = 7.0
    x.dst[:] = 0
    info, lam = srv.wait(t)
    srv.close()
    assert ref_info["state"] == info["state"] == dl.DUALIP_REQ_DONE
    assert info["iters"] == ref_info["iters"] == 200
    assert np.array_equal(lam, ref_lam)
