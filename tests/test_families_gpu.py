"""Several constraint families (Section 3.2, Definition 1) on the GPU against
the FP64 oracle: every edge has m coefficients, the dual has m J entries
(row k J + j), and the evaluation, the primal and the ascent follow the same
definition as with one family.  Tolerances are those of the parity tests."""
import numpy as np
import pytest

import oracle
import synth
from test_parity_gpu import check_eval

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


@pytest.mark.parametrize("m,weighted", [(2, False), (3, False), (2, True)])
def test_families_parity(dl, m, weighted):
    # c2-shaped sources (Poisson(50) degrees, Zipf destinations), several tiles'
    # worth of warps, at three gammas and two dual points
    inst = synth.add_families(synth.greedy_budgets(synth.config("c2", scale=0.01)), m, seed=5)
    rng = np.random.default_rng(40 + m)
    P = Po = None
    for gamma in (0.5, 0.01, 1e-3):
        for lam in (np.zeros(m * inst.J), rng.uniform(0, 1.5, m * inst.J)):
            P, Po, grad, ev = check_eval(dl, inst, lam, gamma, weighted, P=P, Po=Po)
    assert P.m == m and P.J == m * inst.J


def test_families_widely_spread_weights(dl):
    """Two families with coefficients over four orders of magnitude and primal
    scaling (w = sum_k a_k^2): the weighted rounds are FP64."""
    base = synth.greedy_budgets(synth.config("c2", scale=0.005))
    inst = synth.add_families(base, 2, seed=8, a_range=(0.01, 100.0))
    rng = np.random.default_rng(48)
    P = Po = None
    for gamma in (0.1, 1e-3):
        P, Po, _, _ = check_eval(dl, inst, rng.uniform(0, 1, 2 * inst.J), gamma, True, P=P, Po=Po)


def test_families_edge_cases_box_and_primal(dl):
    import torch

    # empty sources, a source of 5000 edges, one-edge sources; unit box too
    degs = np.array([0, 1, 3, 5000, 0, 40, 1, 700])
    base = synth.greedy_budgets(synth.from_degrees(degs, 6000, 17, synth.DST_UNIFORM))
    inst = synth.add_families(base, 2, seed=6)
    rng = np.random.default_rng(7)
    for box in (False, True):
        for gamma in (0.3, 1e-3):
            check_eval(dl, inst, rng.uniform(0, 1, 2 * inst.J), gamma, box=box)
    P = dl.Problem.from_instance(inst)
    lam = rng.uniform(0, 1, 2 * inst.J).astype(np.float32)
    x = P.primal(torch.from_numpy(lam).cuda(), 0.05).cpu().numpy().astype(np.float64)
    xo = oracle.Problem(inst).eval(lam.astype(np.float64), 0.05, want_x=True).x
    assert np.all(np.abs(x - xo) <= 2e-6 * np.maximum(1.0, np.abs(xo)))


def test_families_solve_matches_oracle(dl):
    inst = synth.add_families(
        synth.greedy_budgets(synth.matching(8_000, 200, 27, ("poisson", 20, 1, 200))), 2, seed=8)
    opts = dict(gamma0=0.1, gamma_final=1e-3, halve_every=25, max_step=10.0, init_step=1e-5)
    Po = oracle.Problem(inst)
    ro = Po.solve(max_iters=4000, **opts)
    P = dl.Problem.from_instance(inst)
    lam, rg = P.solve(max_iters=4000, **opts)
    assert rg["iters"] > 0
    ev = Po.eval(lam.cpu().numpy().astype(np.float64), 1e-3)
    assert abs(rg["dual_obj"] - ev.dual) <= 1e-6 * abs(ev.dual)  # evaluation parity at lambda
    if ro["converged"] and rg["converged"]:
        assert abs(ev.dual - ro["dual"]) <= 2e-4 * abs(ro["dual"])
    # both rows of every destination stay dual feasible
    assert np.all(lam.cpu().numpy() >= 0)


def test_families_misuse(dl):
    inst = synth.add_families(synth.config("c1"), 2, seed=9)
    with pytest.raises(dl.DualipError):
        dl.Problem.from_instance(inst, storage="bf16")  # FP32 only
    P = dl.Problem.from_instance(inst)
    with pytest.raises(dl.DualipError):
        dl.Batch([P])  # the batched form takes one family
