"""dualip_solve on the GPU against the FP64 oracle's ascent (same definition)."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def dl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04621_gb300 import build

    build.build()
    import paper_2603_04621_gb300 as d

    return d


OPTS = dict(gamma0=0.1, gamma_final=1e-3, halve_every=25, max_step=10.0, init_step=1e-5)


def test_c1_two_thousand_iterations(dl):
    """c1 with binding (greedy-load) budgets, exactly 2000 ascent iterations."""
    inst = synth.greedy_budgets(synth.config("c1"))
    Po = oracle.Problem(inst)
    ro = Po.solve(max_iters=2000, stop_on_tol=False, want_trace=True, **OPTS)
    P = dl.Problem.from_instance(inst)
    lam, rg, tr = P.solve(max_iters=2000, stop_on_tol=0, trace=True, **OPTS)
    assert rg["iters"] == ro["iters"] == 2000
    # identical gamma schedule, and the early trajectory agrees closely
    assert np.array_equal(tr[:, 0], ro["trace"][:, 0])
    g_o, g_g = ro["trace"][:60, 1], tr[:60, 1]
    assert np.all(np.abs(g_g - g_o) <= 1e-5 * np.abs(g_o))
    # both reach the same optimum of the final smoothed dual
    lam = lam.cpu().numpy().astype(np.float64)
    ev = Po.eval(lam, 1e-3)
    assert abs(rg["dual_obj"] - ev.dual) <= 1e-6 * abs(ev.dual)  # evaluation parity at lam
    assert abs(ev.dual - ro["dual"]) <= 1e-6 * abs(ro["dual"])
    # dual KKT at the GPU's point
    scale = np.abs(ev.ax) + np.abs(inst.b)
    assert np.all(lam >= 0)
    assert np.all(ev.grad <= 1e-4 * scale + 1e-6)
    assert abs(ev.mu_dot_grad) <= 1e-4 * abs(ev.dual)


def test_solve_to_gap_matches_oracle(dl):
    inst = synth.greedy_budgets(synth.matching(30_000, 600, 21, ("poisson", 50, 1, 500)))
    Po = oracle.Problem(inst)
    ro = Po.solve(max_iters=3000, **OPTS)
    assert ro["converged"]
    P = dl.Problem.from_instance(inst)
    lam, rg = P.solve(max_iters=3000, **OPTS)
    assert rg["converged"]
    assert rg["gap_rel"] <= 1e-4 and rg["infeas_rel"] <= 1e-4
    # same stopping rule, similar work, same objective to the stopping tolerance
    assert abs(rg["iters"] - ro["iters"]) <= max(60, 0.25 * ro["iters"])
    assert abs(rg["dual_obj"] - ro["dual"]) <= 2e-4 * abs(ro["dual"])
    ev = Po.eval(lam.cpu().numpy().astype(np.float64), 1e-3)
    assert abs(rg["dual_obj"] - ev.dual) <= 1e-6 * abs(ev.dual)


@pytest.mark.parametrize("row_normalize,weighted", [(0, False), (1, True)])
def test_solve_variants(dl, row_normalize, weighted):
    inst = synth.greedy_budgets(synth.matching(8_000, 200, 22, ("poisson", 30, 1, 200)))
    Po = oracle.Problem(inst, weighted=weighted)
    ro = Po.solve(max_iters=400, stop_on_tol=False, row_normalize=bool(row_normalize), **OPTS)
    P = dl.Problem.from_instance(inst, primal_scaling=weighted)
    lam, rg = P.solve(max_iters=400, stop_on_tol=0, row_normalize=row_normalize, **OPTS)
    ev = Po.eval(lam.cpu().numpy().astype(np.float64), 1e-3)
    assert abs(rg["dual_obj"] - ev.dual) <= 1e-6 * abs(ev.dual)
    assert abs(ev.dual - ro["dual"]) <= 1e-4 * abs(ro["dual"])


def test_graph_and_eager_agree(dl):
    inst = synth.greedy_budgets(synth.matching(5_000, 100, 23, ("poisson", 20, 1, 100)))
    P = dl.Problem.from_instance(inst)
    l1, r1 = P.solve(max_iters=200, stop_on_tol=0, use_graph=1, **OPTS)
    l2, r2 = P.solve(max_iters=200, stop_on_tol=0, use_graph=0, **OPTS)
    # the same kernels in the same order, and every sum is exact or in a fixed
    # order: the two ascents are the same bit for bit
    assert np.array_equal(l1.cpu().numpy(), l2.cpu().numpy())
    assert r1 == r2


def test_state_export_import_resume(dl):
    """An ascent stopped after k iterations, exported, imported into a fresh
    handle of the same problem and resumed for n more iterations ends exactly
    where k + n uninterrupted iterations end (across gamma changes and adaptive
    restarts), and the resumed solve reaches the oracle's optimum."""
    inst = synth.greedy_budgets(synth.matching(20_000, 400, 24, ("poisson", 30, 1, 300)))
    kw = dict(stop_on_tol=0, **OPTS)
    A = dl.Problem.from_instance(inst)
    lam_a, ra, tr_a = A.solve(max_iters=180, trace=True, **kw)
    B = dl.Problem.from_instance(inst)
    B.solve(max_iters=67, **kw)
    state = B.export_state()
    B.close()
    C = dl.Problem.from_instance(inst)
    C.import_state(state)
    lam_c, rc, tr_c = C.solve(max_iters=113, resume=1, trace=True, **kw)
    assert np.array_equal(lam_a.cpu().numpy(), lam_c.cpu().numpy())
    assert ra["dual_obj"] == rc["dual_obj"] and ra["gap_rel"] == rc["gap_rel"]
    assert np.array_equal(tr_a[67:], tr_c)  # trace rows of the resumed call start at 0
    # resuming on the same handle needs no export
    lam_r, rr = A.solve(max_iters=40, resume=1, **kw)
    lam_c2, rc2 = C.solve(max_iters=40, resume=1, **kw)
    assert np.array_equal(lam_r.cpu().numpy(), lam_c2.cpu().numpy())
    # to convergence from the imported state: the oracle's optimum
    lam_f, rf = C.solve(max_iters=5000, resume=1, **OPTS)
    assert rf["converged"]
    ro = oracle.Problem(inst).solve(max_iters=5000, **OPTS)
    assert ro["converged"]
    assert abs(rf["dual_obj"] - ro["dual"]) <= 2e-4 * abs(ro["dual"])
    # misuse
    D = dl.Problem.from_instance(inst)
    with pytest.raises(dl.DualipError):
        D.solve(resume=1)  # nothing to resume
    with pytest.raises(dl.DualipError):
        D.export_state()
    other = synth.greedy_budgets(synth.matching(2_000, 50, 25, ("poisson", 10, 1, 50)))
    with pytest.raises(dl.DualipError):
        dl.Problem.from_instance(other).import_state(state)
    bad = state.copy()
    bad[:8] = 0
    with pytest.raises(dl.DualipError):
        D.import_state(bad)


def test_gamma_schedule_golden(dl):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "gamma_schedule_section7.txt"))
            if ln.strip() and not ln.startswith("#")]
    prm = {r[0]: float(r[1]) for r in rows if not r[0].isdigit()}
    pts = [(int(r[0]), float(r[1])) for r in rows if r[0].isdigit()]
    inst = synth.greedy_budgets(synth.config("c1"))
    P = dl.Problem.from_instance(inst)
    _, _, tr = P.solve(max_iters=160, stop_on_tol=0, trace=True, gamma0=prm["gamma0"],
                       gamma_final=prm["gamma_final"], halve_every=int(prm["halve_every"]))
    for k, g in pts:
        assert tr[k, 0] == pytest.approx(g, rel=1e-15)


def test_warm_start_and_invalid_opts(dl):
    inst = synth.greedy_budgets(synth.config("c1"))
    P = dl.Problem.from_instance(inst)
    lam, r = P.solve(max_iters=2000, **OPTS)
    assert r["converged"]
    # warm start from the solution at the final gamma converges at the first check
    lam2, r2 = P.solve(lam0=lam, gamma0=1e-3, gamma_final=1e-3, halve_every=0, max_step=0.1,
                       max_iters=500)
    assert r2["converged"] and r2["iters"] <= 50
    with pytest.raises(dl.DualipError):
        P.solve(gamma0=1e-3, gamma_final=1e-2)
    with pytest.raises(dl.DualipError):
        P.solve(max_iters=0)


def test_recurring_solve_warm_starts_on_a_perturbed_instance(dl):
    """Recurring solves: the costs move by about 1%, and the previous optimum
    started at the final gamma reaches the 1e-4 gap in fewer iterations than
    the cold schedule, at the same dual value."""
    base = synth.greedy_budgets(synth.config("c2"))  # converges in 190 iterations
    P = dl.Problem.from_instance(base)
    lam, r = P.solve()
    assert r["converged"]
    rng = np.random.default_rng(17)
    c2 = (base.c * (1.0 + 0.01 * rng.standard_normal(base.E))).astype(np.float32)
    moved = synth.Instance(base.off, base.dst, c2, base.a, base.b, base.J)
    Q = dl.Problem.from_instance(moved)
    _, cold = Q.solve()
    _, warm = Q.solve(lam0=lam, gamma0=1e-3, gamma_final=1e-3, halve_every=0)
    assert cold["converged"] and warm["converged"]
    assert warm["iters"] < cold["iters"]
    assert abs(warm["dual_obj"] - cold["dual_obj"]) <= 3e-4 * abs(cold["dual_obj"])
