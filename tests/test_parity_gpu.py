"""Parity of the CUDA dual evaluation (through the C ABI) with the FP64 oracle.

Tolerances (the gradient bound is per entry, because A x - b cancels):
  |grad_gpu_j - grad_oracle_j| <= 1e-5 * (|(A x)_j| + |b_j|) + 1e-6
  |g_gpu - g_oracle| <= 1e-6 * max(1, |g|)     (same for c^T x, ridge term)
  |Δ lambda^T (A x - b)| <= 1e-6 * max(1, sum_j |lambda_j| (|(A x)_j| + |b_j|))
                                               (a dot product that cancels)
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-5
OBJ_RTOL = 1e-6


@pytest.fixture(scope="module")
def dl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04621_gb300 import build

    build.build()
    import paper_2603_04621_gb300 as d

    return d


def bf16_round(x):
    """float32 -> bfloat16 (round to nearest even) -> float32, for finite x."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32)


def decoded(inst):
    return synth.Instance(inst.off, inst.dst, bf16_round(inst.c), bf16_round(inst.a), inst.b,
                          inst.J, name=inst.name + "[bf16]")


def dot_tol(lam, ax, b):
    """Bound on lambda^T (A x - b): 1e-6 relative to the sum of its terms' sizes."""
    lam = np.abs(np.asarray(lam, dtype=np.float64))
    return OBJ_RTOL * max(1.0, float(np.sum(lam * (np.abs(ax) + np.abs(np.asarray(b, np.float64))))))


def check_eval(d, inst, lam, gamma, weighted=False, storage="f32", P=None, Po=None, box=False):
    import torch

    P = P or d.Problem.from_instance(inst, storage=storage, primal_scaling=weighted,
                                     projection="box" if box else "simplex")
    ref_inst = decoded(inst) if storage == "bf16" else inst
    Po = Po or oracle.Problem(ref_inst, weighted=weighted, box=box)
    lam32 = np.asarray(lam, dtype=np.float32)
    grad, ev = P.dual_grad(torch.from_numpy(lam32).cuda(), gamma)
    grad = grad.cpu().numpy().astype(np.float64)
    eo = Po.eval(lam32.astype(np.float64), gamma)
    tol = GRAD_RTOL * (np.abs(eo.ax) + np.abs(inst.b.astype(np.float64))) + 1e-6
    err = np.abs(grad - eo.grad)
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, (f"{bad.size} gradient entries out of tolerance; worst "
                           f"{(err / tol).max():.3g}x at j={bad[:5]}, gpu={grad[bad[:5]]}, "
                           f"oracle={eo.grad[bad[:5]]}")
    for key, ref in (("dual_obj", eo.dual), ("primal_obj", eo.primal_lin), ("reg", eo.reg)):
        assert abs(ev[key] - ref) <= OBJ_RTOL * max(1.0, abs(ref)), (key, ev[key], ref)
    # lambda^T (A x - b) cancels near the optimum (terms of size |lambda_j| |(A x)_j|
    # summing to a small value), so it is relative to the size of its terms
    assert abs(ev["lambda_dot_grad"] - eo.mu_dot_grad) <= dot_tol(lam32, eo.ax, inst.b)
    assert abs(ev["infeas_l2"] - eo.infeas) <= 1e-5 * max(1.0, eo.infeas) + 1e-6 * np.linalg.norm(
        inst.b)
    return P, Po, grad, ev


def lam_points(inst, rng, n=3):
    pts = [np.zeros(inst.J)]
    for _ in range(n):
        pts.append(rng.uniform(0.0, 2.0, inst.J))
    return pts


@pytest.mark.parametrize("gamma", [0.1, 1e-3])
def test_c1_parity(dl, gamma):
    inst = synth.config("c1")
    rng = np.random.default_rng(1)
    P = Po = None
    for lam in lam_points(inst, rng):
        P, Po, _, _ = check_eval(dl, inst, lam, gamma, P=P, Po=Po)


@pytest.mark.parametrize("gamma", [0.1, 0.01, 1e-3])
def test_c2_shape_parity(dl, gamma):
    # the c2 laws at 2% of the sources: ~1M edges, >400 tiles, ragged tail
    inst = synth.config("c2", scale=0.02)
    rng = np.random.default_rng(2)
    P = Po = None
    for lam in lam_points(inst, rng, 2):
        P, Po, _, _ = check_eval(dl, inst, lam, gamma, P=P, Po=Po)


@pytest.mark.parametrize("weighted", [False, True])
def test_greedy_budget_parity_at_solver_points(dl, weighted):
    inst = synth.greedy_budgets(synth.matching(20_000, 500, 7, ("poisson", 50, 1, 500)))
    Po = oracle.Problem(inst, weighted=weighted)
    res = Po.solve(max_iters=300, stop_on_tol=False)
    P = None
    for gamma in (0.1, 1e-3):
        P, Po, _, _ = check_eval(dl, inst, res["mu"], gamma, weighted, P=P, Po=Po)


def test_adversarial_degrees(dl):
    # segment lengths around every class boundary of the kernel, plus
    # sources larger than a shared-memory tile
    degs = [0, 1, 31, 32, 33, 63, 64, 65, 96, 97, 127, 128, 129, 500, 1024, 1025, 2047, 2048,
            2049, 5000, 0, 3, 0, 100_000, 7]
    J = 120_000
    inst = synth.from_degrees(np.array(degs), J, 11, synth.DST_UNIFORM, b_frac=0.5)
    rng = np.random.default_rng(3)
    P = Po = None
    for gamma in (0.5, 1e-3, 1e-6):
        for lam in (np.zeros(J), rng.uniform(0, 1, J)):
            P, Po, _, _ = check_eval(dl, inst, lam, gamma, P=P, Po=Po)
            P, Po, _, _ = check_eval(dl, inst, lam, gamma, P=P, Po=Po)  # reuse: scratch reset


@pytest.mark.parametrize("weighted", [False, True])
def test_block_class_hub_sources(dl, weighted):
    """Sources far larger than a stage among ordinary ones, up to a million
    edges, at a slack, a moderate and a tiny gamma: the block class (all
    consumer warps of a CTA on one source, from global memory) up to 16
    stages, the multi-block class (chunks over the whole grid, the last CTA
    of a source finds its threshold) from there, with chunk-ragged degrees."""
    degs = np.array([1_000_000, 5, 250_000, 40, 3_201, 0, 60_000, 2, 20_000, 45_000, 51_200,
                     65_537, 4_801, 4_096])
    inst = synth.from_degrees(degs, 1_100_000, 19, synth.DST_UNIFORM, b_frac=0.3)
    rng = np.random.default_rng(44)
    P = Po = None
    for gamma in (50.0, 1e-2, 1e-5):
        for lam in (np.zeros(inst.J), rng.uniform(0, 1, inst.J)):
            P, Po, _, _ = check_eval(dl, inst, lam, gamma, weighted, P=P, Po=Po)


@pytest.mark.parametrize("weighted", [False, True])
def test_hub_sources_bf16_primal_and_repeat(dl, weighted):
    """Hub sources with BF16 storage against the oracle on the decoded data,
    the primal x edge by edge, and repeated evaluations bit for bit (the
    candidate lists fill in whatever order the chunks finish)."""
    import torch

    degs = np.array([400_000, 3, 90_000, 0, 77, 300_000, 12_345])
    inst = synth.from_degrees(degs, 500_000, 23, synth.DST_UNIFORM, b_frac=0.3)
    rng = np.random.default_rng(45)
    P = Po = None
    for gamma in (1.0, 3e-3):
        lam = rng.uniform(0, 1, inst.J)
        P, Po, _, _ = check_eval(dl, inst, lam, gamma, weighted, storage="bf16", P=P, Po=Po)
    lam = torch.from_numpy(rng.uniform(0, 1, inst.J).astype(np.float32)).cuda()
    for gamma in (1.0, 3e-3):
        g0, e0 = P.dual_grad(lam, gamma)
        for _ in range(3):
            g1, e1 = P.dual_grad(lam, gamma)
            assert torch.equal(g1, g0) and e1 == e0
        x = P.primal(lam, gamma).cpu().numpy().astype(np.float64)
        xo = Po.eval(lam.cpu().numpy().astype(np.float64), gamma, want_x=True).x
        assert np.all(np.abs(x - xo) <= 2e-5 * np.maximum(1.0, np.abs(xo)) + 1e-6)
        per_src = np.add.reduceat(x, inst.off[:-1][degs > 0])
        assert per_src.max() <= 1.0 + 1e-5
    P.close()


@pytest.mark.parametrize("order", ["caller", "degree"])
def test_hub_edges_in_destination_order(dl, order):
    """Hub sources are stored with their edges sorted by destination.  The
    primal comes back in the caller's edge order, with repeated destinations
    in a hub (ties of the sort) and hubs among sources kept in the caller's
    order (ascending degrees) or stored in degree order (widely spread small
    degrees around them)."""
    import torch

    rng = np.random.default_rng(47)
    if order == "caller":
        degs = np.array([3, 10, 40, 300, 70_000, 200_000])
    else:
        degs = np.concatenate([[200_000], rng.integers(5, 101, 6_000), [70_000],
                               rng.integers(5, 101, 6_000)])
    inst = synth.from_degrees(degs, 400_000, 29, synth.DST_UNIFORM, b_frac=0.3)
    hub = int(np.argmax(degs))
    e0 = int(inst.off[hub])
    # repeated (i, j) pairs inside the largest hub: separate variables with the
    # same destination, at places far apart in the caller's order
    inst.dst[e0 + 1000:e0 + 1100] = inst.dst[e0 + 150_000:e0 + 150_100]
    inst.dst[e0 + 7] = inst.dst[e0 + 199_990]
    for gamma, lam in ((1e-3, rng.uniform(0, 1, inst.J)), (5.0, np.zeros(inst.J))):
        P, Po, _, _ = check_eval(dl, inst, lam, gamma)
        lam32 = torch.from_numpy(lam.astype(np.float32)).cuda()
        x = P.primal(lam32, gamma).cpu().numpy().astype(np.float64)
        xo = Po.eval(lam.astype(np.float32).astype(np.float64), gamma, want_x=True).x
        assert np.all(np.abs(x - xo) <= 2e-5 * np.maximum(1.0, np.abs(xo)) + 1e-6), (
            np.abs(x - xo).max())
        P.close()


@pytest.mark.parametrize("storage,weighted", [("f32", False), ("f32", True), ("bf16", False)])
def test_small_degree_sources_at_solver_points(dl, storage, weighted):
    """The small-degree variant (mean degree at most 16: one lane per source of
    span <= 16, which projects a source with near-ties or a slack sum exactly
    on its own) on the Appendix B generator, at dual points of an actual ascent
    (where many sources leave the single-candidate exit) and at random ones."""
    inst = synth.appb(30_000, 400, 8.0)
    assert inst.E <= 16 * inst.I  # (with primal scaling: weights over eight orders)
    ref = decoded(inst) if storage == "bf16" else inst
    Po = oracle.Problem(ref, weighted=weighted)
    pts = [Po.solve(gamma0=0.01, gamma_final=0.01, halve_every=0, max_iters=n,
                    stop_on_tol=False)["mu"] for n in (30, 300)]
    pts.append(np.random.default_rng(46).uniform(0, 2, inst.J))
    P = None
    for lam in pts:
        for gamma in (0.1, 0.01, 1e-3):
            P, Po, _, _ = check_eval(dl, inst, lam, gamma, weighted, storage, P=P, Po=Po)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_widely_spread_weights_every_class(dl, storage):
    """Primal scaling with coefficients spread over four orders of magnitude
    (weights a^2 over eight): an active edge with a large alpha = 1/(gamma w)
    has x = alpha (d - t) with d - t far below |t|, which the weighted exact
    paths form in FP64.  Sources for the warp (degrees up to 500), block (a
    few stages) and multi-block (over 16 stages) classes, at dual points of a
    short ascent and at random ones."""
    degs = np.array([3, 40, 300, 5_000, 60_000, 12, 0, 90])
    inst = synth.greedy_budgets(synth.from_degrees(degs, 70_000, 29, synth.DST_UNIFORM,
                                                   a_lo=0.01, a_hi=100.0))
    ref = decoded(inst) if storage == "bf16" else inst
    Po = oracle.Problem(ref, weighted=True)
    pts = [Po.solve(gamma0=0.01, gamma_final=0.01, halve_every=0, max_iters=20,
                    stop_on_tol=False)["mu"], np.random.default_rng(47).uniform(0, 1, inst.J)]
    P = None
    for lam in pts:
        for gamma in (0.1, 1e-3):
            P, Po, _, _ = check_eval(dl, inst, lam, gamma, True, storage, P=P, Po=Po)


def test_many_tiny_sources_and_all_hot(dl):
    # degree-1 sources (tile capped by the source count) into 3 destinations
    inst = synth.from_degrees(np.ones(50_000, dtype=np.int64), 3, 12, synth.DST_UNIFORM,
                              c_law=synth.C_NEG_UNIFORM, b_frac=0.3)
    for gamma in (1.0, 1e-3):
        check_eval(dl, inst, np.array([0.0, 0.5, 5.0]), gamma)


def test_large_lambda_and_empty_rows(dl):
    inst = synth.matching(3000, 20_000, 13, ("poisson", 20, 0, 60), "zipf")
    assert np.bincount(inst.dst, minlength=inst.J).min() == 0  # some rows are empty
    P, Po, grad, ev = check_eval(dl, inst, np.full(inst.J, 1e6), 1e-3)
    assert ev["primal_obj"] == 0.0 and ev["reg"] == 0.0
    assert np.array_equal(grad, -inst.b.astype(np.float64))


def test_empty_problem(dl):
    inst = synth.Instance(np.zeros(5, dtype=np.int64), np.zeros(0, np.int32),
                          np.zeros(0, np.float32), np.zeros(0, np.float32),
                          np.arange(4, dtype=np.float32), 4)
    P, Po, grad, ev = check_eval(dl, inst, np.ones(4), 0.1)
    assert np.array_equal(grad, -np.arange(4))
    assert ev["dual_obj"] == pytest.approx(-6.0)


@pytest.mark.parametrize("storage,weighted", [("f32", False), ("f32", True), ("bf16", False)])
def test_unit_box_projection_parity(dl, storage, weighted):
    """The unit-box clamp (x_e in [0, 1], no sum constraint) against the oracle:
    c2-shaped sources, adversarial degrees (oversized sources read from global
    memory), and the primal x edge by edge."""
    import torch

    rng = np.random.default_rng(31)
    inst = synth.config("c2", scale=0.01)
    P = Po = None
    for gamma in (2.0, 0.05, 1e-3):
        P, Po, _, _ = check_eval(dl, inst, rng.uniform(0, 2, inst.J), gamma, weighted, storage,
                                 P=P, Po=Po, box=True)
    degs = [0, 1, 33, 500, 3300, 7, 0, 5000, 2]
    big = synth.from_degrees(np.array(degs), 8_000, 33, synth.DST_UNIFORM, b_frac=0.5)
    check_eval(dl, big, rng.uniform(0, 1, big.J), 0.2, weighted, storage, box=True)
    lam = rng.uniform(0, 1.5, inst.J).astype(np.float32)
    x = P.primal(torch.from_numpy(lam).cuda(), 0.05).cpu().numpy().astype(np.float64)
    xo = Po.eval(lam.astype(np.float64), 0.05, want_x=True).x
    assert np.all((x >= 0) & (x <= 1))
    assert np.all(np.abs(x - xo) <= 2e-6 * np.maximum(1.0, np.abs(xo)))


def test_unit_box_solve_matches_oracle(dl):
    inst = synth.greedy_budgets(synth.matching(10_000, 300, 26, ("poisson", 20, 1, 200)))
    opts = dict(gamma0=0.1, gamma_final=0.01, halve_every=25, max_step=10.0, init_step=1e-5)
    Po = oracle.Problem(inst, box=True)
    ro = Po.solve(max_iters=3000, **opts)
    P = dl.Problem.from_instance(inst, projection="box")
    lam, rg = P.solve(max_iters=3000, **opts)
    assert ro["converged"] and rg["converged"]
    ev = Po.eval(lam.cpu().numpy().astype(np.float64), 0.01)
    assert abs(rg["dual_obj"] - ev.dual) <= 1e-6 * abs(ev.dual)
    assert abs(ev.dual - ro["dual"]) <= 2e-4 * abs(ro["dual"])
    # the batched and serving forms take simplex problems only
    with pytest.raises(dl.DualipError):
        dl.Batch([P])


@pytest.mark.parametrize("weighted", [False, True])
def test_evaluations_repeat_bit_for_bit(dl, weighted):
    """The pass hands tiles to CTAs and sources to warps dynamically, yet every
    output of an evaluation repeats exactly: A x and the objective partials are
    fixed-point sums (exact in any order) and the per-row terms are reduced in
    a fixed order."""
    import torch

    inst = synth.config("c2", scale=0.05)
    P = dl.Problem.from_instance(inst, primal_scaling=weighted)
    lam = torch.from_numpy(np.random.default_rng(9).uniform(0, 1.5, inst.J).astype(np.float32))
    lam = lam.cuda()
    for gamma in (1e-3, 0.1):
        g0, e0 = P.dual_grad(lam, gamma)
        g0 = g0.cpu().numpy()
        for _ in range(4):
            g1, e1 = P.dual_grad(lam, gamma)
            assert np.array_equal(g1.cpu().numpy(), g0)
            assert e1 == e0
    P.close()


@pytest.mark.parametrize("weighted", [False, True])
def test_bf16_storage_parity(dl, weighted):
    inst = synth.config("c2", scale=0.01)
    rng = np.random.default_rng(4)
    for gamma in (0.1, 1e-3):
        check_eval(dl, inst, rng.uniform(0, 2, inst.J), gamma, weighted, storage="bf16")


def test_primal_matches_oracle(dl):
    import torch

    inst = synth.config("c2", scale=0.005)
    Po = oracle.Problem(inst)
    P = dl.Problem.from_instance(inst)
    lam = np.random.default_rng(5).uniform(0, 2, inst.J).astype(np.float32)
    for gamma in (0.2, 1e-3):
        x = P.primal(torch.from_numpy(lam).cuda(), gamma).cpu().numpy()
        xo = Po.eval(lam.astype(np.float64), gamma, want_x=True).x
        assert np.all(x >= 0)
        assert np.abs(x - xo).max() <= 2e-5, np.abs(x - xo).max()
        sums = np.add.reduceat(x, inst.off[:-1]) if inst.E else x
        assert sums.max() <= 1 + 1e-5


def degree_cv(inst):
    deg = np.diff(inst.off).astype(np.float64)
    return deg.std() / deg.mean()


@pytest.mark.parametrize("storage,weighted", [("f32", False), ("bf16", True)])
def test_degree_order_storage(dl, storage, weighted):
    """Degrees Uniform[5,100] (the batched recipe) spread widely, so the problem
    is stored in degree order: evaluations, the primal in the caller's edge
    order, device inputs and the range check all hold on that path."""
    import torch

    inst = synth.matching(20_000, 3_000, 17, ("uniform", 5, 100), "zipf")
    assert degree_cv(inst) > 0.3  # widely spread degrees: the cost model picks degree order
    rng = np.random.default_rng(9)
    P = Po = None
    for gamma in (0.1, 1e-3):
        P, Po, _, _ = check_eval(dl, inst, rng.uniform(0, 2, inst.J), gamma, weighted,
                                 storage=storage, P=P, Po=Po)
    lam = rng.uniform(0, 2, inst.J).astype(np.float32)
    ref = decoded(inst) if storage == "bf16" else inst
    xo = oracle.Problem(ref, weighted=weighted).eval(lam.astype(np.float64), 1e-2,
                                                     want_x=True).x
    x = P.primal(torch.from_numpy(lam).cuda(), 1e-2).cpu().numpy()
    assert np.abs(x - xo).max() <= 2e-5, np.abs(x - xo).max()
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()  # noqa: E731
    Pd = dl.Problem(t(inst.off), t(inst.dst), t(inst.c), t(inst.a), t(inst.b), inst.J,
                    storage=storage, primal_scaling=weighted)
    check_eval(dl, inst, lam, 1e-2, weighted, storage=storage, P=Pd)
    bad = synth.Instance(inst.off, inst.dst.copy(), inst.c, inst.a, inst.b, inst.J)
    bad.dst[inst.E // 2] = -1
    with pytest.raises(dl.DualipError) as ei:
        dl.Problem.from_instance(bad, storage=storage)
    assert ei.value.status == dl.DUALIP_EINVAL


def test_host_buffer_entry_point(dl):
    inst = synth.config("c2", scale=0.005)
    P = dl.Problem.from_instance(inst)
    Po = oracle.Problem(inst)
    lam = np.random.default_rng(6).uniform(0, 2, inst.J).astype(np.float32)
    grad = np.empty(inst.J, dtype=np.float32)
    import ctypes

    ev = dl.dualip_dual_grad_host(P.h, lam.ctypes.data, 1e-2, grad.ctypes.data, dl._stream())
    eo = Po.eval(lam.astype(np.float64), 1e-2)
    tol = GRAD_RTOL * (np.abs(eo.ax) + np.abs(inst.b)) + 1e-6
    assert np.all(np.abs(grad - eo.grad) <= tol)
    assert abs(ev.dual_obj - eo.dual) <= OBJ_RTOL * abs(eo.dual)
    del ctypes


def test_invalid_inputs_are_rejected(dl):
    import torch

    inst = synth.config("c1")
    bad = synth.Instance(inst.off, inst.dst.copy(), inst.c, inst.a, inst.b, inst.J)
    bad.dst[17] = inst.J  # out of range
    with pytest.raises(dl.DualipError) as ei:
        dl.Problem.from_instance(bad)
    assert ei.value.status == dl.DUALIP_EINVAL
    nan = synth.Instance(inst.off, inst.dst, inst.c.copy(), inst.a, inst.b, inst.J)
    nan.c[3] = np.nan
    with pytest.raises(dl.DualipError):
        dl.Problem.from_instance(nan)
    P = dl.Problem.from_instance(inst)
    lam = torch.zeros(inst.J, device="cuda")
    for g in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(dl.DualipError):
            P.dual_grad(lam, g)
    # the handle stays usable after rejected calls
    check_eval(dl, inst, np.zeros(inst.J), 0.1, P=P)


def test_device_inputs(dl):
    import torch

    inst = synth.config("c2", scale=0.005)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    P = dl.Problem(t(inst.off), t(inst.dst), t(inst.c), t(inst.a), t(inst.b), inst.J)
    check_eval(dl, inst, np.random.default_rng(8).uniform(0, 1, inst.J), 1e-2, P=P)


def test_full_c2_parity(dl):
    """The benchmark workload at full size, in the benchmark's launch configuration."""
    inst = synth.config("c2")
    rng = np.random.default_rng(9)
    lam = rng.uniform(0, 1.0, inst.J)
    check_eval(dl, inst, lam, 1e-3)
