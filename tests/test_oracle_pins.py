"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check is a closed form,
an invariant, a brute-force enumeration or an independent library solve
(scipy's HiGHS / SLSQP), so that a dropped term, a wrong sign, index or
transposed operand in the oracle fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth

RNG = np.random.default_rng(12345)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Per-source projection (Section 3.2, Eqs. 4-5)
# --------------------------------------------------------------------------
def _block_obj(x, r, alpha):
    # per-source objective of the block problem: sum x^2/(2 alpha) - r x
    return float(np.sum(x * x / (2 * alpha) - r * x))


def _brute_force_projection(r, alpha):
    """Minimise sum x^2/(2 alpha) - r x over {x >= 0, sum x <= 1} by trying every
    support S and both states of the sum constraint (pure-Python loops)."""
    d = len(r)
    best, best_x = np.inf, None
    for mask in range(1 << d):
        S = [k for k in range(d) if mask >> k & 1]
        for tight in (False, True):
            x = np.zeros(d)
            if tight:
                if not S:
                    continue
                sa = sum(alpha[k] for k in S)
                tau = (sum(alpha[k] * r[k] for k in S) - 1.0) / sa
                for k in S:
                    x[k] = alpha[k] * (r[k] - tau)
            else:
                for k in S:
                    x[k] = alpha[k] * r[k]
            if np.any(x < -1e-15) or x.sum() > 1 + 1e-13:
                continue
            f = _block_obj(x, r, alpha)
            if f < best - 1e-15:
                best, best_x = f, x
    return best_x


@pytest.mark.parametrize("method", ["sort", "michelot"])
def test_projection_lone_candidate(method):
    """x = alpha (r - t)_+ with sum x <= 1 (Eqs. 4-5).  If r_1 >= 1/alpha_1 and
    every other r_e <= r_1 - 1/alpha_1, the threshold t = r_1 - 1/alpha_1 >= 0
    meets the KKT conditions with x_1 = 1 and x_e = 0 for e > 1.  Once a runner-up
    passes that bound, it takes mass and x_1 < 1."""
    rng = np.random.default_rng(17)
    for _ in range(300):
        d = int(rng.integers(1, 12))
        al = rng.uniform(0.2, 5.0, d)
        t = rng.uniform(0.0, 2.0)
        r = np.empty(d)
        r[0] = t + 1.0 / al[0]
        r[1:] = t - rng.uniform(1e-9, 3.0, d - 1)
        x, tau = oracle.project(r, al, method)
        assert x[0] == pytest.approx(1.0, abs=1e-14) and np.all(x[1:] == 0.0)
        assert tau == pytest.approx(t, abs=1e-12)
        if d > 1:
            r2 = r.copy()
            r2[1] = t + 1e-3
            x2, _ = oracle.project(r2, al, method)
            assert x2[1] > 0.0 and x2[0] < 1.0 and x2.sum() == pytest.approx(1.0, abs=1e-13)


@pytest.mark.parametrize("method", ["sort", "michelot"])
def test_projection_closed_forms(method):
    # d = 1: x = clamp(r * alpha, 0, 1)
    for r in (-2.0, 0.0, 0.3, 0.99, 1.0, 7.5):
        x, _ = oracle.project([r], [1.0], method)
        assert x[0] == pytest.approx(min(max(r, 0.0), 1.0), abs=1e-15)
    # all r <= 0 gives x = 0 and tau = 0
    x, tau = oracle.project([-1.0, -0.5, 0.0, -3.0], [2.0, 1.0, 5.0, 1.0], method)
    assert np.all(x == 0) and tau == 0
    # sum of alpha r_+ <= 1: x = alpha r_+ and tau = 0
    r = np.array([0.1, -0.2, 0.15, 0.3])
    al = np.array([1.0, 3.0, 2.0, 0.5])
    x, tau = oracle.project(r, al, method)
    assert tau == 0 and np.allclose(x, al * np.maximum(r, 0), atol=1e-15)
    # all r equal to t > 0, alpha = 1: x_j = min(t, 1/d)
    for d in (1, 2, 5, 17):
        for t in (0.01, 1.0 / d, 0.5, 3.0):
            x, _ = oracle.project(np.full(d, t), 1.0, method)
            assert np.allclose(x, min(t, 1.0 / d), atol=1e-14)


@pytest.mark.parametrize("weighted", [False, True])
def test_projection_kkt(weighted):
    for trial in range(400):
        d = int(RNG.integers(1, 60))
        r = RNG.normal(0.0, 1.0, d) * RNG.choice([0.01, 1.0, 30.0])
        al = RNG.uniform(0.2, 5.0, d) if weighted else np.full(d, RNG.uniform(0.1, 50.0))
        x, tau = oracle.project(r, al, "sort")
        assert np.all(x >= 0)
        assert x.sum() <= 1 + 1e-12
        assert tau >= 0
        assert abs(tau * (1 - x.sum())) <= 1e-12 * max(1.0, abs(tau))
        act = x > 0
        assert np.allclose(x[act], al[act] * (r[act] - tau), rtol=1e-12, atol=1e-14)
        assert np.all(r[~act] <= tau + 1e-12 * max(1.0, abs(tau)))


def test_projection_brute_force_small():
    for trial in range(150):
        d = int(RNG.integers(1, 9))
        r = RNG.normal(0.3, 1.0, d)
        al = RNG.uniform(0.3, 4.0, d)
        xb = _brute_force_projection(r, al)
        for method in ("sort", "michelot"):
            x, _ = oracle.project(r, al, method)
            assert np.allclose(x, xb, atol=1e-12), (r, al, x, xb)


def test_projection_sort_matches_michelot():
    for trial in range(300):
        d = int(RNG.integers(1, 300))
        r = RNG.lognormal(0.0, 1.0, d) - RNG.uniform(0, 3, d)
        al = RNG.uniform(0.5, 2000.0, d)
        x1, t1 = oracle.project(r, al, "sort")
        x2, t2 = oracle.project(r, al, "michelot")
        assert abs(t1 - t2) <= 1e-13 * max(1.0, abs(t1))
        assert np.allclose(x1, x2, atol=1e-13)


# --------------------------------------------------------------------------
# Dual function and Danskin gradient (Section 3.1, Eq. 2)
# --------------------------------------------------------------------------
def _tiny(I=40, J=7, seed=5, deg=("uniform", 1, 5), lognormal=True):
    inst = synth.matching(I, J, seed, deg, "uniform", c_law="lognormal" if lognormal else "uniform")
    return synth.greedy_budgets(inst)


def _dense_A(inst):
    A = np.zeros((inst.J, inst.E))
    A[inst.dst, np.arange(inst.E)] = inst.a
    return A


@pytest.mark.parametrize("weighted", [False, True])
def test_sources_are_independent_blocks(weighted):
    """Section 3.1: C is a product of one simplex per source, so the minimiser
    splits by source.  Reordering the sources, and the edges inside each
    source, reorders x the same way and leaves A x, the gradient and every
    scalar as they were (up to the order of FP64 sums)."""
    inst = _tiny(I=300, J=12, seed=51, deg=("uniform", 1, 12))
    rng = np.random.default_rng(52)
    perm = rng.permutation(inst.I)
    edges = []
    for i in perm:
        seg = np.arange(inst.off[i], inst.off[i + 1])
        edges.append(rng.permutation(seg))
    e_new = np.concatenate(edges).astype(np.int64)
    deg = np.diff(inst.off)[perm]
    off2 = np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)
    moved = synth.Instance(off2, inst.dst[e_new], inst.c[e_new], inst.a[e_new], inst.b, inst.J)
    lam = rng.uniform(0.0, 1.5, inst.J)
    for gamma in (0.3, 1e-3):
        e1 = oracle.Problem(inst, weighted=weighted).eval(lam, gamma, want_x=True)
        e2 = oracle.Problem(moved, weighted=weighted).eval(lam, gamma, want_x=True)
        assert np.allclose(e2.x, e1.x[e_new], rtol=0, atol=1e-13)
        assert np.allclose(e2.ax, e1.ax, rtol=1e-12, atol=1e-13)
        assert np.allclose(e2.grad, e1.grad, rtol=1e-12, atol=1e-13)
        for key in ("dual", "primal_lin", "reg", "infeas"):
            a, b = getattr(e1, key), getattr(e2, key)
            assert abs(a - b) <= 1e-12 * max(1.0, abs(a)), key


@pytest.mark.parametrize("weighted", [False, True])
def test_gradient_is_central_difference(weighted):
    inst = _tiny()
    P = oracle.Problem(inst, weighted=weighted)
    for gamma in (0.5, 0.05, 0.003):
        for trial in range(4):
            mu = RNG.uniform(0.0, 1.5, inst.J)
            ev = P.eval(mu, gamma)
            for j in range(inst.J):
                h = 1e-6 * max(1.0, abs(mu[j]))
                e = np.zeros(inst.J)
                e[j] = h
                fd = (P.eval(mu + e, gamma).dual - P.eval(mu - e, gamma).dual) / (2 * h)
                scale = abs(ev.ax[j]) + abs(inst.b[j]) + 1.0
                assert abs(fd - ev.grad[j]) <= 1e-6 * scale, (gamma, j, fd, ev.grad[j])


def test_dual_value_matches_definition_by_hand():
    """g(mu) = sum_e (c_e + a_e mu_j) x_e + (gamma/2) sum x^2 - mu^T b, with x the
    block projections computed here by brute force, and grad = A x - b."""
    inst = _tiny(I=12, J=4, seed=9)
    P = oracle.Problem(inst)
    A = _dense_A(inst)
    gamma = 0.07
    mu = RNG.uniform(0, 1, inst.J)
    x = np.zeros(inst.E)
    for i in range(inst.I):
        s = slice(inst.off[i], inst.off[i + 1])
        r = -(inst.c[s].astype(float) + inst.a[s].astype(float) * mu[inst.dst[s]])
        x[s] = _brute_force_projection(r, np.full(r.shape, 1.0 / gamma))
    g = float((inst.c + A.T @ mu) @ x + 0.5 * gamma * x @ x - mu @ inst.b)
    ev = P.eval(mu, gamma, want_x=True)
    assert np.allclose(ev.x, x, atol=1e-12)
    assert ev.dual == pytest.approx(g, rel=1e-12, abs=1e-12)
    assert np.allclose(ev.grad, A @ x - inst.b, atol=1e-10)
    assert ev.primal_lin == pytest.approx(float(inst.c.astype(float) @ x), abs=1e-12)
    assert ev.reg == pytest.approx(0.5 * gamma * float(x @ x), abs=1e-14)
    assert ev.infeas == pytest.approx(float(np.linalg.norm(np.maximum(A @ x - inst.b, 0))),
                                      abs=1e-10)


def test_concavity_and_lipschitz():
    inst = _tiny(I=200, J=15, seed=3, deg=("uniform", 1, 10))
    P = oracle.Problem(inst)
    A = _dense_A(inst)
    norm2 = float(np.linalg.norm(A, 2) ** 2)
    assert P.norm2_sq() == pytest.approx(norm2, rel=1e-12)
    for gamma in (0.3, 0.01):
        L = norm2 / gamma
        for trial in range(20):
            m1, m2 = RNG.uniform(0, 2, inst.J), RNG.uniform(0, 2, inst.J)
            e1, e2 = P.eval(m1, gamma), P.eval(m2, gamma)
            for t in (0.25, 0.5, 0.8):
                et = P.eval(t * m1 + (1 - t) * m2, gamma)
                assert et.dual >= t * e1.dual + (1 - t) * e2.dual - 1e-9 * (1 + abs(et.dual))
            assert np.linalg.norm(e1.grad - e2.grad) <= L * np.linalg.norm(m1 - m2) * (1 + 1e-12)


def test_weak_duality():
    # b >= 0 makes x = 0 feasible with objective 0, so g(mu) <= 0 for mu >= 0
    inst = _tiny(I=100, J=10, seed=11)
    P = oracle.Problem(inst)
    for trial in range(30):
        mu = RNG.uniform(0, 3, inst.J) * RNG.choice([0.0, 1.0, 10.0])
        assert P.eval(mu, RNG.choice([1.0, 0.1, 0.001])).dual <= 1e-12


# --------------------------------------------------------------------------
# Row normalisation, primal scaling (Section 5.1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("weighted", [False, True])
def test_row_scale_makes_unit_rows(weighted):
    inst = _tiny(I=300, J=20, seed=17, deg=("uniform", 1, 10))
    inst.b[3] = 1.0
    P = oracle.Problem(inst, weighted=weighted)
    D = P.row_scale()
    A = _dense_A(inst)
    w = np.where(inst.a != 0, inst.a.astype(float) ** 2, 1.0) if weighted else np.ones(inst.E)
    As = (D[:, None] * A) / np.sqrt(w)[None, :]
    M = As @ As.T
    nz = np.abs(A).sum(1) > 0
    # Lemma 1 with one family: diag(A' A'^T) = I, and here all of A' A'^T = I
    assert np.allclose(np.diag(M)[nz], 1.0, atol=1e-12)
    assert np.allclose(M - np.diag(np.diag(M)), 0.0, atol=1e-15)
    assert np.all(D[~nz] == 1.0)


def test_row_scale_zero_row_is_one():
    inst = _tiny(I=30, J=9, seed=2)
    used = np.unique(inst.dst)
    P = oracle.Problem(inst)
    D = P.row_scale()
    unused = np.setdiff1d(np.arange(inst.J), used)
    assert np.all(D[unused] == 1.0)


def test_primal_scaling_constant_v_is_gamma_rescale():
    # v = |a| = kappa everywhere gives w = kappa^2: same as gamma * kappa^2 unweighted
    inst = _tiny(I=80, J=9, seed=21)
    kappa = np.float32(1.75)
    inst.a[:] = kappa
    Pw = oracle.Problem(inst, weighted=True)
    Pu = oracle.Problem(inst, weighted=False)
    for gamma in (0.2, 0.01):
        mu = RNG.uniform(0, 1, inst.J)
        ew = Pw.eval(mu, gamma, want_x=True)
        eu = Pu.eval(mu, gamma * float(kappa) ** 2, want_x=True)
        assert np.allclose(ew.x, eu.x, atol=1e-13)
        assert ew.dual == pytest.approx(eu.dual, rel=1e-13)


# --------------------------------------------------------------------------
# Tiny LPs: exact optimum, regularisation bounds, solver fixed point
# --------------------------------------------------------------------------
def _lp_parts(inst):
    """min c^T x, G x <= h with G = [per-source sums; A; -I]."""
    E = inst.E
    rows, h = [], []
    for i in range(inst.I):
        row = np.zeros(E)
        row[inst.off[i]:inst.off[i + 1]] = 1.0
        rows.append(row)
        h.append(1.0)
    A = _dense_A(inst)
    for j in range(inst.J):
        rows.append(A[j])
        h.append(float(inst.b[j]))
    for e in range(E):
        row = np.zeros(E)
        row[e] = -1.0
        rows.append(row)
        h.append(0.0)
    return inst.c.astype(float), np.array(rows), np.array(h)


def _lp_vertex_enum(inst):
    c, G, h = _lp_parts(inst)
    n = G.shape[1]
    best = np.inf
    for S in itertools.combinations(range(G.shape[0]), n):
        GS = G[list(S)]
        if abs(np.linalg.det(GS)) < 1e-12:
            continue
        x = np.linalg.solve(GS, h[list(S)])
        if np.all(G @ x <= h + 1e-9):
            best = min(best, float(c @ x))
    return best


def _tiny_lp(seed):
    inst = synth.matching(4, 3, seed, ("uniform", 1, 2), "uniform", c_law="uniform")
    # tighten budgets so that some bind
    return synth.greedy_budgets(inst, rho=(0.3, 0.6))


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_tiny_lp_bounds_and_recovery(seed):
    scipy_opt = pytest.importorskip("scipy.optimize")
    inst = _tiny_lp(seed)
    c, G, h = _lp_parts(inst)
    p_enum = _lp_vertex_enum(inst)
    lp = scipy_opt.linprog(c, A_ub=G, b_ub=h, bounds=(None, None), method="highs")
    assert lp.status == 0
    assert p_enum == pytest.approx(lp.fun, abs=1e-9)
    P = oracle.Problem(inst)
    for gamma in (0.2, 0.02, 1e-3):
        res = P.solve(gamma0=gamma, gamma_final=gamma, halve_every=0, max_step=1.0 / P.norm2_sq()
                      * gamma, init_step=1e-3 * gamma, max_iters=20000, stop_on_tol=False,
                      row_normalize=False)
        ev = P.eval(res["mu"], gamma)
        gstar = ev.dual
        # the regularised optimum of the same QP, solved directly
        cons = [{"type": "ineq", "fun": lambda x, G=G, h=h: h - G @ x}]
        qp = scipy_opt.minimize(lambda x: c @ x + 0.5 * gamma * x @ x, np.zeros(inst.E),
                                jac=lambda x: c + gamma * x, constraints=cons, method="SLSQP",
                                options=dict(ftol=1e-14, maxiter=500))
        assert gstar == pytest.approx(qp.fun, abs=2e-6 * max(1.0, abs(qp.fun)))
        # p*_LP <= g*(gamma) <= p*_LP + gamma * I / 2
        assert p_enum - 1e-9 <= gstar + 2e-6
        assert gstar <= p_enum + gamma * inst.I / 2 + 1e-9
        # dual KKT at the solver's point: mu >= 0, grad <= tol, mu_j grad_j ~ 0
        mu = res["mu"]
        assert np.all(mu >= 0)
        assert np.all(ev.grad <= 1e-5)
        assert np.all(np.abs(mu * ev.grad) <= 1e-5)


def test_projected_gradient_reaches_same_optimum():
    """Plain projected gradient with step 1/L converges to the g* of the AGD."""
    inst = _tiny(I=60, J=6, seed=31)
    P = oracle.Problem(inst)
    gamma = 0.05
    L = P.norm2_sq() / gamma
    mu = np.zeros(inst.J)
    for _ in range(20000):
        mu = np.maximum(0.0, mu + P.eval(mu, gamma).grad / L)
    g_pg = P.eval(mu, gamma).dual
    res = P.solve(gamma0=gamma, gamma_final=gamma, halve_every=0, max_step=10 * gamma,
                  max_iters=5000, stop_on_tol=False)
    assert P.eval(res["mu"], gamma).dual == pytest.approx(g_pg, abs=1e-8 * max(1, abs(g_pg)))


def test_adaptive_restart_reaches_the_quasi_newton_optimum():
    """The ascent with its adaptive momentum restart converges to the optimum of
    the smoothed, row-normalised dual that an unrelated method (L-BFGS-B with
    bounds lambda' >= 0, from scipy) finds, and gets there in fewer iterations
    than the ascent without the restart (the restart keeps the accelerated
    method monotone where its step overshoots)."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    inst = synth.greedy_budgets(synth.config("c1"))
    P = oracle.Problem(inst)
    D = P.row_scale()
    gamma = 1e-3

    def neg(lp):
        ev = P.eval(D * lp, gamma)
        return -ev.dual, -(D * ev.grad)

    r = scipy_opt.minimize(neg, np.zeros(inst.J), jac=True, method="L-BFGS-B",
                           bounds=[(0, None)] * inst.J,
                           options=dict(maxiter=20000, maxfun=40000, ftol=1e-15, gtol=1e-12))
    gstar = -r.fun
    kw = dict(max_iters=20000, tol_gap=1e-9, tol_infeas=1e-9)
    on = P.solve(restart_on_decrease=True, **kw)
    off = P.solve(restart_on_decrease=False, **kw)
    assert on["converged"] and off["converged"]
    assert on["restarts"] > 0 and off["restarts"] == 0
    for res in (on, off):
        assert abs(P.eval(res["mu"], gamma).dual - gstar) <= 1e-11 * abs(gstar)
    assert on["iters"] < off["iters"]


def test_lemma2_along_trajectory():
    """||(A x(mu) - b)_+||_2 <= sqrt(2 L (g* - g(mu))), L = ||A||^2 / gamma (Appendix A)."""
    inst = _tiny(I=150, J=8, seed=41)
    P = oracle.Problem(inst)
    gamma = 0.05
    L = P.norm2_sq() / gamma
    ref = P.solve(gamma0=gamma, gamma_final=gamma, halve_every=0, max_step=10 * gamma,
                  max_iters=4000, stop_on_tol=False)
    gstar = P.eval(ref["mu"], gamma).dual
    mu = np.zeros(inst.J)
    for k in range(300):
        ev = P.eval(mu, gamma)
        assert ev.infeas <= np.sqrt(2 * L * max(gstar - ev.dual, 0.0)) + 1e-9
        mu = np.maximum(0.0, mu + ev.grad / L)


def test_gamma_schedule_matches_section7_example():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "gamma_schedule_section7.txt"))
            if ln.strip() and not ln.startswith("#")]
    params = {r[0]: float(r[1]) for r in rows if not r[0].isdigit()}
    pts = [(int(r[0]), float(r[1])) for r in rows if r[0].isdigit()]
    inst = _tiny(I=20, J=4, seed=1)
    P = oracle.Problem(inst)
    res = P.solve(gamma0=params["gamma0"], gamma_final=params["gamma_final"],
                  halve_every=int(params["halve_every"]), max_iters=160, stop_on_tol=False,
                  want_trace=True)
    gam = res["trace"][:, 0]
    for k, g in pts:
        assert gam[k] == pytest.approx(g, rel=1e-15)


# --------------------------------------------------------------------------
# Generator sanity (the shared input module)
# --------------------------------------------------------------------------
def test_generator_properties():
    inst = synth.config("c2", scale=0.01)
    deg = np.diff(inst.off)
    assert deg.min() >= 1 and deg.max() <= 500
    assert abs(deg.mean() - 50) < 1.0
    for i in range(0, inst.I, 997):
        d = inst.dst[inst.off[i]:inst.off[i + 1]]
        assert len(np.unique(d)) == len(d)
    assert np.all((inst.dst >= 0) & (inst.dst < inst.J))
    assert np.all((inst.a >= 0.5) & (inst.a <= 1.5))
    assert np.all(inst.c < 0)
    again = synth.config("c2", scale=0.01)
    assert np.array_equal(inst.dst, again.dst) and np.array_equal(inst.c, again.c)
    bsum = np.bincount(inst.dst, weights=inst.a.astype(float), minlength=inst.J)
    assert np.allclose(inst.b, (0.2 * bsum).astype(np.float32), rtol=1e-6)


# --------------------------------------------------------------------------
# Unit-box projection (Section 6's clamp map): C = [0, 1]^E
# --------------------------------------------------------------------------
@pytest.mark.parametrize("weighted", [False, True])
def test_box_minimiser_by_bounded_search(weighted):
    """Each x_e of the box problem minimises x^2 / (2 alpha_e) + (c_e + a_e mu_j) x
    over [0, 1]: checked edge by edge with scipy's bounded scalar search."""
    scalar = pytest.importorskip("scipy.optimize").minimize_scalar
    inst = _tiny(I=25, J=6, seed=8)
    P = oracle.Problem(inst, weighted=weighted, box=True)
    mu = RNG.uniform(0.0, 1.5, inst.J)
    for gamma in (2.0, 0.3, 0.01):
        x = P.eval(mu, gamma, want_x=True).x
        for e in range(inst.E):
            a = float(inst.a[e])
            w = (a * a if a != 0 else 1.0) if weighted else 1.0
            lin = float(inst.c[e]) + a * mu[inst.dst[e]]
            f = lambda t: t * t * gamma * w / 2 + lin * t  # noqa: E731
            s = scalar(f, bounds=(0.0, 1.0), method="bounded", options=dict(xatol=1e-12))
            xb = min((0.0, 1.0, s.x), key=f)  # the ends are candidates too
            assert abs(x[e] - xb) <= 1e-6, (gamma, e, x[e], xb)


@pytest.mark.parametrize("weighted", [False, True])
def test_box_gradient_is_central_difference(weighted):
    inst = _tiny(seed=9)
    P = oracle.Problem(inst, weighted=weighted, box=True)
    for gamma in (0.5, 0.02):
        mu = RNG.uniform(0.0, 1.5, inst.J)
        ev = P.eval(mu, gamma)
        for j in range(inst.J):
            h = 1e-6 * max(1.0, abs(mu[j]))
            e = np.zeros(inst.J)
            e[j] = h
            fd = (P.eval(mu + e, gamma).dual - P.eval(mu - e, gamma).dual) / (2 * h)
            assert abs(fd - ev.grad[j]) <= 1e-6 * (abs(ev.ax[j]) + abs(inst.b[j]) + 1.0)


def test_box_relates_to_the_simplex():
    """The simplex {x >= 0, sum x <= 1} lies inside the unit box, so the box
    minimum is never above the simplex one: g_box(mu) <= g_simplex(mu); with one
    edge per source the two sets coincide and so do the evaluations."""
    inst = _tiny(I=60, J=8, seed=10)
    Pb, Ps = oracle.Problem(inst, box=True), oracle.Problem(inst)
    for gamma in (1.0, 0.05, 1e-3):
        for _ in range(3):
            mu = RNG.uniform(0.0, 2.0, inst.J)
            assert Pb.eval(mu, gamma).dual <= Ps.eval(mu, gamma).dual + 1e-12
    one = synth.from_degrees(np.ones(200, dtype=np.int64), 5, 3, synth.DST_UNIFORM)
    Pb, Ps = oracle.Problem(one, box=True), oracle.Problem(one)
    mu = RNG.uniform(0.0, 1.0, one.J)
    for gamma in (1.0, 0.01):
        eb, es = Pb.eval(mu, gamma, want_x=True), Ps.eval(mu, gamma, want_x=True)
        # (the simplex reaches x = 1 through its threshold, to within rounding)
        assert np.allclose(eb.x, es.x, rtol=0, atol=1e-12)
        assert abs(eb.dual - es.dual) <= 1e-12 * max(1.0, abs(es.dual))


# --------------------------------------------------------------------------
# Several constraint families (Section 3.2, Definition 1), rows k J + j
# --------------------------------------------------------------------------
def _families(inst, a_list, b_list):
    a = np.stack([np.asarray(x, np.float32) for x in a_list])
    b = np.concatenate([np.asarray(x, np.float32) for x in b_list])
    return synth.Instance(inst.off, inst.dst, inst.c, a, b, inst.J)


def test_families_split_one_family_in_two():
    """Halving every coefficient and budget into two identical families gives
    sum_k mu_k^T (A/2 x - b/2) = ((mu_1 + mu_2)/2)^T (A x - b): the two-family dual
    at (mu_1, mu_2) is the one-family dual at their mean, with the same x and
    half the gradient in each family."""
    inst = _tiny(I=80, J=9, seed=61)
    two = _families(inst, [inst.a / 2, inst.a / 2], [inst.b / 2, inst.b / 2])
    P1, P2 = oracle.Problem(inst), oracle.Problem(two)
    assert P2.m == 2 and P2.R == 2 * inst.J
    for gamma in (0.5, 0.01):
        mu = RNG.uniform(0.0, 2.0, 2 * inst.J)
        mid = (mu[:inst.J] + mu[inst.J:]) / 2
        e1, e2 = P1.eval(mid, gamma, want_x=True), P2.eval(mu, gamma, want_x=True)
        assert np.allclose(e2.x, e1.x, rtol=0, atol=1e-12)
        assert e2.dual == pytest.approx(e1.dual, rel=1e-12)
        assert np.allclose(e2.grad[:inst.J], e1.grad / 2, atol=1e-12)
        assert np.allclose(e2.grad[inst.J:], e1.grad / 2, atol=1e-12)


def test_families_zero_family_leaves_the_rest():
    """A family of zero coefficients changes no score: x and the first family's
    gradient are the one-family ones, its own rows have A x = 0 (gradient -b_2),
    and g gains -mu_2^T b_2."""
    inst = _tiny(I=60, J=7, seed=62)
    b2 = RNG.uniform(0.5, 2.0, inst.J)
    two = _families(inst, [inst.a, np.zeros(inst.E)], [inst.b, b2])
    P1, P2 = oracle.Problem(inst), oracle.Problem(two)
    mu = RNG.uniform(0.0, 1.5, 2 * inst.J)
    e1, e2 = P1.eval(mu[:inst.J], 0.05, want_x=True), P2.eval(mu, 0.05, want_x=True)
    assert np.allclose(e2.x, e1.x, atol=1e-14)
    assert np.allclose(e2.grad[:inst.J], e1.grad, atol=1e-12)
    assert np.allclose(e2.grad[inst.J:], -b2.astype(np.float32), atol=0)
    assert e2.dual == pytest.approx(e1.dual - mu[inst.J:] @ b2.astype(np.float32), rel=1e-12)
    D = P2.row_scale()
    assert np.all(D[inst.J:] == 1.0)  # zero rows keep D = 1


@pytest.mark.parametrize("weighted", [False, True])
def test_families_gradient_and_norm(weighted):
    """Danskin's gradient over all m J rows by central differences, and the
    block-diagonal spectral norm against numpy on the dense operator."""
    inst = synth.add_families(_tiny(I=50, J=6, seed=63), 3, seed=64)
    P = oracle.Problem(inst, weighted=weighted)
    R = 3 * inst.J
    for gamma in (0.4, 0.02):
        mu = RNG.uniform(0.0, 1.0, R)
        ev = P.eval(mu, gamma)
        for r in range(R):
            h = 1e-6 * max(1.0, abs(mu[r]))
            e = np.zeros(R)
            e[r] = h
            fd = (P.eval(mu + e, gamma).dual - P.eval(mu - e, gamma).dual) / (2 * h)
            assert abs(fd - ev.grad[r]) <= 1e-6 * (abs(ev.ax[r]) + abs(inst.b[r]) + 1.0)
    A = np.zeros((R, inst.E))
    for k in range(3):
        A[k * inst.J + inst.dst, np.arange(inst.E)] = inst.a[k]
    w = np.sum(inst.a.astype(np.float64) ** 2, axis=0) if weighted else np.ones(inst.E)
    Aw = A / np.sqrt(w)
    assert P.norm2_sq() == pytest.approx(np.linalg.norm(Aw, 2) ** 2, rel=1e-9)
    D = P.row_scale()
    assert np.allclose(np.sum((D[:, None] * Aw) ** 2, axis=1), 1.0)  # unit rows
    assert P.norm2_sq(D) == pytest.approx(np.linalg.norm(D[:, None] * Aw, 2) ** 2, rel=1e-9)


def test_families_tiny_lp_bounds():
    """Two families on tiny LPs: the solver's g*(gamma) lies between the LP
    optimum (HiGHS on the dense constraints) and that plus gamma I / 2."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    for seed in (1, 2, 3):
        inst = synth.add_families(_tiny_lp(seed), 2, seed=seed, rho=(0.3, 0.6))
        c, G1, h1 = _lp_parts(synth.Instance(inst.off, inst.dst, inst.c, inst.a[0],
                                             inst.b[:inst.J], inst.J))
        A2 = np.zeros((inst.J, inst.E))
        A2[inst.dst, np.arange(inst.E)] = inst.a[1]
        G = np.vstack([G1, A2])
        h = np.concatenate([h1, inst.b[inst.J:].astype(float)])
        lp = scipy_opt.linprog(c, A_ub=G, b_ub=h, bounds=(None, None), method="highs")
        assert lp.status == 0
        P = oracle.Problem(inst)
        for gamma in (0.1, 0.01):
            res = P.solve(gamma0=gamma, gamma_final=gamma, halve_every=0,
                          max_step=gamma / P.norm2_sq(), init_step=1e-3 * gamma,
                          max_iters=20000, stop_on_tol=False, row_normalize=False)
            g = P.eval(res["mu"], gamma).dual
            assert lp.fun - 1e-9 <= g + 2e-6
            assert g <= lp.fun + gamma * inst.I / 2 + 1e-9
