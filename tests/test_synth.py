"""The seeded input generators (shared by both sides; no arithmetic of the
method): they follow the stated laws, are reproducible and independent of the
thread count, and the sub-instance helper picks exactly the chosen sources."""
import numpy as np
import pytest

import synth


def test_independent_of_thread_count():
    a = synth.config("c2", scale=0.005)
    lib = synth._load()
    old = lib.synth_set_threads(1)
    try:
        b = synth.config("c2", scale=0.005)
    finally:
        lib.synth_set_threads(max(old, 1))
    for x, y in ((a.off, b.off), (a.dst, b.dst), (a.c, b.c), (a.a, b.a), (a.b, b.b)):
        assert np.array_equal(x, y)


def test_c2_degree_law_is_poisson_50():
    inst = synth.config("c2", scale=0.05)
    deg = np.diff(inst.off).astype(np.float64)
    assert abs(deg.mean() - 50.0) < 0.3          # Poisson(50): mean 50
    assert abs(deg.var() / 50.0 - 1.0) < 0.05    # and variance 50 (clipping is negligible)
    assert deg.min() >= 1 and deg.max() <= 500


def test_c2_zipf_hot_destination():
    inst = synth.config("c2", scale=0.01)
    counts = np.bincount(inst.dst, minlength=inst.J)
    # p1 = 1 / H_1.1(10k) ~ 0.151 per draw: with 50 distinct draws nearly every
    # source reaches the top destination once
    assert counts.max() >= 0.99 * inst.I
    assert counts.max() <= inst.I  # distinct destinations per source
    # ids carry no hotness order (ranks go through a seeded permutation)
    assert np.argmax(counts) != 0


def test_c1_recipe():
    inst = synth.config("c1")
    assert inst.I == 1000 and inst.J == 50 and inst.E == 10_000
    assert np.all(np.diff(inst.off) == 10)
    assert np.all((inst.c <= 0) & (inst.c >= -1))
    cnt = np.bincount(inst.dst, minlength=50)
    assert cnt.min() > 120 and cnt.max() < 280  # uniform: 200 expected per destination
    bsum = np.bincount(inst.dst, weights=inst.a.astype(np.float64), minlength=50)
    assert np.allclose(inst.b, (0.3 * bsum).astype(np.float32), rtol=1e-6)


def test_greedy_budgets_follow_the_rule():
    inst = synth.config("c2", scale=0.002)
    g = synth.greedy_budgets(inst)
    # greedy load: every source puts its unit on its largest-a edge
    load = np.zeros(inst.J)
    for i in range(inst.I):
        s, e = inst.off[i], inst.off[i + 1]
        k = s + int(np.argmax(inst.a[s:e]))
        load[inst.dst[k]] += inst.a[k]
    rho = g.b.astype(np.float64) / (load + 0.01)
    assert np.all(rho >= 0.5 - 1e-5) and np.all(rho <= 1.0 + 1e-5)
    assert np.array_equal(g.dst, inst.dst)  # the same graph and values


def test_batch_and_trace_shapes():
    shapes = synth.batch_shapes(256)
    I = np.array([s[0] for s in shapes])
    J = np.array([s[1] for s in shapes])
    assert len(shapes) == 256 and I.min() >= 1_000 and I.max() <= 2_000_000
    assert J.min() >= 10 and J.max() <= 50_000
    assert len({s[2] for s in shapes}) == 256  # distinct per-instance seeds
    tr = synth.request_trace(400)
    t = np.array([r["t"] for r in tr])
    assert np.all(np.diff(t) >= 0) and t[0] == 0.0
    assert 400 / t[-1] == pytest.approx(20.0, rel=0.15)  # Poisson arrivals at 20/s
    assert 150 < sum(r["storage"] == "bf16" for r in tr) < 250


def test_subset_sources_picks_exactly_those_sources():
    inst = synth.config("c2", scale=0.002)
    idx = np.array([0, 3, 4, 100, inst.I - 1])
    sub = inst.subset_sources(idx)
    ref = [(inst.dst[inst.off[i]:inst.off[i + 1]], inst.c[inst.off[i]:inst.off[i + 1]])
           for i in idx]
    assert sub.I == len(idx) and sub.J == inst.J
    for k, (d, c) in enumerate(ref):
        assert np.array_equal(sub.dst[sub.off[k]:sub.off[k + 1]], d)
        assert np.array_equal(sub.c[sub.off[k]:sub.off[k + 1]], c)
    empty = inst.subset_sources(np.array([], dtype=np.int64))
    assert empty.I == 0 and empty.E == 0


def test_batched_and_request_degree_laws():
    # c4 instances: degrees UniformInt[5,100] clipped to J
    inst = synth.batch_instance(40_000, 5_000, 123)
    deg = np.diff(inst.off)
    assert deg.min() >= 5 and deg.max() <= 100
    assert abs(deg.mean() - 52.5) < 0.5
    counts = np.bincount(deg, minlength=101)[5:101]
    assert counts.min() > 0.8 * counts.mean()  # flat over 5..100
    small = synth.batch_instance(2_000, 12, 124)  # J = 12 clips most degrees
    d = np.diff(small.off)
    assert d.max() <= 12 and np.mean(d == 12) > 0.9
    # c5 requests: degrees Poisson(40) clipped to [1, J]
    req = dict(t=0.0, I=30_000, J=2_000, seed=7_000_001, storage="f32")
    deg = np.diff(synth.request_instance(req).off).astype(np.float64)
    assert abs(deg.mean() - 40.0) < 0.3 and abs(deg.var() / 40.0 - 1.0) < 0.06
    assert deg.min() >= 1 and deg.max() <= 2_000
    # the degree spread of the two laws: c4's is about 0.53, c5's about 0.16
    assert 0.5 < np.std(np.diff(inst.off)) / np.mean(np.diff(inst.off)) < 0.56
    assert 0.14 < deg.std() / deg.mean() < 0.18


def test_appendix_b_generator_laws():
    """The paper's Appendix B construction: each resource j draws K_j distinct
    requests; values are min(v_j u_i eps_ij, c_max) with c = -value; a = s_j value
    (one scale per resource); budgets follow the greedy-load rule; the draw does
    not depend on the thread count."""
    I, J, nu = 50_000, 400, 10.0
    x = synth.appb(I, J, nu)
    assert x.I == I and x.J == J and x.off[0] == 0 and x.off[-1] == x.E
    assert abs(x.E / I - nu) < 0.5  # K_j ~ Poisson(p_j I nu): E ~ I nu
    # distinct resources per request, in increasing id
    for i in range(0, I, 499):
        row = x.dst[x.off[i]:x.off[i + 1]]
        assert np.all(np.diff(row) > 0)
    val = -x.c.astype(np.float64)
    assert np.all(val > 0) and np.all(val <= synth.APPB_DEFAULTS["c_max"] * (1 + 1e-6))
    # a / value is the resource's own scale s_j: one value per resource
    ratio = x.a.astype(np.float64) / val
    for j in range(0, J, 37):
        rj = ratio[x.dst == j]
        if rj.size > 1:
            assert np.allclose(rj, rj[0], rtol=1e-6)
    # budgets: b_j = rho_j (l_j + eps) with rho_j in [0.5, 1]
    load = np.zeros(J)
    for i in range(I):
        s, e = x.off[i], x.off[i + 1]
        if e > s:
            k = s + int(np.argmax(x.a[s:e]))
            load[x.dst[k]] += x.a[k]
    rho = x.b.astype(np.float64) / (load + synth.APPB_DEFAULTS["eps"])
    assert np.all(rho >= 0.5 - 1e-6) and np.all(rho <= 1.0 + 1e-6)
    # row norms spread over orders of magnitude (the regime of Section 5.1)
    rown = np.sqrt(np.bincount(x.dst, weights=x.a.astype(np.float64) ** 2, minlength=J))
    assert np.percentile(rown, 99) / np.percentile(rown, 1) > 30
    # independent of the thread count
    import os

    lib = synth._load()
    lib.synth_set_threads(1)
    try:
        y = synth.appb(I, J, nu)
    finally:
        lib.synth_set_threads(os.cpu_count() or 1)
    for f in ("off", "dst", "c", "a", "b"):
        assert np.array_equal(getattr(x, f), getattr(y, f)), f
