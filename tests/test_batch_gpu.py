"""The batched form: several matching LPs in one launch of the pass.

* Every problem's gradient equals its lone dualip_dual_grad bit for bit (A x is
  exact in fixed point and each problem keeps its own data), and its scalars
  agree to the order of their partial sums; each is also within the parity
  bounds of the FP64 oracle.
* The same holds for every tile shape, and after the autotuner.
* The batched ascent ends every problem as its lone solve does, and a
  problem's trajectory is the same alone (a batch of one) and among others,
  bit for bit at a fixed iteration count.
"""
import numpy as np
import pytest

import oracle
import synth
from test_parity_gpu import GRAD_RTOL, OBJ_RTOL, decoded

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


def small_batch(n=10, seed=4242, i_range=(100, 30_000), j_range=(10, 4_000), greedy=False):
    insts = [synth.batch_instance(I, J, s)
             for I, J, s in synth.batch_shapes(n, seed, i_range, j_range)]
    if greedy:
        insts = [synth.greedy_budgets(x) for x in insts]
    return insts


def lam_joint(insts, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.uniform(0, 2, x.J) for x in insts]).astype(np.float32)


@pytest.mark.parametrize("storage,weighted", [("f32", False), ("f32", True), ("bf16", False)])
def test_batch_matches_lone_and_oracle(dl, storage, weighted):
    import torch

    insts = small_batch()
    probs = [dl.Problem.from_instance(x, storage=storage, primal_scaling=weighted) for x in insts]
    B = dl.Batch(probs)
    lam = lam_joint(insts, 1)
    gammas = list(np.geomspace(1e-3, 0.2, len(insts)))
    lt = torch.from_numpy(lam).cuda()
    for shape in (None, (1024, 64), (512, 16), (3072, 256)):
        if shape:
            B.set_tile_shape(*shape)
        grad, evs = B.dual_grad(lt, gammas)
        g = grad.cpu().numpy()
        for k, (x, P) in enumerate(zip(insts, probs)):
            lk = lt[B.joff[k]:B.joff[k + 1]]
            g1, e1 = P.dual_grad(lk, gammas[k])
            gk = g[B.joff[k]:B.joff[k + 1]]
            assert np.array_equal(gk, g1.cpu().numpy()), (shape, k)
            # c^T x and the ridge term are exact fixed-point sums: equal bit for bit
            for key in ("primal_obj", "reg"):
                assert evs[k][key] == e1[key], (shape, k, key)
            for key in ("dual_obj", "infeas_l2", "lambda_dot_grad"):
                assert abs(evs[k][key] - e1[key]) <= 1e-9 * max(1.0, abs(e1[key])), (k, key)
            if shape is None:
                ref = decoded(x) if storage == "bf16" else x
                eo = oracle.Problem(ref, weighted=weighted).eval(
                    lam[B.joff[k]:B.joff[k + 1]].astype(np.float64), gammas[k])
                tol = GRAD_RTOL * (np.abs(eo.ax) + np.abs(x.b.astype(np.float64))) + 1e-6
                assert np.all(np.abs(gk - eo.grad) <= tol), k
                assert abs(evs[k]["dual_obj"] - eo.dual) <= OBJ_RTOL * max(1.0, abs(eo.dual))
    B.close()


@pytest.mark.parametrize("weighted", [False, True])
def test_batch_with_sources_larger_than_a_stage(dl, weighted):
    """A batch holding sources larger than a stage takes the pass instance with
    the block class.  Sources up to 16 stages are projected by the same code as
    alone (the gradient bit for bit); a larger one, which alone goes to the
    multi-block class, agrees with the oracle within the parity bounds."""
    import torch

    blockish = synth.greedy_budgets(synth.from_degrees(np.array([5_000, 40, 3, 20_000, 0, 12]),
                                                       30_000, 61, synth.DST_UNIFORM))
    hubbish = synth.greedy_budgets(synth.from_degrees(np.array([70_000, 9, 300, 4_000]),
                                                      80_000, 62, synth.DST_UNIFORM))
    insts = [blockish, hubbish]
    probs = [dl.Problem.from_instance(x, primal_scaling=weighted) for x in insts]
    B = dl.Batch(probs)
    lam = lam_joint(insts, 3)
    lt = torch.from_numpy(lam).cuda()
    for gammas in ([1e-3, 1e-3], [0.2, 0.05]):
        grad, evs = B.dual_grad(lt, gammas)
        g = grad.cpu().numpy()
        for k, (x, P) in enumerate(zip(insts, probs)):
            lk = lt[B.joff[k]:B.joff[k + 1]]
            gk = g[B.joff[k]:B.joff[k + 1]]
            g1, e1 = P.dual_grad(lk, gammas[k])
            if k == 0:
                assert np.array_equal(gk, g1.cpu().numpy())
            eo = oracle.Problem(x, weighted=weighted).eval(
                lam[B.joff[k]:B.joff[k + 1]].astype(np.float64), gammas[k])
            tol = GRAD_RTOL * (np.abs(eo.ax) + np.abs(x.b.astype(np.float64))) + 1e-6
            assert np.all(np.abs(gk - eo.grad) <= tol), k
            assert abs(evs[k]["dual_obj"] - eo.dual) <= OBJ_RTOL * max(1.0, abs(eo.dual)), k
    B.close()


def test_batch_autotune_keeps_results(dl):
    import torch

    insts = small_batch(n=6, seed=77)
    probs = [dl.Problem.from_instance(x) for x in insts]
    B = dl.Batch(probs)
    lt = torch.from_numpy(lam_joint(insts, 2)).cuda()
    gam = [1e-2] * len(insts)
    g0, e0 = B.dual_grad(lt, gam)
    r = B.autotune()
    info = B.info()
    assert r["n_candidates"] >= 1
    assert info["tile_edges"] == r["tile_edges"][r["chosen"]]
    assert info["tile_sources"] == r["tile_sources"][r["chosen"]]
    assert sum(r["degree_hist"]) == sum(x.I for x in insts)
    assert all(t > 0 for t in r["ms"])
    g1, e1 = B.dual_grad(lt, gam)
    assert torch.equal(g0, g1)
    B.close()


def test_batch_rejects_bad_input(dl):
    insts = small_batch(n=2, seed=5)
    p32 = dl.Problem.from_instance(insts[0])
    p16 = dl.Problem.from_instance(insts[1], storage="bf16")
    with pytest.raises(dl.DualipError):
        dl.Batch([p32, p16])
    with pytest.raises(dl.DualipError):
        dl.Batch([p32, p32])
    with pytest.raises(dl.DualipError):
        dl.dualip_batch_create([])
    B = dl.Batch([p32])
    import torch

    lt = torch.zeros(insts[0].J, device="cuda")
    with pytest.raises(dl.DualipError):
        B.dual_grad(lt, [0.0])
    with pytest.raises(dl.DualipError):
        B.set_tile_shape(4096, 16)
    B.close()


def test_batch_solve_converges_like_lone_solves(dl):
    """Each problem of the batch ends as its lone dualip_solve does: converged
    to the same 1e-4 gap (so to the same dual value within it), or out of
    iterations.  (Some of these random instances do not reach the tolerances
    within max_iters under the default steps; the FP64 oracle's ascent does
    not either.)"""
    import torch

    insts = small_batch(n=8, seed=99, greedy=True)
    probs = [dl.Problem.from_instance(x) for x in insts]
    kw = dict(max_iters=3000)
    lone = [P.solve(**kw)[1] for P in probs]
    assert sum(r["converged"] for r in lone) >= 5
    B = dl.Batch(probs)
    lam, res = B.solve(**kw)
    for k, (P, r1) in enumerate(zip(probs, lone)):
        if r1["converged"]:
            assert res[k]["converged"], (k, res[k])
            assert abs(res[k]["dual_obj"] - r1["dual_obj"]) <= 3e-4 * max(1.0, abs(r1["dual_obj"]))
        else:
            assert res[k]["iters"] == kw["max_iters"] or res[k]["converged"]
        # the returned lambda gives the reported scalars
        lk = lam[int(B.joff[k]):int(B.joff[k + 1])]
        _, ev = P.dual_grad(lk, res[k]["gamma"])
        assert abs(ev["dual_obj"] - res[k]["dual_obj"]) <= 1e-6 * max(1.0, abs(ev["dual_obj"]))
    B.close()
    del torch


def test_batch_trajectory_alone_equals_in_mix(dl):
    """A fixed number of ascent iterations: lambda of each problem is the same
    bit for bit in a batch of one and among the others."""
    insts = small_batch(n=6, seed=123, greedy=True)
    probs = [dl.Problem.from_instance(x) for x in insts]
    B = dl.Batch(probs)
    kw = dict(max_iters=60, stop_on_tol=0)
    lam_mix, _ = B.solve(**kw)
    B.close()
    for k in (0, 3, 5):
        Bk = dl.Batch([probs[k]])
        lam_k, _ = Bk.solve(**kw)
        Bk.close()
        import torch

        assert torch.equal(lam_k, lam_mix[int(B.joff[k]):int(B.joff[k + 1])]), k
