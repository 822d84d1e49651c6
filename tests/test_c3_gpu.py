"""The c3 shape: 25M sources x 1M destinations, Poisson(80) degrees in [1, 2000],
Zipf(1.1) destinations, about 2.0B edges (int64 offsets), with the edge values
(c, a) stored in BF16 or FP32.

(1) A seeded 1% source subsample of c3 (250,000 sources, all 1M destinations),
    BF16 storage:
    * against the FP64 oracle on the BF16-decoded values -- the accumulation
      error of the path, held to the FP32 parity bounds;
    * against the FP64 oracle on the FP32 values -- the quantisation error of
      BF16 storage, reported.  It has no small bound at small gamma (a score
      perturbation of 2^-9 |c| can move a near-tied source's mass), so only
      the structural bound |Delta (A x)_j| <= sum_{e->j} |a_e| is asserted.
(2) The full c3 instance, both storages, in the launch configuration the
    benchmark times (gamma = 1e-3, lambda ~ U(0,1) seed 7): gradient entries of
    sampled destinations (the oracle projects every source with an edge into
    them, so their (A x)_j is complete) and the primal blocks of sampled
    sources (dualip_get_primal against the oracle's projection).
"""
import numpy as np
import pytest

import oracle
import synth
from test_parity_gpu import GRAD_RTOL, check_eval, decoded

pytestmark = pytest.mark.gpu

GAMMA = 1e-3
LAM_SEED = 7


@pytest.fixture(scope="module")
def dl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04621_gb300 import build

    build.build()
    import paper_2603_04621_gb300 as d

    return d


@pytest.fixture(scope="module")
def c3():
    return synth.config("c3")


def lam_for(J):
    return np.random.default_rng(LAM_SEED).uniform(0.0, 1.0, J).astype(np.float32)


def test_c3_shape(c3):
    assert c3.I == 25_000_000 and c3.J == 1_000_000
    assert 1.9e9 < c3.E < 2.1e9 and c3.off.dtype == np.int64
    deg = np.diff(c3.off)
    assert deg.min() >= 1 and deg.max() <= 2000


@pytest.mark.parametrize("gamma", [0.1, GAMMA])
def test_c3_subsample_bf16(dl, c3, gamma):
    import torch

    idx = np.sort(np.random.default_rng(1003).choice(c3.I, c3.I // 100, replace=False))
    sub = c3.subset_sources(idx)
    lam = lam_for(c3.J)
    # (i) accumulation error: the oracle on the values the kernel reads
    P, _, grad, ev = check_eval(dl, sub, lam, gamma, storage="bf16")
    # (ii) quantisation error: the oracle on the FP32 values
    eo = oracle.Problem(sub).eval(lam.astype(np.float64), gamma)
    scale = np.abs(eo.ax) + np.abs(sub.b.astype(np.float64))
    err = np.abs(grad - eo.grad)
    bound = np.bincount(sub.dst, weights=np.abs(sub.a).astype(np.float64), minlength=sub.J)
    assert np.all(err <= bound * (1 + 2**-7) + 1e-6)
    rel = err / np.maximum(scale, 1e-30)
    print(f"\nc3 1% subsample, gamma={gamma}: BF16 vs FP32 data: grad rel err "
          f"median {np.median(rel):.3g}, p99 {np.quantile(rel, 0.99):.3g}, max {rel.max():.3g}; "
          f"dual obj rel err {abs(ev['dual_obj'] - eo.dual) / abs(eo.dual):.3g}")
    P.close()
    del torch


def sampled_destinations(inst, rng, n=40):
    """Destinations whose incoming sources the oracle can project one by one:
    random ids with in-degree <= 200k, plus the id at each of a few in-degree
    quantiles below that."""
    indeg = np.bincount(inst.dst, minlength=inst.J)
    ok = np.nonzero((indeg > 0) & (indeg <= 200_000))[0]
    pick = set(rng.choice(ok, n, replace=False).tolist())
    order = ok[np.argsort(indeg[ok])]
    for q in (0.0, 0.5, 0.9, 0.999, 1.0):
        pick.add(int(order[min(len(order) - 1, int(q * len(order)))]))
    return np.array(sorted(pick), dtype=np.int64)


@pytest.mark.parametrize("storage", ["bf16", "f32"])
def test_c3_full_size_sampled(dl, c3, storage):
    import torch

    rng = np.random.default_rng(31 if storage == "bf16" else 32)
    lam = lam_for(c3.J)
    P = dl.Problem.from_instance(c3, storage=storage)
    grad, ev = P.dual_grad(torch.from_numpy(lam).cuda(), GAMMA)
    grad = grad.cpu().numpy().astype(np.float64)

    # gradient entries of sampled destinations: every source with an edge into
    # them goes to the oracle
    js = sampled_destinations(c3, rng)
    mark = np.zeros(c3.J, dtype=bool)
    mark[js] = True
    hit_edges = np.nonzero(mark[c3.dst])[0]
    srcs = np.unique(np.searchsorted(c3.off, hit_edges, side="right") - 1)
    sub = c3.subset_sources(srcs)
    sub = decoded(sub) if storage == "bf16" else sub
    eo = oracle.Problem(sub).eval(lam.astype(np.float64), GAMMA)
    tol = GRAD_RTOL * (np.abs(eo.ax[js]) + np.abs(c3.b[js].astype(np.float64))) + 1e-6
    err = np.abs(grad[js] - eo.grad[js])
    assert np.all(err <= tol), (storage, js[err > tol][:5], (err / tol).max())

    # primal blocks of sampled sources
    x = P.primal(torch.from_numpy(lam).cuda(), GAMMA)
    si = np.sort(rng.choice(c3.I, 2000, replace=False))
    sub2 = c3.subset_sources(si)
    deg = np.diff(sub2.off)
    sel = np.repeat(c3.off[si] - sub2.off[:-1], deg) + np.arange(sub2.E, dtype=np.int64)
    xg = x[torch.from_numpy(sel).cuda()].cpu().numpy().astype(np.float64)
    sub2 = decoded(sub2) if storage == "bf16" else sub2
    xo = oracle.Problem(sub2).eval(lam.astype(np.float64), GAMMA, want_x=True).x
    assert np.all(xg >= 0)
    assert np.abs(xg - xo).max() <= 2e-5, np.abs(xg - xo).max()
    sums = np.add.reduceat(xg, sub2.off[:-1])  # every degree is >= 1
    assert sums.max() <= 1 + 1e-5

    # scalars at full size: the identity g = c^T x + ridge + lambda^T (A x - b)
    assert abs(ev["dual_obj"] - (ev["primal_obj"] + ev["reg"] + ev["lambda_dot_grad"])) <= \
        1e-12 * max(1.0, abs(ev["dual_obj"]))
    assert ev["reg"] >= 0 and ev["infeas_l2"] >= 0
    del x
    P.close()
