"""The allocation-free evaluation, checked against the FP64 oracle and the
handle-based path.

dualip_dual_grad_noalloc serves callers that may not allocate device memory
(their device memory belongs to another allocator or a fixed arena, or their
request path cannot take cudaMalloc's implicit synchronisation).  It reads the
caller's device arrays directly and keeps its scratch in one fixed device
array.  Here it is called several times in a row through the C ABI, with
different dual points, and each result is compared

* with the FP64 oracle at the parity bounds of the main path (per entry
  1e-5 (|A x| + |b|) + 1e-6, scalars 1e-6 relative), and
* with dualip_dual_grad on a handle built from the same arrays, within twice
  that bound (each path is within the bound of the oracle).

The cases cover no sources at all, sources with no edges, a gamma large enough
that sources leave their sum constraint slack, and an edge whose destination
is out of range (skipped, every output NaN, nothing faults).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-5
OBJ_RTOL = 1e-6
KEYS = ("dual_obj", "primal_obj", "reg", "infeas_l2", "lambda_dot_grad")


@pytest.fixture(scope="module")
def dl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_04621_gb300 import build

    build.build()
    import paper_2603_04621_gb300 as d

    return d


def to_dev(inst):
    import torch

    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda()
            for k, v in dict(off=inst.off, dst=inst.dst, c=inst.c, a=inst.a, b=inst.b).items()}


def noalloc(dl, inst, dev, lam, gamma, weighted):
    import torch

    grad = torch.empty(inst.J, dtype=torch.float32, device="cuda")
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    dl.dualip_dual_grad_noalloc(inst.I, inst.J, dev["off"].data_ptr(), dev["dst"].data_ptr(),
                                dev["c"].data_ptr(), dev["a"].data_ptr(), dev["b"].data_ptr(),
                                int(weighted), lam.data_ptr(), gamma, grad.data_ptr(),
                                out.data_ptr(), dl._stream())
    torch.cuda.synchronize()
    return grad.cpu().numpy().astype(np.float64), out.cpu().numpy()


def check_oracle(inst, g, o, eo, lam, factor=1.0):
    b = inst.b.astype(np.float64)
    tol = factor * (GRAD_RTOL * (np.abs(eo.ax) + np.abs(b)) + 1e-6)
    err = np.abs(g - eo.grad)
    assert np.all(err <= tol), f"worst {(err / tol).max():.3g}x the gradient bound"
    for k, ref in zip(KEYS, (eo.dual, eo.primal_lin, eo.reg, eo.infeas, eo.mu_dot_grad)):
        if k == "infeas_l2":
            bound = 1e-5 * max(1.0, ref) + 1e-6 * np.linalg.norm(b)
        elif k == "lambda_dot_grad":  # a dot product that may cancel: relative to its terms
            terms = np.abs(np.asarray(lam, np.float64)) * (np.abs(eo.ax) + np.abs(b))
            bound = OBJ_RTOL * max(1.0, float(terms.sum()))
        else:
            bound = OBJ_RTOL * max(1.0, abs(ref))
        assert abs(o[KEYS.index(k)] - ref) <= factor * bound, (k, o[KEYS.index(k)], ref)


@pytest.mark.parametrize("weighted", [False, True])
def test_noalloc_matches_oracle_and_handle_path(dl, weighted):
    import torch

    inst = synth.greedy_budgets(synth.config("c2", scale=0.01))
    dev = to_dev(inst)
    P = dl.Problem.from_instance(inst, primal_scaling=weighted)
    Po = oracle.Problem(inst, weighted=weighted)
    rng = np.random.default_rng(42)
    # gamma = 100 leaves most sources' sum constraints slack
    for call, gamma in enumerate((1e-3, 0.05, 100.0)):
        lam_h = rng.uniform(0, 1.5, inst.J).astype(np.float32)
        lam = torch.from_numpy(lam_h).cuda()
        g, o = noalloc(dl, inst, dev, lam, gamma, weighted)
        eo = Po.eval(lam_h.astype(np.float64), gamma)
        check_oracle(inst, g, o, eo, lam_h)
        ref_grad, ref = P.dual_grad(lam, gamma)
        torch.cuda.synchronize()
        gr = ref_grad.cpu().numpy().astype(np.float64)
        b = inst.b.astype(np.float64)
        tol = 2 * (GRAD_RTOL * (np.abs(gr + b) + np.abs(b)) + 1e-6)
        assert np.all(np.abs(g - gr) <= tol), (call, np.max(np.abs(g - gr) / tol))
        dot_scale = float(np.sum(np.abs(lam_h) * (np.abs(gr + b) + np.abs(b))))
        for k, key in enumerate(KEYS):
            scale = max(1.0, abs(ref[key]))
            bound = 2e-6 * scale
            if key == "infeas_l2":
                bound = 2e-5 * scale + 2e-6 * np.linalg.norm(b)
            elif key == "lambda_dot_grad":
                bound = 2e-6 * max(1.0, dot_scale)
            assert abs(o[k] - ref[key]) <= bound, (call, key, o[k], ref[key])
    if gamma == 100.0:
        # the slack branch was taken: some source has sum x < 1 with x > 0
        x = Po.eval(lam_h.astype(np.float64), gamma, want_x=True).x
        sums = np.add.reduceat(x, inst.off[:-1][np.diff(inst.off) > 0])
        assert np.any((sums > 0) & (sums < 1 - 1e-9))


def test_noalloc_widely_spread_weights(dl):
    """Primal scaling with coefficients over four orders of magnitude: the
    allocation-free threshold is formed in FP64 too."""
    import torch

    degs = np.array([3, 40, 300, 2_000, 12, 0, 90])
    inst = synth.greedy_budgets(synth.from_degrees(degs, 5_000, 31, synth.DST_UNIFORM,
                                                   a_lo=0.01, a_hi=100.0))
    dev = to_dev(inst)
    Po = oracle.Problem(inst, weighted=True)
    rng = np.random.default_rng(49)
    for gamma in (0.1, 1e-3):
        lam_h = rng.uniform(0, 1, inst.J).astype(np.float32)
        g, o = noalloc(dl, inst, dev, torch.from_numpy(lam_h).cuda(), gamma, True)
        check_oracle(inst, g, o, Po.eval(lam_h.astype(np.float64), gamma), lam_h)


def test_noalloc_no_sources_and_empty_sources(dl):
    import torch

    J = 300
    rng = np.random.default_rng(5)
    lam_h = rng.uniform(0, 1, J).astype(np.float32)
    lam = torch.from_numpy(lam_h).cuda()
    # I = 0: grad = -b exactly, g = -lambda^T b
    empty = synth.Instance(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32),
                           np.zeros(0, np.float32), rng.uniform(0.5, 2, J).astype(np.float32), J)
    g, o = noalloc(dl, empty, to_dev(empty), lam, 1e-3, False)
    assert np.array_equal(g, -empty.b.astype(np.float64))
    check_oracle(empty, g, o, oracle.Problem(empty).eval(lam_h.astype(np.float64), 1e-3), lam_h)
    # sources with no edges between ordinary ones
    deg = np.array([0, 5, 0, 0, 40, 1, 0, 300, 0])
    inst = synth.from_degrees(deg, J, 13, synth.DST_UNIFORM, b_frac=0.4)
    Po = oracle.Problem(inst)
    for gamma in (1e-3, 0.5):
        g, o = noalloc(dl, inst, to_dev(inst), lam, gamma, False)
        check_oracle(inst, g, o, Po.eval(lam_h.astype(np.float64), gamma), lam_h)


def test_noalloc_out_of_range_destination(dl):
    """One edge names destination J: the pass skips it (nothing is read or
    written out of range), the call returns OK, and every entry of the gradient
    and every scalar is NaN.  The next valid call is correct again."""
    import torch

    inst = synth.config("c2", scale=0.002)
    dev = to_dev(inst)
    dev["dst"][inst.E // 2] = inst.J
    lam_h = np.random.default_rng(8).uniform(0, 1, inst.J).astype(np.float32)
    lam = torch.from_numpy(lam_h).cuda()
    g, o = noalloc(dl, inst, dev, lam, 1e-3, False)
    assert np.all(np.isnan(g)) and np.all(np.isnan(o))
    dev["dst"][inst.E // 2] = int(inst.dst[inst.E // 2])
    g, o = noalloc(dl, inst, dev, lam, 1e-3, False)
    check_oracle(inst, g, o, oracle.Problem(inst).eval(lam_h.astype(np.float64), 1e-3), lam_h)


def test_noalloc_rejects_too_many_destinations(dl):
    import torch

    z = torch.zeros(4, device="cuda")
    with pytest.raises(dl.DualipError) as ei:
        dl.dualip_dual_grad_noalloc(1, (1 << 20) + 1, z.data_ptr(), z.data_ptr(), z.data_ptr(),
                                    z.data_ptr(), z.data_ptr(), 0, z.data_ptr(), 0.1,
                                    z.data_ptr(), z.data_ptr(), dl._stream())
    assert ei.value.status == dl.DUALIP_EINVAL
