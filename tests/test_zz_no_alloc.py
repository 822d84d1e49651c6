"""The allocation-free evaluation agrees with the handle-based one.

dualip_dual_grad_noalloc serves callers that may not allocate device memory
(their device memory belongs to another allocator or a fixed arena, or their
request path cannot take cudaMalloc's implicit synchronisation).  It reads the
caller's device arrays directly and keeps its scratch in one fixed device
array.  Here it is called twice in a row through the C ABI, with different
dual points, and each result is compared with dualip_dual_grad on a handle
built from the same arrays, within twice the per-entry parity bound used
against the FP64 oracle (each path is within that bound of the oracle).
"""
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


@pytest.mark.parametrize("weighted", [False, True])
def test_noalloc_matches_handle_path_twice(dl, weighted):
    import torch

    inst = synth.greedy_budgets(synth.config("c2", scale=0.01))
    dev = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda()
           for k, v in dict(off=inst.off, dst=inst.dst, c=inst.c, a=inst.a, b=inst.b).items()}
    P = dl.Problem.from_instance(inst, primal_scaling=weighted)
    stream = dl._stream()
    rng = np.random.default_rng(42)
    for call, gamma in enumerate((1e-3, 0.05)):
        lam = torch.from_numpy(rng.uniform(0, 1.5, inst.J).astype(np.float32)).cuda()
        grad = torch.empty(inst.J, dtype=torch.float32, device="cuda")
        out = torch.empty(5, dtype=torch.float64, device="cuda")
        dl.dualip_dual_grad_noalloc(inst.I, inst.J, dev["off"].data_ptr(), dev["dst"].data_ptr(),
                                    dev["c"].data_ptr(), dev["a"].data_ptr(),
                                    dev["b"].data_ptr(), int(weighted), lam.data_ptr(), gamma,
                                    grad.data_ptr(), out.data_ptr(), stream)
        ref_grad, ref = P.dual_grad(lam, gamma)
        torch.cuda.synchronize()
        g = grad.cpu().numpy().astype(np.float64)
        gr = ref_grad.cpu().numpy().astype(np.float64)
        b = inst.b.astype(np.float64)
        tol = 2e-5 * (np.abs(gr + b) + np.abs(b)) + 2e-6
        assert np.all(np.abs(g - gr) <= tol), (call, np.max(np.abs(g - gr) / tol))
        o = out.cpu().numpy()
        for k, key in enumerate(("dual_obj", "primal_obj", "reg", "infeas_l2",
                                 "lambda_dot_grad")):
            scale = max(1.0, abs(ref[key]))
            bound = 2e-6 * scale if key != "infeas_l2" else 2e-5 * scale + 2e-6 * np.linalg.norm(b)
            assert abs(o[k] - ref[key]) <= bound, (call, key, o[k], ref[key])


def test_noalloc_rejects_too_many_destinations(dl):
    import torch

    z = torch.zeros(4, device="cuda")
    with pytest.raises(dl.DualipError) as ei:
        dl.dualip_dual_grad_noalloc(1, (1 << 20) + 1, z.data_ptr(), z.data_ptr(), z.data_ptr(),
                                    z.data_ptr(), z.data_ptr(), 0, z.data_ptr(), 0.1,
                                    z.data_ptr(), z.data_ptr(), dl._stream())
    assert ei.value.status == dl.DUALIP_EINVAL
