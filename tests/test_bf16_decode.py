"""The BF16 decode that the BF16 parity tests feed to the oracle (float32 ->
bfloat16 by round to nearest even -> float32) agrees bit for bit with an
independent conversion (PyTorch's CPU bfloat16 cast), on random values and on
the cases where rounding decides: exact ties in both directions, values just
off a tie, subnormals, signed zero and the largest finite values."""
import numpy as np
import pytest

from test_parity_gpu import bf16_round


def _torch_round(x):
    torch = pytest.importorskip("torch")
    return torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()


def test_random_values_match():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(100_000), -rng.lognormal(0, 1, 100_000),
                        rng.uniform(0.5, 1.5, 100_000)]).astype(np.float32)
    assert np.array_equal(bf16_round(x).view(np.uint32), _torch_round(x).view(np.uint32))


def test_rounding_edge_cases_match():
    base = np.array([0x3F800000, 0x3F810000, 0x40490000, 0x00010000, 0x80000000, 0x00000000,
                     0x7F7F0000, 0xFF7F0000], dtype=np.uint32)
    cases = []
    for b in base:
        for low in (0x0000, 0x7FFF, 0x8000, 0x8001, 0xFFFF, 0x0001):
            cases.append((int(b) & 0xFFFF0000) | low)
    x = np.array(cases, dtype=np.uint32).view(np.float32)
    x = x[np.isfinite(x) & np.isfinite(_torch_round(x))]  # a carry past the largest value overflows
    got, ref = bf16_round(x).view(np.uint32), _torch_round(x).view(np.uint32)
    assert np.array_equal(got, ref), [hex(v) for v in x.view(np.uint32)[got != ref]]
    # ties go to the even mantissa: 1 + 2^-8 -> 1, and 1 + 3 * 2^-8 -> 1 + 2^-6
    t = np.array([0x3F808000, 0x3F818000], dtype=np.uint32).view(np.float32)
    assert list(bf16_round(t).view(np.uint32)) == [0x3F800000, 0x3F820000]
