"""Host logic of the benchmark that needs no GPU: the DRAM traffic it reports
beside the roofline comes from a committed ncu capture.  It is scaled to a
launch (the per-destination bytes fixed, the rest by the edges processed),
and it is withheld when the capture no longer describes the kernel, the
configuration or the tile shape."""
import pytest

import bench


def test_traffic_scaling_keeps_the_destination_bytes_fixed():
    cap = bench.PASS_TRAFFIC[("c2", "f32")]
    if bench.kernel_code_hash() != bench.PASS_CODE_SHA256:
        pytest.skip("the pass kernel changed since the capture: no traffic is reported")
    # the captured case itself scales to its own bytes
    assert bench.pass_traffic(cap["edges"], cap["J"], "c2", "f32") == pytest.approx(cap["bytes"])
    # twice the edges with the same destinations: the per-destination part stays
    two = bench.pass_traffic(2 * cap["edges"], cap["J"], "c2", "f32")
    assert two == pytest.approx(2 * cap["bytes"] - 12 * cap["J"])
    # the c2 launch: within 3 % of the algorithmic bytes (no re-reads)
    E, I, J = 49_991_549, 1_000_000, 10_000
    alg = 12 * E + 4 * (I + 1) + 12 * J
    assert 0.97 < bench.pass_traffic(E, J, "c2", "f32") / alg < 1.03


def test_traffic_is_withheld_when_the_capture_does_not_apply(monkeypatch):
    # no capture for this configuration
    assert bench.pass_traffic(10**6, 10**4, "c3", "f32") is None
    # the batched capture holds for the tile shape it was taken at only
    assert bench.pass_traffic(10**9, 10**6, "c4", "f32", [2048, 128]) is None
    if bench.kernel_code_hash() == bench.PASS_CODE_SHA256:
        assert bench.pass_traffic(10**9, 10**6, "c4", "f32", [3200, 128]) > 0
    # a changed kernel
    monkeypatch.setattr(bench, "kernel_code_hash", lambda: "0" * 64)
    assert bench.pass_traffic(10**8, 10**4, "c2", "f32") is None


def test_kernel_hash_ignores_comments(tmp_path, monkeypatch):
    src = tmp_path / "paper_2603_04621_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "pass.cu").write_text("int f() { return 1; }  // one\n\n// note\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h1 = bench.kernel_code_hash()
    (src / "pass.cu").write_text("// header\nint f() { return 1; }  // two\n")
    assert bench.kernel_code_hash() == h1
    (src / "pass.cu").write_text("int f() { return 2; }\n")
    assert bench.kernel_code_hash() != h1


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` times the oracle on the host cores and prints
    one JSON line with the main arm's metric, unit and direction."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--scale", "0.01"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference"
    assert out["metric"] == bench.METRIC and out["unit"] == bench.UNIT
    assert out["higher_is_better"] is True and out["vs_baseline"] is None
    assert out["n_gpus"] == 1 and out["steps"] == 1 and out["warmup"] == 3
    assert out["value"] > 0 and out["ms_per_step"] > 0
    assert out["data"] == "synthetic" and "workload" in out["config"]
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == out["value"]
    assert cb["unit"] == out["unit"] and cb["sample"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
