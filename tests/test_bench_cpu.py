"""The measurement's arithmetic, on the CPU: the algorithmic counts behind `roofline`, the bound it
picks, the traffic records' source check, the throughput helpers, the host-link bound, and the
reference arm's JSON line (the FP64 oracle on the host cores, which needs no GPU).

The counts are restated here by hand for p = 2 (q = 3 Gauss points, bands of W = 5), so a change of
the bench's formula that moves a figure fails a test rather than the roofline silently.
"""
import json
import os

import pytest

import bench


def test_quadrature_and_step_counts_p2():
    c = bench.algorithmic_costs(2)
    # interpolation: x pass 2 fields x 3 points x 3 coefficients, y pass 3 fields x 9 points x 3
    interp = 2 * 3 * 3 + 3 * 9 * 3                     # 99
    fuel = 3 * 3 + 9 * 3                                # 36
    point = 6 * 9                                       # 54: the point source, 6 FMA per Gauss point
    rhs_r = 4 * 5 + 1                                   # 21: two Kronecker products with W = 5 bands
    fma = interp + fuel + (interp + fuel) + point + rhs_r
    assert fma == 345
    assert c["rhs_quadrature_1"] == {"bytes": 20, "flops": 690}
    line = 4 * 2 + 1                                    # p forward, p + 1 backward, 2p spike
    assert c["xsolve_1"]["flops"] == 2 * 2 * line       # two arrays
    assert c["ysolve_1"]["flops"] == 2 * 2 * (line + 1)  # with the increment base
    assert c["matvec_2"]["flops"] == 2 * rhs_r
    assert c["step_persistent"] == {"bytes": 56, "flops": 846}
    assert sum(c[k]["bytes"] for k in ("rhs_quadrature_1", "xsolve_1", "ysolve_1", "matvec_2", "xsolve_2",
                                       "ysolve_2")) == 92   # the per-pass split's bytes per DOF
    assert bench.min_step_bytes("pr") == 56


def test_roofline_picks_the_bound():
    costs = bench.algorithmic_costs(2)
    dofs = 1_000_000
    # the quadrature's intensity (690 flop / 20 B = 34.5) is above 80 TFLOP/s / 6758 GB/s = 11.9
    r = bench.roofline("rhs_quadrature_1", 0.5, dofs, costs, 4, 6758.0, "measured", 80.0, "probe")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(690 * dofs / 0.5e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 80.0)
    assert r["arithmetic_intensity"] == pytest.approx(34.5)
    # a line pass (36 flop / 16 B) is bandwidth-bound
    r = bench.roofline("xsolve_1", 0.01, dofs, costs, 4, 6758.0, "measured", 80.0, "probe")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(16 * dofs / 0.01e-3 / 1e9)
    # FP64 doubles the bytes
    r8 = bench.roofline("xsolve_1", 0.01, dofs, costs, 8, 6758.0, "measured", 80.0, "probe")
    assert r8["algorithmic_bytes_per_launch"] == 2 * r["algorithmic_bytes_per_launch"]


def test_traffic_record_follows_the_sources(tmp_path, monkeypatch):
    # a copy of one source file and a records file under a stand-in root
    src = os.path.join(bench.ROOT, "paper_2604_19370_gb300", "csrc", "wf_api.cu")
    os.makedirs(tmp_path / "paper_2604_19370_gb300" / "csrc")
    os.makedirs(tmp_path / "profiles")
    with open(src, "rb") as f, open(tmp_path / "paper_2604_19370_gb300" / "csrc" / "wf_api.cu", "wb") as g:
        g.write(f.read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = {"w": {"k": {"source_sha": {"wf_api.cu": bench._source_sha("wf_api.cu")}, "dram_bytes_per_launch": 123},
                 "stale": {"source_sha": {"wf_api.cu": "0" * 16}, "dram_bytes_per_launch": 456}}}
    with open(tmp_path / "profiles" / "traffic.json", "w") as f:
        json.dump(rec, f)
    assert bench._traffic_record("k", "w") == 123.0
    assert bench._traffic_record("stale", "w") is None      # the kernel changed since the capture
    assert bench._traffic_record("k", "other") is None
    # editing the source invalidates the record
    with open(tmp_path / "paper_2604_19370_gb300" / "csrc" / "wf_api.cu", "ab") as g:
        g.write(b"// edit\n")
    assert bench._traffic_record("k", "w") is None


def test_committed_traffic_records_cover_the_dominant_kernels():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    for w in ("c4_ensemble_256x256x256_p2_pr", "c2_1024x1024_p2_pr", "c3_4096x4096_p3_pr"):
        assert "rhs_quadrature_1" in rec[w]
        assert rec[w]["rhs_quadrature_1"]["dram_bytes_per_launch"] > 0


def test_throughput_helpers_single_rank():
    value, slowest = bench.whole_job_throughput(1000.0, 0.5, 1)
    assert slowest == 0.5 and value == pytest.approx(2000.0)
    parts = [list(bench.shard(257, r, 4)) for r in range(4)]
    assert sorted(i for p in parts for i in p) == list(range(257))
    assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    assert bench._percentile([1.0, 2.0, 3.0, 4.0], 0.5) == pytest.approx(2.5)
    assert bench._percentile([1.0, 2.0, 3.0, 4.0], 0.99) == pytest.approx(3.97)


def test_link_bound_takes_the_slowest_constraint():
    # 136 MB each way: 0.648 ms in at 210 GB/s, 0.708 ms out at 192 GB/s, 0.802 ms for both at
    # 339 GB/s combined; the bound is the largest
    r = bench.link_bound((210.0, 192.0, 339.0), 136_000_000, 136_000_000, 1.6)
    assert r["bound_ms_per_step"] == pytest.approx(272e6 / 339e9 * 1e3)
    assert r["frac"] == pytest.approx(r["bound_ms_per_step"] / 1.6)
    # a one-way step is bound by its own direction
    r = bench.link_bound((210.0, 192.0, 339.0), 136_000_000, 0, 1.0)
    assert r["bound_ms_per_step"] == pytest.approx(136e6 / 210e9 * 1e3)


def test_reference_arm_prints_the_contract_line():
    # the reference arm is the FP64 oracle on the host cores: it runs without a GPU
    import subprocess
    import sys

    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=bench.ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 3          # at least three warm-up steps, as run
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["config"]["workload"] == "c4_ensemble_256x256x256_p2_pr"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
