"""Host-side helpers of bench.py (no GPU): roofline arithmetic, the peaks
file, and the rule that a committed ncu traffic figure is used only while the
kernel's source is unchanged."""
import hashlib
import importlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture
def bench():
    sys.path.insert(0, ROOT)
    try:
        yield importlib.import_module("bench")
    finally:
        sys.path.remove(ROOT)


def test_roofline_arithmetic(bench):
    pk = bench.with_simt_peak(dict(hbm=6000.0, sm_mhz=2070.0, src="measured"), 152)
    # 10 launches, 2 ms in all, 1e9 bytes of algorithmic traffic per launch: 5e12 B/s
    r = bench.roofline_of("apply", 2.0, 10, 1e10, 8.0, pk)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(5000.0) and r["frac"] == pytest.approx(5000.0 / 6000.0)
    assert r["share"] == pytest.approx(0.25) and r["avg_launch_us"] == pytest.approx(200.0)
    # 4 launches, 1 ms in all, 2e9 flops per launch: 8e12 flop/s against the FP32 SIMT peak
    g = bench.roofline_of("gj_panel_f32", 1.0, 4, 8e9, 4.0, pk)
    assert g["bound"] == "alu" and g["achieved"] == pytest.approx(8.0)
    assert g["peak"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert g["traffic"] == bench.profiled_traffic("gj_panel_f32")   # the committed capture, if current
    assert "152 SMs" in g["peak_source"]
    # the SM count and clock come from the device and the peaks file, not a constant
    pk2 = bench.with_simt_peak(dict(hbm=6000.0, sm_mhz=1500.0, src="measured"), 100)
    assert bench.roofline_of("gj_panel_f32", 1.0, 4, 8e9, 4.0, pk2)["peak"] == pytest.approx(
        100 * 128 * 2 * 1.5e9 / 1e12)
    d = bench.roofline_of("gemm_f64", 1.0, 1, 1e9, 1.0, pk)
    assert d["peak"] == 1.25 and d["achieved"] == pytest.approx(1.0)
    # tensor-core classes: the K = 256 block updates are bounded by their C stream (flops / 64 bytes),
    # the other TMA launches by the TF32 rate (measured BF16 x 1.1 / 2.25)
    pk3 = dict(pk, bf16=2000.0)
    t = bench.roofline_of("gemm_tma_block", 1.0, 1, 6.4e10, 1.0, pk3)
    assert t["bound"] == "hbm" and t["achieved"] == pytest.approx(1000.0) and t["tflops"] == pytest.approx(64.0)
    assert t["tf32_peak_tflops"] == pytest.approx(2000.0 * 1.1 / 2.25)
    u = bench.roofline_of("gemm_tma_sample", 1.0, 1, 1e10, 1.0, pk3)
    assert u["bound"] == "tensor" and u["achieved"] == pytest.approx(10.0) and u["peak"] == pytest.approx(977.78, rel=1e-4)


def test_peaks_file_and_fallback(bench, tmp_path, monkeypatch):
    pk = bench.peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert pk["src"] == "measured" and pk["hbm"] > 1000
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    fb = bench.peaks()
    assert fb["src"] == "fallback" and fb["hbm"] == 6800.0 and fb["bf16"] == 1900.0 and fb["sm_mhz"] == 2070.0


def test_cpu_cores_is_the_process_affinity(bench):
    assert bench.cpu_cores() == len(os.sched_getaffinity(0))


def test_profiled_traffic_only_for_the_profiled_source(bench, tmp_path, monkeypatch):
    src = tmp_path / "paper_1508_07798_gb300" / "csrc" / "gemm.cu"
    src.parent.mkdir(parents=True)
    src.write_text("// kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    prof = tmp_path / "profiles" / "k_gemm_f32_dram_helmholtz64_p2.md"
    prof.parent.mkdir()
    prof.write_text(f"traffic_bytes_per_launch: 1234\nkernel_source_sha256_prefix: {sha[:16]}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("gemm_f32") == 1234
    assert bench.profiled_traffic("apply") is None
    src.write_text("// kernel source, changed\n")
    assert bench.profiled_traffic("gemm_f32") is None


def test_reference_line_has_the_workload_config(bench, monkeypatch, capsys):
    """The reference arm (the oracle) prints the same config dictionary as the
    GPU arm builds (headline_config), with its own cpu_baseline and e2e; the
    oracle solve itself is replaced by a stub here."""
    import json
    monkeypatch.setattr(bench, "cpu_baseline_run", lambda seed=0: (1234.0, {"iters": 19}))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"])
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    assert line["impl"] == "reference" and line["value"] == pytest.approx(1234.0)
    assert line["config"] == bench.headline_config(bench.parse(), 1)
    assert line["config"]["dofs"] == 36864 and line["config"]["workload"] == bench.WORKLOAD
    assert line["e2e"] == dict(value=line["value"], unit="ms", h2d_bytes_per_step=0, d2h_bytes_per_step=0)
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
