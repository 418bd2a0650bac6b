"""Host-side logic of bench.py on CPU: the clock record, the traffic scaling
rule, the roofline figures, the peak's source and the reference arm's JSON
line (no GPU)."""
import json
import types

import pytest

import bench

UUID = "GPU-1111aaaa-2222-3333-4444-555566667777"
OTHER = "GPU-9999aaaa-2222-3333-4444-555566667777"


class _FakeSmi:
    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def kill(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def _clocks(monkeypatch, rows, uuid=UUID):
    monkeypatch.setattr(bench.subprocess, "Popen", lambda *a, **k: _FakeSmi("\n".join(rows) + "\n"))
    return bench.Clocks(uuid)


def test_clock_record_median_max_and_reasons(monkeypatch):
    na, act = "Not Active", "Active"
    rows = [f"{UUID}, 2070, 2070, 900.1, 0x0, {na}, {na}, {na}, {na}",
            f"{UUID}, 1980, 2070, 1390.0, 0x4, {na}, {na}, {na}, {act}",
            f"{UUID}, 2060, 2070, 1200.0, 0x0, {na}, {na}, {na}, {na}",
            # another GPU of the machine: ignored once this GPU's rows are found
            f"{OTHER}, 900, 2070, 300.0, 0x8, {act}, {na}, {na}, {na}",
            "garbage line"]
    rec = _clocks(monkeypatch, rows).stop()
    assert rec == {"sm_mhz": 2060.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3, "matched_by_uuid": True}


def test_clock_record_without_uuid_match_uses_every_row(monkeypatch):
    na = "Not Active"
    rows = [f"{OTHER}, 1500, 2070, 500.0, 0x0, {na}, Active, {na}, {na}"]
    rec = _clocks(monkeypatch, rows).stop()
    assert rec["matched_by_uuid"] is False and rec["reasons"] == ["hw_thermal_slowdown"]
    assert _clocks(monkeypatch, []).stop() is None


def test_traffic_is_scaled_and_dropped_when_the_kernel_changes(monkeypatch):
    t = json.load(open(bench.os.path.join(bench.ROOT, "profiles", "traffic.json")))
    wl = next(k for k in t if not k.startswith("_"))
    rec = t[wl]["k_primal"]
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: rec["source_sha"])
    got = bench.measured_traffic("k_primal", wl, 2 * rec["alg_bytes_per_launch"])
    assert got == pytest.approx(2 * rec["dram_bytes_per_launch"])
    assert bench.measured_traffic("k_primal", "no_such_workload", 1.0) is None
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "0" * 16)
    assert bench.measured_traffic("k_primal", wl, rec["alg_bytes_per_launch"]) is None
    assert bench.measured_traffic("no_such_kernel", wl, 1.0) is None


def test_roofline_of_the_dominant_kernel_and_the_primal_least_bytes(monkeypatch):
    monkeypatch.setattr(bench, "peak_hbm", lambda: (6000.0, "measured"))
    monkeypatch.setattr(bench, "measured_traffic", lambda *a: None)
    # 10 iterations of 1e6 leaves: dual 2 ms, primal 5 ms in all
    res = {"profile": {"ms": [2.0, 5.0], "launches": [10, 10], "alg_bytes": [45e7, 2.1e9],
                       "leaf_iterations": 1e7}}
    r = bench.roofline(res, "at_scale")
    assert r["kernel"] == "k_primal" and r["launches"] == 10
    assert r["achieved"] == pytest.approx(2.1e9 / 5e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0)
    assert r["alg_bytes_per_launch"] == pytest.approx(2.1e8) and r["avg_launch_us"] == pytest.approx(500.0)
    assert r["other"]["kernel"] == "k_dual" and r["other"]["achieved"] == pytest.approx(225.0)
    m = r["k_primal_min_bytes"]
    assert m["bytes_per_leaf"] == 93
    assert m["achieved"] == pytest.approx(93 * 1e7 / 5e-3 / 1e9)
    assert m["frac"] == pytest.approx(m["achieved"] / 6000.0)


def test_peak_from_measured_file_else_fallback(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peak_hbm() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6783.5}))
    assert bench.peak_hbm() == (6783.5, "measured")


def test_reference_arm_line(monkeypatch, capsys):
    """--impl reference: the oracle on the bounded crop, one JSON line with the
    fields the comparison needs and no host<->device bytes."""
    from paper_1608_07411_gb300.scenes import make_scene
    a = types.SimpleNamespace(gpus=1, steps=1, warmup=0, seed=0, iters=0, fp16=False,
                              workload="sphere")
    bench.run_reference(a, make_scene("sphere", 0))
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == bench.METRIC and line["higher_is_better"] is True
    assert line["value"] > 0 and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.METRIC, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("sphere:")
