"""Host logic of bench.py that needs no GPU: the clock-sample summary and the
workload config both arms report."""
import tempfile

import pytest


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clocks_with(lines, skip):
    import bench
    c = object.__new__(bench.Clocks)
    c.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    c.f.write("\n".join(lines) + "\n")
    c.p = _FakeProc()
    c.skip = skip
    return c


def _line(sm, mx=2070, thermal="Not Active", power="Not Active"):
    return f"0, {sm}, {mx}, 900.5, 0x0, Not Active, {thermal}, Not Active, {power}"


def test_clock_summary_uses_samples_inside_the_timed_region():
    c = _clocks_with([_line(600), _line(2070), _line(2055, power="Active"), _line(2070)], skip=1)
    s = c.stop()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_falls_back_to_the_last_earlier_sample():
    c = _clocks_with([_line(1500), _line(2070, thermal="Active")], skip=2)
    s = c.stop()
    assert s["samples"] == 1 and s["sm_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown"]


def test_clock_summary_skips_malformed_lines():
    c = _clocks_with(["garbage", "0, [N/A], 2070, 1, 0x0, a, b, c, d", _line(2040)], skip=0)
    s = c.stop()
    assert s["samples"] == 1 and s["sm_mhz"] == 2040.0


def test_both_arms_share_the_workload_config():
    import bench
    from paper_2311_02542_gb300 import synth as S
    cfg = S.make_scene("room").cfg
    c = bench.workload_config(cfg, "room", 2)
    assert c["workload"] == bench.WORKLOAD and c["rays_per_step"] == 2048 * 2048
    assert c["levels"] == 16 and c["log2_T"] == 21 and c["occ_res"] == [256, 256, 256]
    assert c["parallelism"] == "replicas2"
    assert "mlp_precision" not in c


def test_clock_sampler_without_nvidia_smi_reports_it():
    import shutil

    import bench
    if shutil.which("nvidia-smi"):
        pytest.skip("nvidia-smi present")
    c = bench.Clocks(0)
    c.mark()
    s = c.stop()
    assert s["sm_mhz"] is None and s["reasons"] == ["nvidia-smi unavailable"]


def test_bench_line_ends_with_the_headline_keys():
    """The bulky extras come first; a reader that keeps only the end of the
    line still sees stereo latency, the fp32 comparison and the sweep."""
    import json

    import bench
    line = {"metric": "Mrays/s", "value": 1.0, "stereo_2x2048": {"p50_ms": 6.0}, "plain_fp32": {"value": 2.0},
            "precision_sweep": {"fp16": 1}, "serving": {"x": "y" * 4000}, "roofline": {"frac": 0.4},
            "train_step": {"ms": 1.0}, "clocks": {}}
    out = bench.tail_order(line)
    assert list(out)[:2] == ["metric", "value"]
    assert list(out)[-3:] == ["precision_sweep", "plain_fp32", "stereo_2x2048"]
    assert set(out) == set(line)
    tail = json.dumps(out)[-1500:]
    assert '"stereo_2x2048"' in tail and '"plain_fp32"' in tail and '"precision_sweep"' in tail
