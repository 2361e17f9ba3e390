"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps the JSON line's
contract: exactly K timed steps after W untimed ones, and the keys the GPU arm prints."""
import sys

import bench


def test_reference_arm_times_k_steps_after_w(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "3", "--warmup", "2",
                                      "--bodies", "16"])
    line = bench.reference_arm(bench.parse())
    assert line["impl"] == "reference" and line["steps"] == 3 and line["warmup"] == 2
    assert line["unit"] == "world-steps/s" and line["higher_is_better"] is True and line["dtype"] == "f64"
    assert line["value"] > 0 and line["ms_per_step"] > 0
    n = line["config"]["worlds_sampled"]
    assert abs(line["value"] - 1e3 * n / line["ms_per_step"]) <= 1e-9 * line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "world-steps/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert "steps 4..6 timed after 3 untimed" in cb["sample"]
