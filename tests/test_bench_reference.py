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


def test_algorithmic_bytes_of_the_workloads():
    """The roofline's numerator: 136 B per pile body (q and v read and written, the 8-float
    parameter block read), q and v of an articulated world read and written (and, with
    controls, 16 torques of a hand read); the 4096 x 256 headline comes to 142.6 MB."""
    from paper_2603_12185_gb300 import scenes as S
    assert bench.BYTES_PER_BODY == 136
    sb = S.make_mixed(8, seed=0)                      # worlds: pile16, pile64, pile256, hand, twice
    per_pile = 136 * (16 + 64 + 256)
    assert bench.algorithmic_bytes_per_step(sb) == 2 * per_pile + 2 * (23 + 22) * 8
    assert bench.algorithmic_bytes_per_step(sb, controls=True) == 2 * per_pile + 2 * bench.HAND_BYTES
    assert bench.algorithmic_bytes_per_step(S.make_pile(64, 256, seed=0)) * 64 == 142606336
