"""The benchmark's reference arm on CPU: rank 0 times the FP64 oracle on a slice of
the workload and prints one JSON line carrying the keys every bench line carries,
plus its own cpu_baseline and an e2e entry with no host-device copies."""
import json

import pytest


class _Args:
    workload = "channel_1m"
    steps = 1
    warmup = 0
    gpus = 1


def test_reference_arm_prints_one_line_with_the_contract_keys(monkeypatch, capsys):
    import bench

    real = bench.cpu_oracle_rate
    # a half-second slice instead of the two-minute budget of a real run
    monkeypatch.setattr(bench, "cpu_oracle_rate",
                        lambda name, **kw: real(name, **{**kw, "budget_s": 0.5}))
    monkeypatch.delenv("RANK", raising=False)
    assert bench.run_reference(_Args()) == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "particle-steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"] == "channel_1m"
    # ms_per_step is one step of the whole 983,040-fluid-particle workload at that rate
    assert d["ms_per_step"] == pytest.approx(1e3 * 983040 / d["value"])
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "FP64 steps" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
