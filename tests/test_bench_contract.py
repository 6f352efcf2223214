"""The reference arm's JSON line (CPU only: it times the FP64 oracle on the
host cores): the fields the benchmark contract requires, on one step of the
prox workload."""
import json


def test_reference_arm_line_has_the_contract_fields():
    import bench
    args = type("A", (), {"workload": "prox", "warmup": 0, "steps": 1, "n_inner": 1})()
    line = bench.run_reference(args, 0, 1)
    json.dumps(line)                                    # serialisable as one line
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["steps"] == 1 and line["ms_per_step"] > 0 and line["scaling"] == "weak"
    assert line["vs_baseline"] is None and line["data"] == "synthetic"
    assert line["config"]["workload"].startswith("prox_63_pairs_256x256")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
