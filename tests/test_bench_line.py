"""bench.py's reference arm on the host: the FP64 oracle timed on the small dense case, printed as
the benchmark line (metric, unit and config as the GPU arm's, the oracle's rate, its cpu_baseline and
e2e objects).  A rank other than 0 prints nothing."""
import types

import pytest

import bench

KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "impl", "config", "cpu_baseline", "e2e"}


@pytest.fixture(scope="module")
def small_line():
    args = types.SimpleNamespace(workload="gaussian-100x500-r16", steps=2, warmup=1)
    w = bench.WORKLOADS[args.workload]
    return args, w, bench.run_reference(args, w, 0, 1)


def test_reference_line_keys(small_line):
    args, w, line = small_line
    assert KEYS <= set(line)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["steps"] == 2 and line["warmup"] == 1
    assert line["config"] == bench.workload_config(args, w, 1)
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_other_ranks_silent():
    args = types.SimpleNamespace(workload="gaussian-100x500-r16", steps=1, warmup=0)
    assert bench.run_reference(args, bench.WORKLOADS[args.workload], 1, 2) is None


def test_config_states_l2_handling():
    args = types.SimpleNamespace(workload="spiked-5000x20000-r1024")
    cfg = bench.workload_config(args, bench.WORKLOADS[args.workload], 1)
    assert cfg["l2"].startswith("inputs larger than L2") and cfg["formulations"] == list(range(1, 9))
    args = types.SimpleNamespace(workload="gaussian-100x500-r16")
    assert "not flushed" in bench.workload_config(args, bench.WORKLOADS[args.workload], 1)["l2"]
