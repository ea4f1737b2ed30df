"""Host-side logic of the benchmark: algorithmic bytes, traffic lookup, rate helpers."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_per_cell_at_the_headline_grid(bench):
    ng, n = 300, 256
    spec = 8.0 * 151 / 300                       # one half-spectrum value per cell, complex FP32
    assert spec == pytest.approx(4.0267, abs=1e-4)
    assert bench.bytes_per_cell(3, ng, n) == pytest.approx(3 * spec)          # column G: 1 in, 2 out
    assert bench.bytes_per_cell(4, ng, n) == pytest.approx(4 * spec)          # column pair: 2 in, 2 out
    assert bench.bytes_per_cell(5, ng, n) == pytest.approx(3 * spec)          # column sum: 2 in, 1 out
    assert bench.bytes_per_cell(2, ng, n) == pytest.approx(4 * spec + 16)     # velocity row
    assert bench.bytes_per_cell(1, ng, n) == pytest.approx(3 * spec + 24)     # density row with history
    assert bench.bytes_per_cell(1, ng, n, ckpt_hist=False) == pytest.approx(3 * spec + 20)
    assert bench.bytes_per_cell(6, ng, n) == pytest.approx(3 * spec + 24 + 8 * n * n / ng ** 2)
    # one column-pair launch of K = 8 data sets moves 11.6 MB (the roofline's per-launch bytes)
    assert bench.bytes_per_cell(4, ng, n) * ng * ng * 8 == pytest.approx(11596800.0)


def test_stored_traffic_is_used_only_for_the_profiled_sources(bench, tmp_path, monkeypatch):
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    h = d["kernel_source_hash"]
    assert bench.stored_traffic(4, h) == d["4"]["dram_bytes_per_launch_full"]
    assert bench.stored_traffic(4, "0" * 16) is None
    assert bench.stored_traffic(9, h) is None                 # no such class
    assert len(bench.kernel_source_hash()) == 16


def test_rate_helpers(bench):
    # whole-job rate: units of all ranks over the slowest rank's time
    assert bench.whole_job_rate(1, 5, 500.0) == pytest.approx(10.0)
    assert bench.whole_job_rate(4, 5, 1000.0) == pytest.approx(20.0)
