"""CPU checks of bench.py's measurement arithmetic: the DRAM traffic figure
is used only for the kernel source it was captured on, the HBM roofline
takes the measured copy bandwidth, and the algorithmic bytes of a unit count
what a refactorization and a solve must move."""
import hashlib
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


def test_traffic_is_used_only_for_the_kernel_it_was_captured_on(bench):
    """A capture is valid only for the kernel it was taken on: a stored
    traffic figure is reported when it names the current refactor.cu, and
    the bench reports null traffic once the kernel has changed."""
    src = os.path.join(ROOT, "paper_2411_14082_gb300", "csrc", "refactor.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    for name, t in bench.REFACTOR_TRAFFIC.items():
        want = t["bytes"] if t["refactor_cu_sha256"] == sha else None
        assert bench.refactor_traffic(name) == want, name
    assert bench.refactor_traffic("no such workload") is None


def test_hbm_roofline_uses_the_measured_peak(bench):
    """The measured copy bandwidth when the peaks file is there, else the
    stated fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak, src = bench.hbm_peak_gbs()
    if os.path.exists(path):
        assert src == "measured" and peak == json.load(open(path))["hbm_gbs"]
    else:
        assert src == "fallback" and peak == 6800.0
    r = bench.hbm_roofline(2.0e9, 0.5, traffic=4.0e9)
    assert r["algorithmic_gbs"] == pytest.approx(4.0)
    assert r["frac"] == pytest.approx(4.0 / peak)
    assert r["dram_gbs"] == pytest.approx(8.0) and r["dram_frac"] == pytest.approx(8.0 / peak)


def test_unit_bytes_counts_each_array_once(bench):
    """One unit: A's values, row ids and slot map read once, column
    pointers, the factor written with its indices, then both solves reading
    the factor with its indices once, plus the right-hand side, the
    permutations and the intermediate vectors.  It grows by 24 bytes per
    factor entry and 16 per entry of A."""
    base = bench.unit_bytes(100, 500, 2000)
    assert bench.unit_bytes(100, 500, 2001) - base == 24
    assert bench.unit_bytes(100, 501, 2000) - base == 16
    assert bench.unit_bytes(0, 0, 0) == 4 + 16
