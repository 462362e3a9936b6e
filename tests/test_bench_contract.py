"""Host-side pieces of bench.py (no GPU): the algorithmic flop table equals the
oracle's counting build, and the peak arithmetic."""
import importlib

import pytest


def test_alg_flops_table_matches_oracle_count(orc):
    bench = importlib.import_module("bench")
    for (n, nt, gr), flops in bench.ALG_FLOPS.items():
        assert orc.count_flops(n, nt, gr)["flops"] == flops


def test_fp64_peak_from_unit_counts():
    bench = importlib.import_module("bench")
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.2586, rel=1e-4)
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(1.25, rel=0.01)   # nominal FP64 figure


def test_kernel_source_hash_is_stable():
    bench = importlib.import_module("bench")
    assert bench.kernel_source_hash() == bench.kernel_source_hash()
    assert len(bench.kernel_source_hash()) == 16
