"""Host logic of bench.py that needs no GPU: the captured DRAM traffic of the
level-0 sweep is reported only while the sweep kernel's source region is the
one that was captured."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_captured_traffic_follows_the_kernel_region(monkeypatch):
    got = bench.captured_traffic()
    assert got is None or got == bench.TRAFFIC_CAPTURE["bytes_per_sweep"]
    changed = dict(bench.TRAFFIC_CAPTURE, sha256="0" * 64)
    monkeypatch.setattr(bench, "TRAFFIC_CAPTURE", changed)
    assert bench.captured_traffic() is None
    missing = dict(bench.TRAFFIC_CAPTURE, regions=(("paper_2104_13755_gb300/csrc/kernels.cuh", "no such marker",
                                                     "// Damped Jacobi update"),))
    monkeypatch.setattr(bench, "TRAFFIC_CAPTURE", missing)
    assert bench.captured_traffic() is None


def test_sweep_bytes_formula():
    # one pass over the SELL entries (value + index), row pointers, and
    # b read, x read, x write per row and right-hand side
    n, z = 1000, 7000
    assert bench.sweep_bytes(n, z) == z * 12 + 4 * (n + 1) + 3 * 8 * n
    assert bench.sweep_bytes(n, z, s=4, k=2) == z * 8 + 4 * (n + 1) + 3 * 4 * 2 * n


def test_captured_cycle_traffic_follows_the_sources(monkeypatch):
    """The DRAM traffic of one captured cycle is reported only while the
    kernel and layout sources hash to the captured ones."""
    got = bench.captured_cycle_traffic()
    assert got is None or got == bench.CYCLE_TRAFFIC["bytes_per_cycle"]
    monkeypatch.setattr(bench, "CYCLE_TRAFFIC", dict(bench.CYCLE_TRAFFIC, sha256="0" * 64))
    assert bench.captured_cycle_traffic() is None
