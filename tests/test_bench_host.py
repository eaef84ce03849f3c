"""Host-side bookkeeping of bench.py: the method-only flop counts per element and the guard
that ties the recorded flux-kernel DRAM traffic to the kernel code it was measured on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_flop_counts_per_element_n5():
    # each step of the method counted once per element (n = 5, Navier-Stokes, 9 kept
    # gradient components): the steps add up to the total and to the kernels' shares
    f = bench.residual_flops_per_element(5)
    st = f["steps"]
    assert sum(st.values()) == f["total"] == 153375
    assert f["trace"] + f["grad"] + f["face"] + f["flux"] == f["total"]
    assert f["flux"] == st["interior"] + st["div"] == 87675
    # one 1D sweep of length n costs 2n - 1 flops: the 6 face traces of 5 variables on 25 lines
    assert st["trace"] == 6 * 5 * 25 * 9


def test_code_digest_ignores_comments_only():
    a = bench.code_digest(["int f(int x) {\n    return x + 1;  // add one\n}\n"])
    b = bench.code_digest(["/* doc */\nint f(int x) {\n\n    return x + 1;\n}   \n"])
    c = bench.code_digest(["int f(int x) {\n    return x + 2;\n}\n"])
    assert a == b
    assert a != c


def test_recorded_traffic_only_for_its_grid():
    t = bench.flux_traffic((bench.FLUX_TRAFFIC["ne"],) * 3)
    assert t is None or t == bench.FLUX_TRAFFIC["bytes"]
    assert bench.flux_traffic((24, 24, 24)) is None
