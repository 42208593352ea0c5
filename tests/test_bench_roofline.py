"""The roofline arithmetic of bench.py at the main workload's degree (N = 7):
the counts that the bench line, the profiles and the design notes quote."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_volume_counts_at_N7():
    # 28 flops per symmetric pair, 7 pairs per node, 9 per node, 3 per side node
    assert bench.volume_flops_per_node(7) == pytest.approx(208.0)
    # the two-point form as written: 40 per pair, 20 per node
    assert bench.volume_flops_per_node_direct(7) == 300
    # W, velocities, 16N of pair constants, scalings, source, R, interface traces
    assert bench.volume_bytes_per_node(7) == pytest.approx(220.0)
    assert bench.volume_adjoint_flops_per_node(7) == pytest.approx(277.5)


def test_fp64_peak_at_2070_mhz():
    # 152 SMs x 2 DFMA per clock x 2 flops x 2.07 GHz
    assert bench.fp64_peak_gflops(2070.0) == pytest.approx(1258.56)


@pytest.mark.parametrize("N", range(1, 13))
def test_direct_form_counts_more_than_the_kernel(N):
    # the symmetric pair evaluated once is never more work than the direct form
    assert bench.volume_flops_per_node(N) < bench.volume_flops_per_node_direct(N)
