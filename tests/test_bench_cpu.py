"""Host-side pieces of bench.py: the per-launch DRAM traffic it reports for
the dominant kernel comes from the committed Nsight Compute summary of the
benchmark workload, and the replicas' aggregation takes the slowest rank."""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def args(**kw):
    a = dict(precision="fp32_refine", G=64, M=20000, k=16)
    a.update(kw)
    return argparse.Namespace(**a)


def test_traffic_of_each_step_kernel_is_read_from_the_profile_summary():
    for kernel in ("pass_a", "pass_b"):
        t = bench.ncu_traffic(args(), kernel)
        assert isinstance(t, int) and t > 10 ** 8, (kernel, t)
    # pass B moves about its algorithmic bytes (read u, g, w, Q; write g, w)
    mk, Mn = 20000 * 64 * 16, 20000 * 1234
    alg = 4 * (Mn + 5 * mk)
    assert 0.5 * alg < bench.ncu_traffic(args(), "pass_b") < 1.5 * alg


def test_no_traffic_without_a_matching_summary():
    assert bench.ncu_traffic(args(precision="fp64"), "pass_b") is None
    assert bench.ncu_traffic(args(M=12345), "pass_b") is None
    assert bench.ncu_traffic(args(), "reduce") is None


def test_single_rank_aggregate_is_the_rank_itself():
    ms, value = bench.aggregate(250.0, None, 1)
    assert ms == 250.0 and abs(value - 4.0) < 1e-12
