"""The synthetic workload recipes of bench.py's serving and batch modes match
their stated definitions (families, size ranges, degrees, sample counts)."""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_batch_recipe():
    insts = bench.batch_instances(40, 4)
    for k, inst in enumerate(insts):
        if k % 2 == 0:
            assert inst.family == "diag"
            assert 200 <= inst.n <= 20000
            deg = 2.0 * inst.meta["edges"] / inst.n
            assert 2.0 <= deg <= 25.0  # average degree drawn in [4, 20], sampled
            assert np.array_equal(inst.b, np.ones(inst.n))
        else:
            assert inst.family == "observed"
            h = inst.n1
            assert inst.n == 2 * h and 500 <= h <= 5000
            assert inst.m == math.ceil(5 * h * math.log(h))
            assert inst.meta["rank"] == 3
    # the same seed gives the same instances
    again = bench.batch_instances(4, 4)
    assert all(a.n == b.n and a.m == b.m for a, b in zip(insts[:4], again))


def test_serving_recipe():
    reqs = bench.serve_requests(30, 1000, 20000, 5)
    fams = [inst.family for inst, _ in reqs]
    assert fams == ["diag", "edge", "observed"] * 10
    for k, (inst, U0) in enumerate(reqs):
        assert U0.shape == (inst.n, 2)
        if inst.family == "diag":
            assert 1000 <= inst.n <= 20000
            assert 4.0 <= 2.0 * inst.meta["edges"] / inst.n <= 12.0  # average degree 8
        elif inst.family == "edge":
            assert 1000 <= inst.n <= 20000
            assert inst.has_trace_row and inst.m == 5 * inst.n + 1  # G(n, 5n) + trace
            assert inst.C_J == -1.0 and inst.tau2 == 1.0
        else:
            h = inst.n1
            assert inst.n == 2 * h and inst.m == math.ceil(5 * h * math.log(h))
