"""Pins of the synthetic instance generators against the sizes the paper prints.

* matrix completion: m = ceil(r^2 ln(n1 + n2) (n1 + n2)) reproduces every
  (n1, n2, r; m) row of Table tab:gpuourmethod_vs_cpu (Section 5.2);
* Hamming graphs H(d, 2): n = 2^d and |E| = d 2^(d-1) reproduce the first
  column of Table tab:reduced_hamming_graphs (Section 5.3).
"""
import csv
import os

import numpy as np
import pytest

from paper_2505_13719_b300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return list(csv.DictReader(line for line in f if not line.startswith("#")))


def test_completion_sample_count_matches_paper_table():
    rows = _rows("matrix_completion_sizes.csv")
    assert len(rows) == 22
    for row in rows:
        m = I.completion_sample_count(int(row["n1"]), int(row["n2"]), int(row["r"]))
        assert m == int(row["m"]), row


def test_hypercube_sizes_match_paper_table():
    for row in _rows("hamming_graph_sizes.csv"):
        d = int(row["d"])
        if d > 16:
            # closed form for the large rows, enumeration for the small ones
            assert (1 << d) == int(row["n"]) and d * (1 << (d - 1)) == int(row["edges"])
            continue
        ei, ej = I.hypercube_graph(d)
        assert (1 << d) == int(row["n"])
        assert ei.shape[0] == int(row["edges"])
        assert np.all(np.bitwise_count(ei ^ ej) == 1)


def test_torus_graph_structure():
    ei, ej = I.torus_graph(5, 7)
    assert ei.shape[0] == 2 * 35
    deg = np.bincount(np.concatenate([ei, ej]), minlength=35)
    assert np.all(deg == 4)
    key = ei * 35 + ej
    assert np.unique(key).shape[0] == key.shape[0]


def test_maxcut_laplacian_rows_sum_to_zero():
    inst = I.maxcut_torus(6, "pm1", seed=1)
    rs = np.add.reduceat(inst.C_val, inst.C_rowptr[:-1])
    np.testing.assert_allclose(rs, 0.0, atol=1e-15)
    assert inst.tau2 == inst.n and np.all(inst.b == 1.0)


def test_gnm_graph_distinct_edges():
    ei, ej = I.gnm_graph(1000, 5000, 3)
    assert ei.shape[0] == 5000
    assert np.all(ei < ej)
    assert np.unique(ei * 1000 + ej).shape[0] == 5000


def test_generators_are_seeded():
    a = I.maxcut_er_1000()
    b = I.maxcut_er_1000()
    assert np.array_equal(a.C_col, b.C_col) and np.array_equal(a.C_val, b.C_val)
    assert a.meta["edges"] > 4000 and a.meta["edges"] < 6000
