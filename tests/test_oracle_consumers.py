"""Pins of the oracle's consumers of a solved factor (not in the paper).

maxcut_round's cut value -x^T C x is checked against the weight of the
edges that the sign vector cuts, counted edge by edge from the graph; a
rank-one factor of a cut rounds back to that cut for every normal that is
not orthogonal to it; factor_entries matches the dense product UU^T.
"""
import numpy as np
import pytest

from oracle import hallar_oracle as O
from paper_2505_13719_b300 import instances as I


def cut_weight(ei, ej, w, x):
    return float(sum(wk for i, j, wk in zip(ei, ej, w) if x[i] != x[j]))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_round_cut_value_is_the_cut_edge_weight(seed):
    rng = np.random.default_rng(seed)
    n = 30
    ei, ej = I.er_graph(n, 0.2, seed)
    w = rng.uniform(-1.0, 2.0, ei.shape[0])
    inst = I.maxcut(n, ei, ej, w=w)
    U = rng.standard_normal((n, 4))
    G = rng.standard_normal((8, 4))
    cuts, X = O.maxcut_round(inst, U, G)
    for t in range(8):
        x = np.where(U @ G[t] < 0, -1, 1)
        assert np.array_equal(X[t], x)
        assert abs(cuts[t] - cut_weight(ei, ej, w, x)) <= 1e-12 * (1 + np.abs(w).sum())


def test_rank_one_cut_factor_rounds_to_its_cut():
    n = 16
    ei, ej = I.cycle_graph(n)  # even cycle: bipartite, max cut = n
    inst = I.maxcut(n, ei, ej)
    xs = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    rng = np.random.default_rng(0)
    G = rng.standard_normal((5, 1))
    cuts, X = O.maxcut_round(inst, xs[:, None] * 0.7, G)
    assert np.all(cuts == n)
    for t in range(5):
        assert np.array_equal(X[t], xs * np.sign(G[t, 0]))


def test_factor_entries_match_the_dense_product():
    rng = np.random.default_rng(4)
    U = rng.standard_normal((50, 6))
    a = rng.integers(0, 50, 200)
    b = rng.integers(0, 50, 200)
    X = U @ U.T
    assert np.allclose(O.factor_entries(U, a, b), X[a, b], rtol=1e-14, atol=1e-13)
