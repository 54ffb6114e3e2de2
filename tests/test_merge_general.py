"""The host half of general sparse input (Section 4.1, eqs. support S ell and
index list; Alg. 4 forms M on the pattern S from the lists L_ij):
``hallar_merge_general`` of the C ABI, checked against the oracle's
definition of A~*(p~) on random HSLR problems, and against its input rules.
Host arithmetic only: no GPU."""
import numpy as np
import pytest

from oracle import hallar_oracle as O
from paper_2505_13719_b300 import instances as I


@pytest.fixture(scope="module")
def H():
    from paper_2505_13719_b300.build import build_library
    build_library()
    from paper_2505_13719_b300 import hallar
    return hallar


def random_upper(n, m, count, seed):
    rng = np.random.default_rng(seed)
    ell = rng.integers(0, m + 1, size=count)
    a = rng.integers(0, n, size=count)
    b = rng.integers(0, n, size=count)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    v = rng.standard_normal(count)
    return ell, lo, hi, v


@pytest.mark.parametrize("n,m,count,seed", [(7, 3, 40, 1), (30, 12, 400, 2), (5, 0, 9, 3)])
def test_merged_lists_reproduce_the_adjoint_matrix(H, n, m, count, seed):
    ell, a, b, v = random_upper(n, m, count, seed)
    rowptr, col, lptr, lidx, lval = H.hallar_merge_general(n, m, ell, a, b, v)
    inst = I.hslr(n, (ell, a, b, v), [], np.zeros(m), tau2=1.0)
    rng = np.random.default_rng(seed + 10)
    pt = rng.standard_normal(m + 1)
    ref = O.adjoint_matrix(inst, pt)[0].toarray()
    M = np.zeros((n, n))
    for i in range(n):
        for e in range(rowptr[i], rowptr[i + 1]):
            j = col[e]
            assert e == rowptr[i] or col[e - 1] < j        # columns ascending
            lst = lidx[lptr[e]:lptr[e + 1]]
            assert np.all(np.diff(lst) > 0)                # each matrix once, ascending
            M[i, j] = float(np.dot(pt[lst], lval[lptr[e]:lptr[e + 1]]))
    np.testing.assert_allclose(M, ref, rtol=1e-13, atol=1e-13)
    # the pattern is the union of the supports, both triangles
    support = np.zeros((n, n), dtype=bool)
    for l in range(m + 1):
        D = np.zeros((n, n))
        sel = ell == l
        np.add.at(D, (a[sel], b[sel]), v[sel])
        D = D + np.triu(D, 1).T
        support |= D != 0.0
    stored = np.zeros((n, n), dtype=bool)
    for i in range(n):
        stored[i, col[rowptr[i]:rowptr[i + 1]]] = True
    assert np.array_equal(stored, support)


def test_repeats_are_summed_and_zeros_dropped(H):
    # (1, 0, 2) listed twice sums to 3; (2, 1, 1) cancels to 0 and (0, 0, 0)
    # is 0: neither is stored
    rowptr, col, lptr, lidx, lval = H.hallar_merge_general(
        3, 2, [1, 1, 2, 2, 0], [0, 0, 1, 1, 0], [2, 2, 1, 1, 0], [1.0, 2.0, 0.5, -0.5, 0.0])
    assert list(rowptr) == [0, 1, 1, 2]
    assert list(col) == [2, 0] and list(lidx) == [1, 1] and list(lval) == [3.0, 3.0]
    empty = H.hallar_merge_general(4, 1, [], [], [], [])
    assert list(empty[0]) == [0] * 5 and empty[1].size == 0 and list(empty[2]) == [0]


@pytest.mark.parametrize("ell,ii,jj,val,msg", [
    ([3], [0], [1], [1.0], "matrix index"),      # l > m
    ([1], [2], [1], [1.0], "upper triangle"),    # i > j
    ([1], [0], [4], [1.0], "upper triangle"),    # j >= n
    ([1], [0], [1], [float("nan")], "non-finite"),
])
def test_bad_entries_are_rejected(H, ell, ii, jj, val, msg):
    with pytest.raises(H.HallarError, match=msg) as e:
        H.hallar_merge_general(4, 2, ell, ii, jj, val)
    assert e.value.status == H.HALLAR_EINVAL
