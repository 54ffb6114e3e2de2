"""Host-side problem validation and merge (hallar_check_problem): the same
code path hallar_create runs before any upload, exercised without a GPU.
Merged sizes are checked against counts taken from the instances' own CSR
and constraint lists, the induced 1-norm of C against the oracle, and every
validation error against its message."""
import numpy as np
import pytest

from oracle import hallar_oracle as O
from paper_2505_13719_b300 import instances as I
from tests.test_oracle_operators import random_instance


@pytest.fixture(scope="module")
def H():
    from paper_2505_13719_b300.build import build_library
    build_library()
    from paper_2505_13719_b300 import hallar
    return hallar


def offdiag_entries(inst):
    """Distinct stored off-diagonal positions of C's sparse part."""
    if inst.C_rowptr is None:
        return 0
    count = 0
    for i in range(inst.n):
        cols = inst.C_col[inst.C_rowptr[i]:inst.C_rowptr[i + 1]]
        count += len({int(j) for j in cols if j != i})
    return count


INSTANCES = [
    ("maxcut ER", lambda: I.maxcut(300, *I.er_graph(300, 0.05, 1))),
    ("maxcut torus", lambda: I.maxcut_torus(12, "pm1", seed=2)),
    ("theta C9", lambda: I.theta(9, *I.cycle_graph(9))),
    ("completion", lambda: I.completion(30, 40, 2, 500, seed=3)),
    ("edge with C", lambda: random_instance("edge", 200, 4, trace=True, with_c=True,
                                            cj=-0.5, ci=0.2)),
    ("diag with C_J", lambda: random_instance("diag", 150, 5, with_c=True, cj=0.3, ci=-0.1)),
]


@pytest.mark.parametrize("name,make", INSTANCES, ids=[x[0] for x in INSTANCES])
def test_merged_sizes_and_norm(H, name, make):
    inst = make()
    m, nnz, cn = H.check_instance(inst)
    assert m == inst.m
    pairs = 0 if inst.family == "diag" else len(inst.cons_i)
    assert nnz == offdiag_entries(inst) + 2 * pairs
    assert cn == pytest.approx(O.c_norm1(inst), rel=1e-12)


def base():
    inst = I.maxcut(20, *I.cycle_graph(20))
    return dict(n=inst.n, n1=0, C_rowptr=inst.C_rowptr.copy(), C_col=inst.C_col.copy(),
                C_val=inst.C_val.copy(), C_J=0.0, C_I=0.0, family="diag",
                cons_i=np.zeros(0, np.int32), cons_j=np.zeros(0, np.int32),
                has_trace_row=False, b=np.ones(inst.n), tau2=float(inst.n))


def edge_base():
    ei, ej = I.cycle_graph(9)
    d = base()
    d.update(n=9, C_rowptr=None, C_col=None, C_val=None, C_J=-1.0, family="edge",
             cons_i=ei.astype(np.int32), cons_j=ej.astype(np.int32), has_trace_row=True,
             b=np.concatenate([np.zeros(len(ei)), [1.0]]), tau2=1.0)
    return d


def asym(d):
    d["C_val"][np.argmax(d["C_col"] != np.repeat(np.arange(d["n"]), np.diff(d["C_rowptr"])))] += 1.0
    return d


CASES = [
    ("n <= 0", lambda d: d.update(n=0), "n must be"),
    ("tau2 <= 0", lambda d: d.update(tau2=0.0), "tau2"),
    ("b non-finite", lambda d: d["b"].__setitem__(3, np.nan), "b has a non-finite"),
    ("C non-finite", lambda d: d["C_val"].__setitem__(0, np.inf), "non-finite value"),
    ("C column out of range", lambda d: d["C_col"].__setitem__(0, 20), "out of range"),
    ("C asymmetric", asym, "symmetric"),
    ("rowptr not monotone", lambda d: d["C_rowptr"].__setitem__(5, d["C_rowptr"][7]),
     "monotone"),
    ("C_J not finite", lambda d: d.update(C_J=np.nan), "C_J"),
]


@pytest.mark.parametrize("name,mutate,msg", CASES, ids=[c[0] for c in CASES])
def test_validation_errors(H, name, mutate, msg):
    d = base()
    mutate(d)
    with pytest.raises(H.HallarError) as e:
        H.hallar_check_problem(**d)
    assert e.value.status == H.HALLAR_EINVAL
    assert msg in str(e.value), str(e.value)


def test_pair_validation_errors(H):
    d = edge_base()
    H.hallar_check_problem(**d)  # valid
    d2 = edge_base()
    d2["cons_j"] = d2["cons_j"].copy()
    d2["cons_j"][0] = d2["cons_i"][0]
    with pytest.raises(H.HallarError) as e:
        H.hallar_check_problem(**d2)
    assert "i == j" in str(e.value)
    d3 = edge_base()
    d3["cons_j"] = d3["cons_j"].copy()
    d3["cons_j"][1] = 9
    with pytest.raises(H.HallarError) as e:
        H.hallar_check_problem(**d3)
    assert "out of range" in str(e.value)


def test_diag_family_rejects_pairs_at_the_c_abi(H):
    # the binding never passes pairs for the diagonal family; the C entry
    # point itself must refuse them
    import ctypes as C
    d = base()
    rp = np.ascontiguousarray(d["C_rowptr"], np.int64)
    ci = np.ascontiguousarray(d["C_col"], np.int32)
    cv = np.ascontiguousarray(d["C_val"], np.float64)
    pi = np.array([0], np.int32)
    pj = np.array([1], np.int32)
    b = np.ones(d["n"])
    st = H._lib.hallar_check_problem(d["n"], 0, rp.ctypes.data, ci.ctypes.data, cv.ctypes.data,
                                     0.0, 0.0, H.HALLAR_DIAG, 1, pi.ctypes.data, pj.ctypes.data,
                                     0, b.ctypes.data, float(d["n"]), None, None, None)
    assert st == H.HALLAR_EINVAL
    assert "DIAG" in H.hallar_last_error()
