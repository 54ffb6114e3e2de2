"""Pins of the oracle's operators against dense brute force and invariants.

The dense checks below build every A_l and C as explicit n x n matrices from
the family definitions (eq. Definition of Linear Operators, eq. A tilde
operator) and evaluate Frobenius products and matrix products directly; the
oracle evaluates the same quantities from entry lists.  A dropped term, a
wrong sign, a transposed pair or a wrong index in the oracle breaks one of
these.
"""
import math

import numpy as np
import pytest

from oracle import hallar_oracle as O
from paper_2505_13719_b300 import instances as I


def random_instance(family, n, seed, n1=0, trace=True, with_c=True, cj=0.0, ci=0.0):
    rng = np.random.default_rng(seed)
    # sparse symmetric C with a diagonal
    if with_c:
        k = max(1, n)
        ei = rng.integers(0, n, size=k)
        ej = rng.integers(0, n, size=k)
        keep = ei != ej
        ei, ej = ei[keep], ej[keep]
        key = np.unique(np.minimum(ei, ej) * n + np.maximum(ei, ej))
        ei, ej = key // n, key % n
        w = rng.standard_normal(ei.shape[0])
        diag = rng.standard_normal(n)
        rowptr, col, val = I._sym_csr(n, ei, ej, w, diag=diag)
    else:
        rowptr, col, val = I._empty_csr(n)
    if family == "diag":
        return I.Instance(name="t", family="diag", n=n, n1=0, C_rowptr=rowptr, C_col=col,
                          C_val=val, C_J=cj, C_I=ci, cons_i=np.zeros(0, np.int32),
                          cons_j=np.zeros(0, np.int32), has_trace_row=False,
                          b=rng.standard_normal(n), tau2=float(n))
    if family == "edge":
        ei, ej = I.gnm_graph(n, 2 * n, seed + 1)
        m = ei.shape[0] + (1 if trace else 0)
        return I.Instance(name="t", family="edge", n=n, n1=0, C_rowptr=rowptr, C_col=col,
                          C_val=val, C_J=cj, C_I=ci, cons_i=ei.astype(np.int32),
                          cons_j=ej.astype(np.int32), has_trace_row=trace,
                          b=rng.standard_normal(m), tau2=3.0)
    n2 = n - n1
    keys = rng.choice(n1 * n2, size=min(n1 * n2, 3 * n), replace=False)
    ci_, cj_ = keys // n2, keys % n2
    m = ci_.shape[0] + (1 if trace else 0)
    return I.Instance(name="t", family="observed", n=n, n1=n1, C_rowptr=rowptr, C_col=col,
                      C_val=val, C_J=cj, C_I=ci, cons_i=ci_.astype(np.int32),
                      cons_j=cj_.astype(np.int32), has_trace_row=trace,
                      b=rng.standard_normal(m), tau2=5.0)


def dense_C(inst):
    n = inst.n
    C = np.zeros((n, n))
    for i in range(n):
        for e in range(inst.C_rowptr[i], inst.C_rowptr[i + 1]):
            C[i, inst.C_col[e]] += inst.C_val[e]
    C += inst.C_J * np.ones((n, n)) + inst.C_I * np.eye(n)
    return C


def dense_As(inst):
    n = inst.n
    As = []
    if inst.family == "diag":
        for i in range(n):
            A = np.zeros((n, n))
            A[i, i] = 1.0
            As.append(A)
        return As
    off = inst.n1 if inst.family == "observed" else 0
    for i, j in zip(inst.cons_i, inst.cons_j):
        A = np.zeros((n, n))
        A[i, j + off] += 0.5
        A[j + off, i] += 0.5
        As.append(A)
    if inst.has_trace_row:
        As.append(np.eye(n))
    return As


CASES = [
    ("diag", 17, 0, False, True, 0.0, 0.0),
    ("diag", 23, 0, False, True, -0.7, 0.3),
    ("edge", 19, 0, True, False, -1.0, 0.0),
    ("edge", 21, 0, False, True, 0.4, -0.2),
    ("edge", 16, 0, True, True, -1.0, 0.25),
    ("observed", 20, 8, False, False, 0.0, 0.5),
    ("observed", 18, 7, True, True, 0.3, 0.5),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("r", [1, 3, 7])
def test_constraint_map_matches_dense(case, r):
    fam, n, n1, trace, with_c, cj, ci = case
    inst = random_instance(fam, n, 11 + r, n1=n1, trace=trace, with_c=with_c, cj=cj, ci=ci)
    U = np.random.default_rng(5 + r).standard_normal((n, r))
    X = U @ U.T
    T = O.eval_A_tilde(inst, U)
    ref = np.array([np.sum(dense_C(inst) * X)] + [np.sum(A * X) for A in dense_As(inst)])
    assert T.shape == (inst.m + 1,)
    np.testing.assert_allclose(T, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("case", CASES)
def test_adjoint_matches_dense(case):
    fam, n, n1, trace, with_c, cj, ci = case
    inst = random_instance(fam, n, 3, n1=n1, trace=trace, with_c=with_c, cj=cj, ci=ci)
    rng = np.random.default_rng(9)
    U = rng.standard_normal((n, 4))
    pt = rng.standard_normal(inst.m + 1)
    M = pt[0] * dense_C(inst) + sum(pl * A for pl, A in zip(pt[1:], dense_As(inst)))
    W = O.adjoint_apply(inst, pt, U)
    np.testing.assert_allclose(W, M @ U, rtol=1e-12, atol=1e-12 * np.abs(M @ U).max())


@pytest.mark.parametrize("case", CASES)
def test_adjoint_identity(case):
    # <A(UU^T), y> = <UU^T, A*(y)> = <A*(y) U, U>
    fam, n, n1, trace, with_c, cj, ci = case
    inst = random_instance(fam, n, 4, n1=n1, trace=trace, with_c=with_c, cj=cj, ci=ci)
    rng = np.random.default_rng(10)
    U = rng.standard_normal((n, 3))
    y = rng.standard_normal(inst.m)
    lhs = float(O.constraint_map(inst, U) @ y)
    rhs = float(np.sum(O.adjoint_apply(inst, np.concatenate([[0.0], y]), U) * U))
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + 1.0)
    # the cost row: C.UU^T = <C U, U>
    c0 = O.cost_dot(inst, U)
    e0 = np.zeros(inst.m + 1)
    e0[0] = 1.0
    assert abs(c0 - float(np.sum(O.adjoint_apply(inst, e0, U) * U))) <= 1e-11 * (abs(c0) + 1)


@pytest.mark.parametrize("case", CASES[:5])
def test_gradient_finite_differences(case):
    fam, n, n1, trace, with_c, cj, ci = case
    inst = random_instance(fam, n, 6, n1=n1, trace=trace, with_c=with_c, cj=cj, ci=ci)
    rng = np.random.default_rng(12)
    U = 0.5 * rng.standard_normal((n, 2))
    p = rng.standard_normal(inst.m)
    beta = 1.7
    gr = O.al_grad(inst, U, p, beta)
    grad = 2.0 * gr.W
    h = 1e-6
    for _ in range(6):
        Dir = rng.standard_normal(U.shape)
        fp = O.al_value(inst, U + h * Dir, p, beta)
        fm = O.al_value(inst, U - h * Dir, p, beta)
        fd = (fp - fm) / (2 * h)
        an = float(np.sum(grad * Dir))
        assert abs(fd - an) <= 1e-6 * (abs(an) + 1.0)
    # entrywise on a few coordinates
    for (a, b) in [(0, 0), (n - 1, 1), (n // 2, 0)]:
        E = np.zeros_like(U)
        E[a, b] = 1.0
        fd = (O.al_value(inst, U + h * E, p, beta) - O.al_value(inst, U - h * E, p, beta)) / (2 * h)
        assert abs(fd - grad[a, b]) <= 1e-6 * (abs(grad[a, b]) + 1.0)


@pytest.mark.parametrize("case", CASES)
def test_al_value_and_gradient_matrix(case):
    # g(U) = C.X + p^T(A(X) - b) + beta/2 |A(X) - b|^2 and G.UU^T = <W, U>,
    # G = C + A*(p + beta(A(X) - b)), all formed densely
    fam, n, n1, trace, with_c, cj, ci = case
    inst = random_instance(fam, n, 7, n1=n1, trace=trace, with_c=with_c, cj=cj, ci=ci)
    rng = np.random.default_rng(13)
    U = rng.standard_normal((n, 3))
    p = rng.standard_normal(inst.m)
    beta = 0.9
    X = U @ U.T
    C = dense_C(inst)
    As = dense_As(inst)
    AX = np.array([np.sum(A * X) for A in As])
    r = AX - inst.b
    g_ref = np.sum(C * X) + p @ r + 0.5 * beta * r @ r
    G = C + sum(q * A for q, A in zip(p + beta * r, As))
    gr = O.al_grad(inst, U, p, beta)
    assert abs(gr.g - g_ref) <= 1e-11 * (abs(g_ref) + np.abs(r).sum() + 1)
    np.testing.assert_allclose(gr.resid, r, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(gr.W, G @ U, rtol=1e-12, atol=1e-11 * np.abs(G @ U).max())
    assert abs(float(np.sum(gr.W * U)) - float(np.sum(G * X))) <= 1e-10 * (np.abs(G * X).sum())


@pytest.mark.parametrize("case", CASES)
def test_value_change(case):
    fam, n, n1, trace, with_c, cj, ci = case
    inst = random_instance(fam, n, 8, n1=n1, trace=trace, with_c=with_c, cj=cj, ci=ci)
    rng = np.random.default_rng(14)
    X = rng.standard_normal((n, 3))
    Y = X + 0.3 * rng.standard_normal((n, 3))
    p = rng.standard_normal(inst.m)
    dg, rY = O.al_value_change(inst, X, Y, p, 1.3)
    ref = O.al_value(inst, Y, p, 1.3) - O.al_value(inst, X, p, 1.3)
    assert abs(dg - ref) <= 1e-10 * (abs(ref) + 1.0)
    np.testing.assert_allclose(rY, O.constraint_map(inst, Y) - inst.b, rtol=1e-12, atol=1e-11)
    # a tiny step: the difference form keeps relative accuracy where the plain
    # difference of values loses it
    Yt = X + 1e-9 * rng.standard_normal((n, 3))
    dg_small, _ = O.al_value_change(inst, X, Yt, p, 1.3)
    gr = O.al_grad(inst, X, p, 1.3)
    first_order = float(np.sum(2.0 * gr.W * (Yt - X)))
    assert abs(dg_small - first_order) <= 1e-6 * abs(first_order)


def test_maxcut_cost_is_minus_cut():
    # C = -L/4: C . xx^T = -(weight of the cut of x) for x in {-1, 1}^n
    rng = np.random.default_rng(3)
    n = 30
    ei, ej = I.er_graph(n, 0.3, 4)
    w = rng.uniform(0.5, 2.0, size=ei.shape[0])
    inst = I.maxcut(n, ei, ej, w)
    for _ in range(5):
        x = rng.choice([-1.0, 1.0], size=n)
        cut = sum(wk for a, b, wk in zip(ei, ej, w) if x[a] != x[b])
        assert abs(O.cost_dot(inst, x[:, None]) + cut) <= 1e-12 * cut


def test_c_norm1_matches_dense():
    for case in CASES:
        fam, n, n1, trace, with_c, cj, ci = case
        inst = random_instance(fam, n, 15, n1=n1, trace=trace, with_c=with_c, cj=cj, ci=ci)
        ref = np.abs(dense_C(inst)).sum(axis=0).max()
        assert abs(O.c_norm1(inst) - ref) <= 1e-12 * ref


def test_projection_onto_ball():
    rng = np.random.default_rng(0)
    U = rng.standard_normal((10, 3))
    tau = 2.0
    P = O.project_ball(U, tau)
    assert abs(np.linalg.norm(P) - tau) < 1e-12
    # variational inequality of the projection: <U - P, V - P> <= 0 on the ball
    for _ in range(20):
        V = rng.standard_normal((10, 3))
        V = V * (tau * rng.random() / np.linalg.norm(V))
        assert float(np.sum((U - P) * (V - P))) <= 1e-12
    small = 0.1 * U / np.linalg.norm(U)
    assert np.array_equal(O.project_ball(small, tau), small)
