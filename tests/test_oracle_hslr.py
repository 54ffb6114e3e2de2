"""Pins of the oracle on general problems in HSLR form (Section 3.2, eq.
HSLR-rep-body: A_l = A_l^sp + K_l D_l K_l^T, C = A_0) and of the SDPA
reader (Section 3.2; Section 4.3, eq. constraint matrix density).

* Operators against dense brute force built here from the raw inputs
  (A_l as n x n arrays, never through the oracle): the constraint map, the
  cost, the adjoint product (Algs. 3 and 5), the value change.
* The adjoint identity <A*(p)U, U> = p . A(UU^T) and a finite-difference
  check of the AL gradient.
* A closed form through the low-rank path: theta(C_5) = sqrt(5) with
  C = -11^T given as the rank-one term 1 (-1) 1^T, and the same solve with
  C given as sparse entries.
* The SDPA reader: a Max-Cut SDP of an odd cycle written as SDPA text by the
  test, read back, solved to its closed form (n/2)(1 + cos(pi/n)); the
  density split at 0.1; malformed inputs.
"""
import math

import numpy as np
import pytest

from oracle import hallar_oracle as O
from paper_2505_13719_b300 import instances as I
from paper_2505_13719_b300 import sdpa


def random_hslr(n=9, m=4, seed=5):
    """A random HSLR problem and its dense matrices A_0..A_m, built
    independently of the oracle."""
    rng = np.random.default_rng(seed)
    ell, a, b, v = [], [], [], []
    dense = [np.zeros((n, n)) for _ in range(m + 1)]
    for l in range(m + 1):
        for _ in range(6):
            i, j = sorted(rng.integers(0, n, size=2))
            w = float(rng.standard_normal())
            ell.append(l); a.append(i); b.append(j); v.append(w)
            dense[l][i, j] += w
            if i != j:
                dense[l][j, i] += w
    terms = []
    for l in (0, 2, 3):
        r = 2 if l != 3 else 1
        K = rng.standard_normal((n, r))
        D = rng.standard_normal((r, r))
        D = D + D.T  # symmetric, not diagonal
        terms.append((l, K, D))
        dense[l] += K @ D @ K.T
    inst = I.hslr(n, (np.array(ell), np.array(a), np.array(b), np.array(v)), terms,
                  rng.standard_normal(m), tau2=4.0)
    return inst, dense


def test_hslr_operators_match_dense_brute_force():
    inst, A = random_hslr()
    rng = np.random.default_rng(8)
    U = rng.standard_normal((inst.n, 3))
    X = U @ U.T
    T = O.eval_A_tilde(inst, U)
    ref = np.array([float(np.sum(A[l] * X)) for l in range(inst.m + 1)])
    np.testing.assert_allclose(T, ref, rtol=1e-12, atol=1e-12)
    pt = rng.standard_normal(inst.m + 1)
    W = O.adjoint_apply(inst, pt, U)
    Wref = sum(pt[l] * A[l] for l in range(inst.m + 1)) @ U
    np.testing.assert_allclose(W, Wref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(O.dense_adjoint(inst, pt),
                               sum(pt[l] * A[l] for l in range(inst.m + 1)),
                               rtol=1e-12, atol=1e-12)


def test_hslr_value_change_and_adjoint_identity():
    inst, A = random_hslr(seed=9)
    rng = np.random.default_rng(10)
    Xf = rng.standard_normal((inst.n, 2))
    Yf = Xf + 1e-3 * rng.standard_normal((inst.n, 2))
    p = rng.standard_normal(inst.m)
    beta = 3.0

    def g_dense(U):
        M = U @ U.T
        r = np.array([np.sum(A[l] * M) for l in range(1, inst.m + 1)]) - inst.b
        return float(np.sum(A[0] * M) + p @ r + 0.5 * beta * r @ r)

    dg, _ = O.al_value_change(inst, Xf, Yf, p, beta)
    assert abs(dg - (g_dense(Yf) - g_dense(Xf))) <= 1e-10 * (1 + abs(dg))
    # <A*(p)U, U> = p~ . A~(UU^T)
    pt = np.concatenate([[0.7], p])
    lhs = float(np.sum(O.adjoint_apply(inst, pt, Xf) * Xf))
    assert abs(lhs - float(pt @ O.eval_A_tilde(inst, Xf))) <= 1e-12 * (1 + abs(lhs))
    # grad g = 2 (C + A*(p + beta r)) U, by central differences
    gr = O.al_grad(inst, Xf, p, beta)
    E = rng.standard_normal(Xf.shape)
    h = 1e-6
    fd = (g_dense(Xf + h * E) - g_dense(Xf - h * E)) / (2 * h)
    assert abs(fd - float(np.sum(2.0 * gr.W * E))) <= 1e-6 * (1 + abs(fd))


def theta_c5_hslr(lowrank_cost: bool):
    """theta(C_5) (eq. lovasz): min -11^T . X s.t. X_ij = 0 on the edges,
    tr X = 1, X psd; C as the rank-one term K D K^T = 1 (-1) 1^T or as
    sparse entries."""
    n = 5
    ei, ej = I.cycle_graph(n)
    m = ei.shape[0] + 1
    ell = list(range(1, m))
    a = [int(x) for x in ei]
    b = [int(x) for x in ej]
    v = [0.5] * (m - 1)  # A_l = (e_i e_j^T + e_j e_i^T)/2
    ell += [m] * n; a += list(range(n)); b += list(range(n)); v += [1.0] * n
    terms = []
    if lowrank_cost:
        terms = [(0, np.ones((n, 1)), np.array([[-1.0]]))]
    else:
        iu, ju = np.triu_indices(n)
        ell += [0] * iu.shape[0]; a += list(iu); b += list(ju); v += [-1.0] * iu.shape[0]
    bvec = np.zeros(m)
    bvec[-1] = 1.0
    return I.hslr(n, (np.array(ell), np.array(a), np.array(b), np.array(v)), terms,
                  bvec, tau2=1.0, sense=-1.0)


@pytest.mark.parametrize("lowrank_cost", [True, False])
def test_theta_c5_in_hslr_form(lowrank_cost):
    inst = theta_c5_hslr(lowrank_cost)
    res = O.hallar_solve(inst, I.initial_factor(inst.n, 2, 7), opt=O.Options(tol=1e-7))
    assert res.converged
    assert abs(inst.sense * res.pval - math.sqrt(5.0)) <= 1e-6 * math.sqrt(5.0)
    assert O.c_norm1(inst) == pytest.approx(5.0)


def maxcut_sdpa_text(n, ei, ej):
    """Max-Cut SDP of a graph in SDPA-sparse text: max (1/4) L . Y s.t.
    Y_ii = 1 (F_0 = L/4, F_i = e_i e_i^T, c_i = 1), written by this test."""
    deg = np.zeros(n)
    np.add.at(deg, ei, 1.0)
    np.add.at(deg, ej, 1.0)
    lines = ['"Max-Cut SDP of a cycle', f"{n} = m", "1 = nblocks", f"{n}",
             " ".join(["1.0"] * n)]
    for i in range(n):
        lines.append(f"0 1 {i + 1} {i + 1} {deg[i] / 4.0}")
    for i, j in zip(ei, ej):
        lines.append(f"0,1,{min(i, j) + 1},{max(i, j) + 1},-0.25")
    for i in range(n):
        lines.append(f"{i + 1} 1 {i + 1} {i + 1} 1.0")
    return "\n".join(lines) + "\n"


def test_sdpa_maxcut_odd_cycle_closed_form():
    n = 7
    ei, ej = I.cycle_graph(n)
    inst = sdpa.parse(maxcut_sdpa_text(n, ei, ej), tau2=float(n))
    assert inst.m == n and inst.family == "hslr"
    # F_0 = L/4 of C_7 has 7 + 14 nonzeros: d_0 = 21/49 > 0.1 is dense; each
    # e_i e_i^T has d = 1/49
    assert inst.meta["dense"][0] and not inst.meta["dense"][1:].any()
    res = O.hallar_solve(inst, I.initial_factor(n, 2, 3), opt=O.Options(tol=1e-7))
    assert res.converged
    ref = (n / 2.0) * (1.0 + math.cos(math.pi / n))
    assert abs(inst.sense * res.pval - ref) <= 1e-6 * ref
    # the same problem through the built-in diagonal family
    base = I.maxcut(n, ei, ej)
    U = np.random.default_rng(4).standard_normal((n, 3))
    np.testing.assert_allclose(O.eval_A_tilde(inst, U), O.eval_A_tilde(base, U),
                               rtol=1e-13, atol=1e-13)
    # write / parse round trip
    again = sdpa.parse(sdpa.write(inst), tau2=float(n))
    np.testing.assert_allclose(O.eval_A_tilde(again, U), O.eval_A_tilde(inst, U),
                               rtol=1e-15, atol=1e-15)


def test_sdpa_density_split():
    # eq. constraint matrix density: d_l = nnz / n^2, dense above 0.1
    n = 6
    lines = ["2", "1", f"{n}", "1.0 2.0"]
    iu, ju = np.triu_indices(n)
    lines += [f"1 1 {i + 1} {j + 1} 1.0" for i, j in zip(iu, ju)]  # all ones: d = 1
    lines += ["2 1 1 1 1.0", "2 1 2 3 1.0"]                          # d = 3/36
    inst = sdpa.parse("\n".join(lines), tau2=2.0)
    np.testing.assert_allclose(inst.meta["density"], [0.0, 1.0, 3.0 / 36.0])
    assert list(inst.meta["dense"]) == [False, True, False]


@pytest.mark.parametrize("text", [
    "1\n2\n3 3\n1.0\n",                 # two blocks
    "1\n1\n-3\n1.0\n",                  # a diagonal (LP) block
    "1\n1\n3\n1.0\n1 1 2 1 1.0\n",      # below the diagonal
    "1\n1\n3\n1.0\n1 1 4 4 1.0\n",      # index out of range
    "1\n1\n3\n1.0\n1 1 1 1\n",          # short entry line
])
def test_sdpa_rejects_malformed_input(text):
    with pytest.raises(ValueError):
        sdpa.parse(text, tau2=1.0)


def test_device_binding_refuses_the_general_family():
    from paper_2505_13719_b300 import hallar as H
    with pytest.raises(ValueError, match="implements"):
        H.create_from_instance(theta_c5_hslr(True))
