"""Pins of the oracle's full HALLaR solve (Alg. 1 with ADAP-AIPP / ADAP-FISTA)
against SDP values known in closed form, and its certificates.

Closed forms:
* Max-Cut SDP of K_n = n^2/4; of a bipartite graph with nonnegative weights
  = total weight; of the odd cycle C_n = (n/2)(1 + cos(pi/n)).
* Lovasz theta: theta(C_n) = n cos(pi/n)/(1 + cos(pi/n)) for odd n;
  theta(K_n) = 1; theta of the empty graph = n (optimal X = 11^T/n);
  theta(Q_d) = 2^(d-1) (Q_d is bipartite, hence perfect, eq. lovasz remark).
* Matrix completion (eq. matcomp-sdp): with enough samples the optimum is
  ||M||_* and the off-diagonal block of X is M.
"""
import math

import numpy as np
import pytest

from oracle import hallar_oracle as O
from paper_2505_13719_b300 import instances as I
from tests.test_oracle_operators import dense_As, dense_C

TOL = 1e-7


def solve(inst, r0=2, seed=7, **kw):
    opt = O.Options(tol=TOL, **kw)
    return O.hallar_solve(inst, I.initial_factor(inst.n, r0, seed), opt=opt)


def check_certificate(inst, res):
    # S = C + A*p + theta I psd (eq. St) by dense eigendecomposition, and
    # the relative KKT residuals of eq. termination2 below the tolerance
    S = dense_C(inst) + sum(q * A for q, A in zip(res.p, dense_As(inst))) + res.theta * np.eye(inst.n)
    lam = np.linalg.eigvalsh(S)[0]
    assert lam >= -1e-5 * (1 + np.abs(dense_C(inst)).sum(axis=0).max())
    assert res.converged and res.kkt <= TOL
    assert np.linalg.norm(res.U) <= math.sqrt(inst.tau2) * (1 + 1e-12)


CASES = [
    ("maxcut K8", lambda: I.maxcut(8, *I.complete_graph(8)), 16.0),
    ("maxcut C5", lambda: I.maxcut(5, *I.cycle_graph(5)), 2.5 * (1 + math.cos(math.pi / 5))),
    ("maxcut C7", lambda: I.maxcut(7, *I.cycle_graph(7)), 3.5 * (1 + math.cos(math.pi / 7))),
    ("maxcut C6", lambda: I.maxcut(6, *I.cycle_graph(6)), 6.0),
    ("maxcut torus 4x4", lambda: I.maxcut(16, *I.torus_graph(4, 4)), 32.0),
    ("maxcut weighted bipartite", lambda: _weighted_bipartite(), None),
    ("theta C5", lambda: I.theta(5, *I.cycle_graph(5)), math.sqrt(5.0)),
    ("theta C7", lambda: I.theta(7, *I.cycle_graph(7)),
     7 * math.cos(math.pi / 7) / (1 + math.cos(math.pi / 7))),
    ("theta K6", lambda: I.theta(6, *I.complete_graph(6)), 1.0),
    ("theta empty 6", lambda: I.theta(6, np.zeros(0, int), np.zeros(0, int)), 6.0),
    ("theta Q4", lambda: I.theta(16, *I.hypercube_graph(4)), 8.0),
    ("theta C5 no trace row", lambda: I.theta(5, *I.cycle_graph(5), trace_row=False), math.sqrt(5.0)),
]


def _weighted_bipartite():
    rng = np.random.default_rng(3)
    a, b = 5, 6
    ei, ej, w = [], [], []
    for i in range(a):
        for j in range(b):
            if rng.random() < 0.6:
                ei.append(i)
                ej.append(a + j)
                w.append(rng.uniform(0.5, 2.0))
    inst = I.maxcut(a + b, ei, ej, w)
    inst.meta["ref"] = float(np.sum(w))
    return inst


@pytest.mark.parametrize("name,make,ref", CASES, ids=[c[0] for c in CASES])
def test_closed_form_values(name, make, ref):
    inst = make()
    if ref is None:
        ref = inst.meta["ref"]
    res = solve(inst)
    assert abs(res.user_value - ref) <= 1e-5 * abs(ref), (res.user_value, ref)
    check_certificate(inst, res)


def test_empty_graph_theta_solution_is_unique():
    # theta of the empty graph: X = 11^T / n is the unique optimum
    n = 6
    inst = I.theta(n, np.zeros(0, int), np.zeros(0, int))
    res = solve(inst)
    X = res.U @ res.U.T
    np.testing.assert_allclose(X, np.ones((n, n)) / n, atol=1e-4)


def test_matrix_completion_recovers_nuclear_norm():
    inst = I.completion(10, 12, 2, 100, seed=5)
    res = solve(inst)
    nuc = inst.meta["nuclear_norm"]
    assert abs(res.user_value - nuc) <= 1e-4 * nuc
    X = res.U @ res.U.T
    M = inst.meta["G"] @ inst.meta["H"].T
    assert np.linalg.norm(X[:10, 10:] - M) <= 1e-3 * np.linalg.norm(M)
    check_certificate(inst, res)


def test_weak_duality_and_gap():
    inst = I.maxcut(12, *I.er_graph(12, 0.5, 9))
    res = solve(inst)
    # dval <= P* <= pval up to the tolerance; the closed form is unknown here,
    # so check the pair against each other and against a dense eigenvalue
    assert res.dval <= res.pval + 1e-6 * (1 + abs(res.pval))
    assert abs(res.pval - res.dval) <= 2e-7 * (1 + abs(res.pval) + abs(res.dval))
    check_certificate(inst, res)


def test_aipp_output_invariants():
    # ADAP-AIPP returns R in grad g(W) + N_B(W), |R| <= rho, g(W) <= g(W0)
    inst = I.maxcut(20, *I.er_graph(20, 0.3, 2))
    rng = np.random.default_rng(1)
    U0 = O.project_ball(rng.standard_normal((20, 3)), math.sqrt(inst.tau2))
    p = rng.standard_normal(inst.m) * 0.1
    beta = 2.0
    cnt = O.Counters()
    sub = O._Subproblem(inst, p, beta, cnt)
    st = O.AippState(lam=1.0)
    rho = 1e-4
    tau = math.sqrt(inst.tau2)
    W, R = O.adap_aipp(sub, U0, rho, st, O.Options(), tau)
    assert np.linalg.norm(R) <= rho
    assert O.al_value(inst, W, p, beta) <= O.al_value(inst, U0, p, beta)
    grad = 2.0 * O.al_grad(inst, W, p, beta).W
    N = R - grad
    nrmW = np.linalg.norm(W)
    assert nrmW <= tau * (1 + 1e-12)
    if nrmW < tau * (1 - 1e-9):
        assert np.linalg.norm(N) <= 1e-8 * (1 + np.linalg.norm(grad))
    else:
        c = float(np.sum(N * W)) / nrmW ** 2
        assert c >= -1e-8
        assert np.linalg.norm(N - c * W) <= 1e-8 * (1 + np.linalg.norm(grad))


def test_rank_trim_keeps_leading_subspace():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((30, 6)) @ np.diag([5, 4, 3, 2, 1e-3, 1e-4])
    Yt = O.trim_rank(Y, 4)
    X, Xt = Y @ Y.T, Yt @ Yt.T
    assert Yt.shape == (30, 4)
    assert np.linalg.norm(X - Xt) <= 1e-2 * np.linalg.norm(X)


def test_kkt_measures_at_a_closed_form_optimum():
    # For a bipartite graph with unit weights and C = -L/4 an exact optimal
    # pair is known: X = v v^T with v the +-1 two-colouring (v_i v_j = -1 on
    # every edge, so C.X = -|E|) and multipliers p_i = deg_i / 2, for which
    # S = C + Diag(p) = (D + A)/4 is the signless Laplacian over 4, psd with
    # v itself as null vector ((A v)_i = -deg_i v_i), and -b^T p = -|E|.
    N = 6
    inst = I.maxcut_torus(N, "unit")
    n = inst.n
    ei, ej = I.torus_graph(N, N)
    colour = np.full(n, -1)
    colour[0] = 0
    adj = [[] for _ in range(n)]
    for a, b in zip(ei, ej):
        adj[a].append(b)
        adj[b].append(a)
    stack = [0]
    while stack:
        i = stack.pop()
        for j in adj[i]:
            if colour[j] < 0:
                colour[j] = 1 - colour[i]
                stack.append(j)
    assert all(colour[a] != colour[b] for a, b in zip(ei, ej))  # bipartite
    v = np.where(colour == 0, 1.0, -1.0)
    U = v[:, None]
    deg = np.bincount(np.concatenate([ei, ej]), minlength=n).astype(float)
    p = deg / 2.0
    E = float(len(ei))
    S = dense_C(inst) + np.diag(p)
    lam = float(np.linalg.eigvalsh(S)[0])
    assert abs(lam) <= 1e-12
    cn = O.c_norm1(inst)
    assert cn == pytest.approx(2.0)  # |C_ii| + sum_j |C_ij| = 1 + 4 / 4
    pval, dval, rp, rg, rd = O.kkt_measures(inst, U, p, 0.0, lam, cn)
    assert pval == pytest.approx(-E, rel=1e-15) and dval == pytest.approx(-E, rel=1e-15)
    assert rp == 0.0 and rg <= 1e-15 and rd <= 1e-12
    # moving p up keeps S psd but opens a duality gap of 0.1 n
    pval, dval, rp, rg, rd = O.kkt_measures(inst, U, p + 0.1, 0.0, lam + 0.1, cn)
    assert rg == pytest.approx(0.1 * n / (1 + 2 * E + 0.1 * n), rel=1e-12) and rd == 0.0
    # moving p down makes S indefinite by 0.1: dual infeasibility 0.1 / (1 + |C|_1)
    pval, dval, rp, rg, rd = O.kkt_measures(inst, U, p - 0.1, 0.0, lam - 0.1, cn)
    assert rd == pytest.approx(0.1 / (1 + cn), rel=1e-10)
    # shrinking U breaks diag(X) = 1 by 0.19 on every row
    pval, dval, rp, rg, rd = O.kkt_measures(inst, 0.9 * U, p, 0.0, lam, cn)
    assert rp == pytest.approx(0.19 * math.sqrt(n) / (1 + n), rel=1e-12)


def test_adap_fista_on_a_quadratic_with_a_closed_form_prox():
    # p = 0 and beta = 0 leave g(U) = C.UU^T; with C = c I (no edges, C_I = c)
    # psi(U) = lam c |U|^2 + 1/2 |U - U0|^2 has the minimiser U0 / (1 + 2 lam c)
    # and Hessian H = 1 + 2 lam c.  ADAP-FISTA (Appendix A.1) started at U0
    # must stop at step 5 with |(L - mu)(x~ - y)| <= sigma |y - U0|; the
    # step-2 test forces L >= 2 H / (1 - chi), which bounds |y - U*| by
    # sigma |y - U0|.  With the ball inactive, V = grad psi(y) exactly.
    n, r, c, lam = 50, 3, 0.5, 0.7
    inst = I.maxcut(n, np.zeros(0, int), np.zeros(0, int))
    inst.C_I = c
    rng = np.random.default_rng(21)
    U0 = 0.3 * rng.standard_normal((n, r))
    opt = O.Options()
    sub = O._Subproblem(inst, np.zeros(n), 0.0, O.Counters())
    status, y, L, V, dg = O.adap_fista(sub, lam, U0, 0.5, 1.0, opt, math.sqrt(inst.tau2))
    assert status == "success"
    H = 1.0 + 2.0 * lam * c
    Ustar = U0 / H
    assert L >= 2.0 * H / (1.0 - opt.chi)
    assert np.linalg.norm(y - Ustar) <= opt.sigma * np.linalg.norm(y - U0)
    grad_psi = H * y - U0
    assert np.linalg.norm(V - grad_psi) <= 1e-12 * np.linalg.norm(U0)
    dg0 = dg[0]
    assert dg0 == pytest.approx(c * (np.sum(y * y) - np.sum(U0 * U0)), rel=1e-12)

    def psi(U):
        return lam * c * float(np.sum(U * U)) + 0.5 * float(np.sum((U - U0) ** 2))
    assert psi(y) < psi(U0)


def test_rank_trim_is_the_best_low_rank_approximation():
    # Eckart-Young: Y Q_k (Q_k the top-k eigenvectors of Y^T Y) gives
    # X_k = Y Q_k Q_k^T Y^T, the best rank-k approximation of X = Y Y^T, whose
    # Frobenius error is sqrt(sum_{i>k} s_i^4) with s the singular values of
    # Y (eigenvalues of X are s_i^2); the remainder X - X_k is psd
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((40, 7)) @ np.diag([3.0, 2.5, 2.0, 1.5, 1.0, 0.5, 0.25])
    s = np.linalg.svd(Y, compute_uv=False)
    X = Y @ Y.T
    for k in (1, 3, 6):
        Yk = O.trim_rank(Y, k)
        assert Yk.shape == (40, k)
        Xk = Yk @ Yk.T
        assert np.linalg.norm(X - Xk) == pytest.approx(math.sqrt(np.sum(s[k:] ** 4)), rel=1e-10)
        assert np.linalg.eigvalsh(X - Xk)[0] >= -1e-10 * s[0] ** 2


def test_penalty_cap_scales_with_the_cost_norm():
    # Reading: beta_t doubles up to beta_max (1 + ||C||_1).  On theta(Q_6)
    # (||C||_1 = n = 64) U ~ 1 stays a fixed point of the subproblem until
    # the edge multipliers reach about n/d, so beta keeps doubling; with
    # beta_max = 1 it must stop at exactly 1 + 64 = 65 and never pass it
    inst = I.theta(64, *I.hypercube_graph(6))
    assert O.c_norm1(inst) == 64.0
    res = O.hallar_solve(inst, I.initial_factor(inst.n, 2, 7),
                         opt=O.Options(tol=1e-7, beta_max=1.0, max_outer=14))
    betas = [h["beta"] for h in res.history]
    assert max(betas) == 65.0
    assert betas[:8] == sorted(betas[:8])
    assert all(b == 65.0 or b == 2.0 ** round(math.log2(b)) for b in betas)


def test_lambda_restart_option_reaches_the_closed_form():
    # options.lambda_kappa > 0: every ADAP-AIPP call starts at lambda_kappa /
    # beta_t instead of the carried lambda; a schedule choice, so the solve
    # must still reach theta(C_9) = 9 cos(pi/9) / (1 + cos(pi/9))
    inst = I.theta(9, *I.cycle_graph(9))
    ref = 9 * math.cos(math.pi / 9) / (1 + math.cos(math.pi / 9))
    res = O.hallar_solve(inst, I.initial_factor(9, 2, 7), opt=O.Options(tol=1e-7, lambda_kappa=100.0))
    assert res.converged
    assert abs(inst.sense * res.pval - ref) <= 1e-6 * ref
