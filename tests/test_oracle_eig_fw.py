"""Pins of the oracle's eigensolver and Frank-Wolfe step.

Lanczos is checked against dense symmetric eigendecomposition and against
closed-form spectra: the unit-weight N x N torus Laplacian has eigenvalues
(2 - 2cos(2 pi a/N)) + (2 - 2cos(2 pi b/N)), so for even N the largest is 8
and lambda_min(-L/4 + c I) = c - 2; the hypercube Q_d Laplacian has
eigenvalues 2k, k = 0..d, so lambda_min(-L/4 + c I) = c - d/2.
The Frank-Wolfe step (eqs. FW stepsize, tilde Y) is checked as the exact
line search of L_beta along the segment to tau^2 yy^T (Section 2 remark).
"""
import math

import numpy as np
import pytest

from oracle import hallar_oracle as O
from paper_2505_13719_b300 import instances as I
from tests.test_oracle_operators import dense_As, dense_C, random_instance


@pytest.mark.parametrize("fam,n,n1", [("diag", 60, 0), ("edge", 80, 0), ("observed", 70, 30)])
def test_lanczos_matches_dense_eigh(fam, n, n1):
    inst = random_instance(fam, n, 21, n1=n1, trace=True, with_c=True, cj=-0.3, ci=0.1)
    rng = np.random.default_rng(2)
    ps = rng.standard_normal(inst.m)
    G = dense_C(inst) + sum(q * A for q, A in zip(ps, dense_As(inst)))
    w, V = np.linalg.eigh(G)
    er = O.min_eig(inst, ps, tol=1e-10, seed=3, kmax=n)
    assert er.converged
    assert abs(er.lam - w[0]) <= 1e-9 * max(1.0, abs(w[0]))
    Gv = G @ er.v
    assert np.linalg.norm(Gv - er.lam * er.v) <= 1e-8
    if w[1] - w[0] > 1e-6:
        assert abs(abs(float(er.v @ V[:, 0])) - 1.0) <= 1e-8


@pytest.mark.parametrize("N", [8, 16, 32])
def test_lanczos_torus_closed_form(N):
    ei, ej = I.torus_graph(N, N)
    inst = I.maxcut(N * N, ei, ej)
    c = 0.37
    # G = C + diag(p') with C = -L/4 (diagonal included), so p' = c gives
    # G = -L/4 + c I
    ps = np.full(inst.n, c)
    er = O.min_eig(inst, ps, tol=1e-9, seed=1, kmax=300)
    assert er.converged
    assert abs(er.lam - (c - 2.0)) <= 1e-8


@pytest.mark.parametrize("d", [3, 5, 7])
def test_lanczos_hypercube_closed_form(d):
    ei, ej = I.hypercube_graph(d)
    inst = I.maxcut(1 << d, ei, ej)
    c = -0.2
    er = O.min_eig(inst, np.full(inst.n, c), tol=1e-10, seed=4, kmax=200)
    assert er.converged
    assert abs(er.lam - (c - d / 2.0)) <= 1e-9


def test_splitmix_matches_the_published_output_words():
    # SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) from state 0 produces
    # the 64-bit words e220a8397b1dcdaf, 6e789e6aa1b965f4, 06c45d188009454f
    # (the reference sequence of the published generator); the oracle's
    # values are 2 (w >> 11) 2^-53 - 1 of those words
    words = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    want = np.array([2.0 * (w >> 11) / 2.0 ** 53 - 1.0 for w in words])
    assert np.array_equal(O.splitmix64_uniform(0, 3), want)


def test_splitmix_uniform_range_and_determinism():
    a = O.splitmix64_uniform(42, 100000)
    b = O.splitmix64_uniform(42, 100000)
    assert np.array_equal(a, b)
    assert a.min() >= -1.0 and a.max() < 1.0
    assert abs(a.mean()) < 0.01 and abs(a.var() - 1.0 / 3.0) < 0.01
    assert not np.array_equal(a, O.splitmix64_uniform(43, 100000))


def _L_dense(inst, X, p, beta):
    C = dense_C(inst)
    As = dense_As(inst)
    r = np.array([np.sum(A * X) for A in As]) - inst.b
    return np.sum(C * X) + p @ r + 0.5 * beta * r @ r


@pytest.mark.parametrize("fam", ["diag", "edge"])
def test_fw_step_is_exact_line_search(fam):
    inst = random_instance(fam, 15, 31, trace=True, with_c=True)
    rng = np.random.default_rng(8)
    Y = rng.standard_normal((15, 3))
    Y *= math.sqrt(inst.tau2) * 0.8 / np.linalg.norm(Y)
    p = rng.standard_normal(inst.m) - 3.0  # shift G so that it has a negative eigenvalue
    beta = 2.0
    gr = O.al_grad(inst, Y, p, beta)
    G = dense_C(inst) + sum(q * A for q, A in zip(gr.pshift, dense_As(inst)))
    w, V = np.linalg.eigh(G)
    theta = max(-w[0], 0.0)
    assert theta > 0.0
    y = V[:, 0]
    gap = float(np.sum(gr.W * Y)) + inst.tau2 * theta
    Yt, alpha = O.fw_step(inst, Y, y, theta, gap, beta, inst.tau2)
    X0 = Y @ Y.T
    S = inst.tau2 * np.outer(y, y)
    Xa = (1 - alpha) * X0 + alpha * S
    # the new factor represents the Frank-Wolfe iterate
    np.testing.assert_allclose(Yt @ Yt.T, Xa, rtol=1e-10, atol=1e-10)
    f = lambda a: _L_dense(inst, (1 - a) * X0 + a * S, p, beta)
    fa = f(alpha)
    for da in (1e-3, 1e-2):
        if alpha + da <= 1.0:
            assert fa <= f(alpha + da) + 1e-9
        if alpha - da >= 0.0:
            assert fa <= f(alpha - da) + 1e-9
    # the derivative at 0 is minus the Frank-Wolfe gap (Section 2 remark)
    h = 1e-6
    d0 = (f(h) - f(0.0)) / h
    assert abs(d0 + gap) <= 1e-3 * abs(gap)
