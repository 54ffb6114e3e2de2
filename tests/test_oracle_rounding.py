"""Pins of the oracle's floating-point reading of the step-2 tests.

Not in the paper: the oracle's ADAP-FISTA step-2 test and ADAP-AIPP step-2
inequality (Appendix A.1 and A) accept a violation of at most
16 u lam sum|terms of g| (u = 2^-53), and ADAP-AIPP stops when a prox step
leaves W unchanged ("stalled").  These tests recheck every accepted step on
tiny instances in exact rational arithmetic (fractions.Fraction of the
float iterates), with g, its gradient and the prox terms written here from
their definitions (eq. AL function, eq. Grad U Space; the families' A_l),
independently of the oracle's operator code:

* an accepted step never violates the exact inequality by more than the
  allowance plus the rounding of the test's own float evaluation;
* "stalled" fires only when W equals the previous iterate bit for bit, and
  every bit-identical prox step is reported as stalled.
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest

from oracle import hallar_oracle as O
from paper_2505_13719_b300 import instances as I

U_RND = 2.0 ** -53


class Exact:
    """g(U) = C.UU^T + p^T r + beta/2 |r|^2, r = A(UU^T) - b, and
    grad g = 2 (C + A*(p + beta r)) U, in rational arithmetic from the
    instance arrays (full CSR of C, implicit C_J 11^T + C_I I; diag family
    A_i = e_i e_i^T; edge family A_l = (e_i e_j^T + e_j e_i^T)/2 plus the
    trace row A = I)."""

    def __init__(self, inst, p, beta):
        self.inst = inst
        self.n = inst.n
        self.p = [F(float(x)) for x in p]
        self.b = [F(float(x)) for x in inst.b]
        self.beta = F(float(beta))
        rp = inst.C_rowptr
        self.C = [(i, int(inst.C_col[e]), F(float(inst.C_val[e])))
                  for i in range(self.n) for e in range(rp[i], rp[i + 1])]
        self.CJ, self.CI = F(float(inst.C_J)), F(float(inst.C_I))
        if inst.family == "diag":
            self.pairs = None
        else:
            off = inst.n1 if inst.family == "observed" else 0
            self.pairs = [(int(i), int(j) + off) for i, j in zip(inst.cons_i, inst.cons_j)]

    @staticmethod
    def q(U):
        return [[F(float(x)) for x in row] for row in U]

    @staticmethod
    def dot(a, b):
        return sum((x * y for x, y in zip(a, b)), F(0))

    def Amap(self, U):
        if self.pairs is None:
            return [self.dot(U[i], U[i]) for i in range(self.n)]
        T = [self.dot(U[i], U[j]) for i, j in self.pairs]
        if self.inst.has_trace_row:
            T.append(sum((self.dot(U[i], U[i]) for i in range(self.n)), F(0)))
        return T

    def g(self, U):
        r_ = len(U[0])
        cval = sum((v * self.dot(U[a], U[b]) for a, b, v in self.C), F(0))
        colsum = [sum((U[i][k] for i in range(self.n)), F(0)) for k in range(r_)]
        cval += self.CJ * self.dot(colsum, colsum)
        cval += self.CI * sum((self.dot(U[i], U[i]) for i in range(self.n)), F(0))
        res = [t - bb for t, bb in zip(self.Amap(U), self.b)]
        return (cval + sum((pp * rr for pp, rr in zip(self.p, res)), F(0))
                + self.beta / 2 * sum((rr * rr for rr in res), F(0)))

    def grad(self, U):
        n, r_ = self.n, len(U[0])
        res = [t - bb for t, bb in zip(self.Amap(U), self.b)]
        ps = [pp + self.beta * rr for pp, rr in zip(self.p, res)]
        W = [[F(0)] * r_ for _ in range(n)]
        for a, b, v in self.C:
            for k in range(r_):
                W[a][k] += v * U[b][k]
        colsum = [sum((U[i][k] for i in range(n)), F(0)) for k in range(r_)]
        for i in range(n):
            for k in range(r_):
                W[i][k] += self.CJ * colsum[k] + self.CI * U[i][k]
        if self.pairs is None:
            for i in range(n):
                for k in range(r_):
                    W[i][k] += ps[i] * U[i][k]
        else:
            for l, (i, j) in enumerate(self.pairs):
                for k in range(r_):
                    W[i][k] += ps[l] / 2 * U[j][k]
                    W[j][k] += ps[l] / 2 * U[i][k]
            if self.inst.has_trace_row:
                for i in range(n):
                    for k in range(r_):
                        W[i][k] += ps[-1] * U[i][k]
        return [[2 * w for w in row] for row in W]


def sqnorm(A):
    return sum((x * x for row in A for x in row), F(0))


def inner(A, B):
    return sum((x * y for ra, rb in zip(A, B) for x, y in zip(ra, rb)), F(0))


def sub(A, B):
    return [[x - y for x, y in zip(ra, rb)] for ra, rb in zip(A, B)]


def run_aipp(inst, U0, p, beta, lam0, max_aipp, rho=1e-10):
    events = []
    cnt = O.Counters()
    sp = O._Subproblem(inst, p, beta, cnt, observer=lambda e, d: events.append((e, d)))
    opt = O.Options(max_aipp=max_aipp)
    W, _R = O.adap_aipp(sp, U0, rho, O.AippState(lam=lam0), opt, math.sqrt(inst.tau2))
    return events


def check_events(inst, p, beta, events, limit=None):
    ex = Exact(inst, p, beta)
    checked = 0
    for ev, d in events[:limit]:
        lam = F(float(d["lam"]))
        if ev == "fista_step2":
            xt, y, ctr = ex.q(d["xt"]), ex.q(d["y"]), ex.q(d["center"])
            L, chi = F(float(d["L"])), F(float(d["chi"]))
            dd = sub(y, xt)
            grad_psi = [[lam * gw + x - c for gw, x, c in zip(rg, rx, rc)]
                        for rg, rx, rc in zip(ex.grad(xt), xt, ctr)]
            psi_y = lam * ex.g(y) + sqnorm(sub(y, ctr)) / 2
            psi_x = lam * ex.g(xt) + sqnorm(sub(xt, ctr)) / 2
            lin = inner(grad_psi, dd) + (1 - chi) * L / 4 * sqnorm(dd)
            violation = (psi_y - psi_x) - lin
            # rounding of the float test itself: its terms, each to a few ulps
            own = (abs(float(inner(grad_psi, dd))) + float(L * sqnorm(dd))
                   + float(sqnorm(sub(y, ctr)) + sqnorm(sub(xt, ctr))))
        else:
            Wp, W, V = ex.q(d["Wprev"]), ex.q(d["W"]), ex.q(d["V"])
            D = sub(W, Wp)
            if d["stalled"]:
                assert np.array_equal(d["W"], d["Wprev"])
                continue
            assert not np.array_equal(d["W"], d["Wprev"])
            # step 2: lam g(W_prev) - [lam g(W) + |D|^2/2] >= <V, W_prev - W>
            violation = lam * (ex.g(W) - ex.g(Wp)) + sqnorm(D) / 2 - inner(V, D)
            own = abs(float(inner(V, D))) + float(sqnorm(D))
        slack = float(d["slack"])
        assert slack == 16.0 * U_RND * d["lam"] * d["mag"]
        bound = slack + 16.0 * U_RND * (d["lam"] * d["mag"] + own)
        assert float(violation) <= bound, (ev, float(violation), slack)
        checked += 1
    return checked


CASES = {
    "maxcut_C5": lambda: I.maxcut(5, *I.cycle_graph(5)),
    "maxcut_K4_weighted": lambda: I.maxcut(4, *I.complete_graph(4),
                                           w=np.array([1.0, -2.0, 0.5, 3.0, 1.5, -1.0])),
    "theta_C5_trace": lambda: I.theta(5, *I.cycle_graph(5)),
}


@pytest.mark.parametrize("lam0,pshift", [(1.0, 0.0), (256.0, 0.0), (1.0, -10.0)])
@pytest.mark.parametrize("name", sorted(CASES))
def test_accepted_steps_respect_the_exact_inequality(name, lam0, pshift):
    # lam0 = 256 starts far above the curvature of g, so ADAP-FISTA's step-2
    # test rejects trials and lam halves; multipliers shifted by -10 make g
    # strongly nonconvex, where ADAP-AIPP's step-2 inequality can reject a
    # FISTA success (theta on C5 has one such rejection)
    inst = CASES[name]()
    rng = np.random.default_rng(3)
    U0 = O.project_ball(rng.standard_normal((inst.n, 2)), math.sqrt(inst.tau2))
    p = rng.standard_normal(inst.m) * 0.5 + pshift
    events = run_aipp(inst, U0, p, 2.0, lam0, max_aipp=6)
    assert any(e == "fista_step2" for e, _ in events)
    assert any(e == "aipp_step2" for e, _ in events)
    assert check_events(inst, p, 2.0, events) > 0


def test_stalled_fires_exactly_on_a_bit_identical_prox_step():
    # W0 = 0 is a stationary point of g (its gradient 2 (C + A*(p')) 0 = 0):
    # the prox step returns 0 again, bit for bit, and ADAP-AIPP must stop there
    inst = I.maxcut(5, *I.cycle_graph(5))
    p = np.random.default_rng(0).standard_normal(inst.m)
    events = run_aipp(inst, np.zeros((5, 2)), p, 1.0, 1.0, max_aipp=5)
    aipp = [d for e, d in events if e == "aipp_step2"]
    assert len(aipp) == 1 and aipp[0]["stalled"]
    assert np.array_equal(aipp[0]["W"], np.zeros((5, 2)))
    # and from a generic start no accepted step is stalled unless identical
    rng = np.random.default_rng(9)
    U0 = O.project_ball(rng.standard_normal((5, 2)), math.sqrt(inst.tau2))
    for e, d in run_aipp(inst, U0, p, 1.0, 1.0, max_aipp=8):
        if e == "aipp_step2":
            assert d["stalled"] == np.array_equal(d["W"], d["Wprev"])


def test_allowance_constants():
    # the documented reading: 16 units of the FP64 roundoff
    assert O.ROUND_SLACK == 16.0 and O.UNIT_ROUNDOFF == 2.0 ** -53


def test_fista_at_the_prox_point_succeeds_within_rounding(monkeypatch):
    # theta(Q_6) at U ~ 1 (|U| = 1 = tau) with p = 0, beta = 1: the centre is
    # the prox point (the gradient is radial and the ball projection undoes
    # the step), so every ADAP-FISTA iterate equals x_0 up to rounding and
    # step 4's inequality compares rounding-level numbers.  Reading: such a
    # call succeeds with y = x_0 (to rounding); without the rounding
    # allowance this case's step 4 reports a failure that would halve
    # ADAP-AIPP's lambda
    inst = I.theta(64, *I.hypercube_graph(6))
    W0 = np.ones((64, 2)) / math.sqrt(128)

    def run():
        sub = O._Subproblem(inst, np.zeros(inst.m), 1.0, O.Counters())
        return O.adap_fista(sub, 1.0, W0, 0.5, 1.0, O.Options(), 1.0)

    st, y, L, V, dg = run()
    assert st == "success"
    assert np.linalg.norm(y - W0) <= O.ROUND_SLACK * O.UNIT_ROUNDOFF * np.linalg.norm(W0)
    monkeypatch.setattr(O, "ROUND_SLACK", 0.0)
    assert run()[0] == "failure"


def test_ball_projection_lands_on_the_sphere_to_a_few_ulps():
    # eq. dimensional ball: P_B(Z) = tau Z / |Z|_F outside the ball.  The
    # step-2 tests read the projected point's radial error times the radial
    # gradient (2n on the theta SDP), so the radius must be exact to a few
    # units of roundoff even for a large factor; checked with exact rational
    # arithmetic on |P_B(Z)|^2
    # the shape of theta(Q_17)'s iterates at the fixed point U ~ 1: many equal
    # entries, where a blocked dot product of the squares is off by 1e-14
    n = 1 << 17
    Z = np.full((n, 2), 0.7071 / math.sqrt(n)) * 1.31073e5
    Y = O.project_ball(Z, 1.0)
    r2 = sum(F(float(v)) ** 2 for v in Y.ravel())
    assert abs(float(r2 - 1)) <= 4 * O.UNIT_ROUNDOFF
    np.testing.assert_array_equal(O.project_ball(Y * 0.5, 1.0), Y * 0.5)
