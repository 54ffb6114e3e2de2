"""Pins of the oracle's phase retrieval SDP (Section 5.4, eq. phase
retrieval SDP): min tr X s.t. <a_i a_i^H, X> = b_i, X Hermitian psd.

* The FFT operators against a brute-force DFT built here from the textbook
  sum a^H x = sum_t e^{-2 pi i j t / n} d_t x_t: the measurement map, the
  adjoint product, and the signal reproducing b exactly.
* The adjoint identity Re tr(U^H A*(p) U) = p . A(UU^H).
* The real embedding (X psd iff [[Re X, -Im X], [Im X, Re X]] psd) in HSLR
  form: the same values and adjoint product as the complex operators.
* Closed form: with 12 coded diffraction masks the relaxation is exact, so
  the optimum is tr X = |x|^2 with X = x x^H; the oracle's solve of the
  embedded problem meets both.
"""
import math

import numpy as np
import pytest

from oracle import hallar_oracle as O
from paper_2505_13719_b300 import instances as I


def dft_rows(inst):
    n = inst.n
    rows = []
    for d in inst.masks:
        for j in range(n):
            rows.append([np.exp(-2j * math.pi * j * t / n) * d[t] for t in range(n)])
    return np.array(rows)


def test_phase_operators_match_the_dft_sum():
    inst = I.phase_retrieval(6, 4, seed=3)
    Ah = dft_rows(inst)
    rng = np.random.default_rng(1)
    U = rng.standard_normal((6, 2)) + 1j * rng.standard_normal((6, 2))
    np.testing.assert_allclose(O.phase_map(inst, U), np.sum(np.abs(Ah @ U) ** 2, axis=1),
                               rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(O.phase_vectors(inst), Ah, rtol=1e-12, atol=1e-12)
    p = rng.standard_normal(inst.m)
    M = (Ah.conj().T * p) @ Ah  # sum_i p_i a_i a_i^H
    np.testing.assert_allclose(O.phase_adjoint(inst, p, U), M @ U, rtol=1e-12, atol=1e-11)
    x = inst.meta["signal"]
    np.testing.assert_allclose(O.phase_map(inst, x), inst.b, rtol=1e-13, atol=1e-13)
    lhs = float(np.real(np.vdot(U, O.phase_adjoint(inst, p, U))))
    assert abs(lhs - float(p @ O.phase_map(inst, U))) <= 1e-11 * (1 + abs(lhs))


def test_real_embedding_matches_the_complex_operators():
    inst = I.phase_retrieval(8, 3, seed=4)
    R = O.phase_to_hslr(inst)
    rng = np.random.default_rng(2)
    U = rng.standard_normal((8, 2)) + 1j * rng.standard_normal((8, 2))
    UR = O.embed_factor(U)
    T = O.eval_A_tilde(R, UR)
    assert T[0] == pytest.approx(float(np.vdot(U, U).real), rel=1e-13)
    np.testing.assert_allclose(T[1:], O.phase_map(inst, U), rtol=1e-12, atol=1e-12)
    p = rng.standard_normal(inst.m)
    W = O.adjoint_apply(R, np.concatenate([[0.3], p]), UR)
    ref = 0.5 * O.embed_factor(0.3 * U + O.phase_adjoint(inst, p, U))
    np.testing.assert_allclose(W, ref, rtol=1e-12, atol=1e-11)
    assert R.tau2 == pytest.approx(2.0 * inst.tau2)


@pytest.mark.parametrize("n,seed", [(8, 1), (16, 2)])
def test_phase_retrieval_recovers_the_signal(n, seed):
    inst = I.phase_retrieval(n, 12, seed=seed)
    R = O.phase_to_hslr(inst)
    res = O.hallar_solve(R, I.initial_factor(2 * n, 1, 3), opt=O.Options(tol=1e-7))
    assert res.converged
    x = inst.meta["signal"]
    nx2 = float(np.vdot(x, x).real)
    assert abs(res.pval - nx2) <= 1e-6 * nx2
    XR = res.U @ res.U.T
    X = 0.5 * ((XR[:n, :n] + XR[n:, n:]) + 1j * (XR[n:, :n] - XR[:n, n:]))
    assert np.linalg.norm(X - np.outer(x, x.conj())) <= 1e-5 * nx2
