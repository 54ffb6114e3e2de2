"""GPU parity of the AL value change g(Y) - g(X) and of the rank trim.

hallar_value_change runs the kernel that the ADAP-FISTA and ADAP-AIPP
step-2 tests use (eq. AL function; Appendix A and A.1) and is compared with
the oracle's al_value_change, which forms the same difference from the pair
products <D_a, Y_b> + <X_a, D_b> (D = Y - X).  FP64 handles match to 1e-12
and mixed handles to 1e-5 (against the oracle on the float-rounded X, Y, p
and r_X), both relative to the sum of the magnitudes of the terms of the
change.  hallar_trim_rank (the rank cap's Gram trim, not in the paper) is
compared with the oracle's trim_rank through the projector Y_k Y_k^T, which
is unique when the Gram eigenvalues are simple, and through the Gram
eigenvalues and the kept columns' Gram at a size spanning many CTAs.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hallar_oracle as O  # noqa: E402
from paper_2505_13719_b300 import instances as I  # noqa: E402
from tests.test_gpu_operators import FAM_IDS, FAMS  # noqa: E402
from tests.test_oracle_operators import random_instance  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13719_b300 import hallar
    return hallar


def change_scale(inst, X, Y, p, beta, rX):
    """Sum of the magnitudes of the terms of g(Y) - g(X): every pair product
    difference bounded by |D_a||Y_b| + |X_a||D_b|, weighted by the size of
    its coefficient (C entries, p_l + beta/2 (2 r_l + dT_l)); the scale of
    the rounding of the change, and of r_Y - r_X."""
    D = Y - X
    nD, nX, nY = (np.linalg.norm(A, axis=1) for A in (D, X, Y))
    ell, a, b, v = O.constraint_entries(inst)
    pair = np.abs(v) * (nD[a] * nY[b] + nX[a] * nD[b])
    Ml = np.bincount(ell, weights=pair, minlength=inst.m)
    dT = O.constraint_map(inst, Y) - O.constraint_map(inst, X)
    coef = np.abs(p) + 0.5 * beta * (2 * np.abs(rX) + np.abs(dT))
    ca, cb, cv = O.cost_entries(inst)
    cterm = float(np.sum(np.abs(cv) * (nD[ca] * nY[cb] + nX[ca] * nD[cb]))) if cv.size else 0.0
    sD, sS = np.abs(D.sum(0)), np.abs(Y.sum(0) + X.sum(0))
    cterm += abs(inst.C_J) * float(np.linalg.norm(sD) * np.linalg.norm(sS))
    cterm += abs(inst.C_I) * float(np.sum(nD * (nY + nX)))
    return cterm + float(coef @ Ml) + 1e-300, Ml


def run_change(H, inst, X, Y, p, beta, rX, prec, host=False, pass_rx=True):
    dt = np.float32 if prec else np.float64
    Xc = np.ascontiguousarray(X.astype(dt))
    Yc = np.ascontiguousarray(Y.astype(dt))
    r = X.shape[1]
    with H.create_from_instance(inst, prec) as hd:
        if host:
            rY = np.empty(inst.m)
            dg = H.hallar_value_change(hd.h, Xc, Yc, r, p, beta, rX if pass_rx else None, rY)
        else:
            rYd = torch.empty(inst.m, dtype=torch.float64, device="cuda")
            rXd = torch.from_numpy(rX).cuda() if pass_rx else None
            dg = H.hallar_value_change(hd.h, torch.from_numpy(Xc).cuda(),
                                       torch.from_numpy(Yc).cuda(), r, torch.from_numpy(p).cuda(),
                                       beta, rXd, rYd)
            torch.cuda.synchronize()
            rY = rYd.cpu().numpy()
    return dg, rY, Xc.astype(np.float64), Yc.astype(np.float64)


def check(inst, dg, rY, Xe, Ye, p, beta, rX, prec):
    # the oracle on what the kernel reads: float-rounded p and r_X in the mixed form
    pe = p.astype(np.float32).astype(np.float64) if prec else p
    rXe = rX.astype(np.float32).astype(np.float64) if prec else rX
    ref_dg, ref_rY = O.al_value_change(inst, Xe, Ye, pe, beta, rXe)
    scale, Ml = change_scale(inst, Xe, Ye, p, beta, rX)
    tol = TOL[prec]
    assert abs(dg - ref_dg) <= tol * scale, (dg, ref_dg, scale)
    rscale = np.linalg.norm(rX) + np.linalg.norm(Ml) + 1e-300
    assert np.linalg.norm(rY - ref_rY) <= tol * rscale


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("fam", FAMS, ids=FAM_IDS)
@pytest.mark.parametrize("r", [1, 3, 10, 32, 33, 64])
def test_value_change_parity(H, fam, r, prec):
    family, n1, trace, with_c, cj, ci = fam
    n = 1537  # ragged: not a multiple of any tile
    inst = random_instance(family, n, 300 + r, n1=n1, trace=trace, with_c=with_c, cj=cj, ci=ci)
    rng = np.random.default_rng(r + 7)
    X = rng.standard_normal((n, r)) / math.sqrt(r)
    # a small step (the regime of the step-2 tests) and a large one
    for step in (1e-3, 1.0):
        Y = X + step * rng.standard_normal((n, r)) / math.sqrt(r)
        p = rng.standard_normal(inst.m)
        beta = 1.3
        Xe = X.astype(np.float32).astype(np.float64) if prec else X
        rX = O.constraint_map(inst, Xe) - inst.b
        dg, rY, Xe, Ye = run_change(H, inst, X, Y, p, beta, rX, prec)
        check(inst, dg, rY, Xe, Ye, p, beta, rX, prec)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("fam", FAMS, ids=FAM_IDS)
def test_value_change_host_pointers_and_internal_rx(H, fam, prec):
    # host arrays, and r_X = NULL (the library evaluates it at X)
    family, n1, trace, with_c, cj, ci = fam
    inst = random_instance(family, 901, 17, n1=n1 if n1 == 0 else 300, trace=trace,
                           with_c=with_c, cj=cj, ci=ci)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((901, 6)) / math.sqrt(6)
    Y = X + 1e-2 * rng.standard_normal((901, 6))
    p = rng.standard_normal(inst.m)
    Xe = X.astype(np.float32).astype(np.float64) if prec else X
    rX = O.constraint_map(inst, Xe) - inst.b
    for pass_rx in (True, False):
        dg, rY, Xe, Ye = run_change(H, inst, X, Y, p, 0.7, rX, prec, host=True, pass_rx=pass_rx)
        check(inst, dg, rY, Xe, Ye, p, 0.7, rX, prec)


def test_value_change_equal_factors_is_zero(H):
    # Y = X: every difference is exactly zero, so dg = 0 and r_Y = r_X exactly
    inst = random_instance("edge", 700, 3, trace=True, with_c=True, cj=-1.0, ci=0.3)
    X = np.random.default_rng(1).standard_normal((700, 5))
    rX = O.constraint_map(inst, X) - inst.b
    p = np.random.default_rng(2).standard_normal(inst.m)
    for prec in (0, 1):
        rXe = rX.astype(np.float32).astype(np.float64) if prec else rX
        dg, rY, _, _ = run_change(H, inst, X, X, p, 2.0, rXe, prec)
        assert dg == 0.0
        assert np.array_equal(rY, rXe)


@pytest.mark.parametrize("prec", [0, 1])
def test_value_change_full_size_torus(H, prec):
    # the Max-Cut torus at its full size (n = 1e6), r = 10 as in the solve
    inst = I.maxcut_torus(1000, "pm1", seed=2)
    rng = np.random.default_rng(8)
    X = rng.standard_normal((inst.n, 10)) / math.sqrt(10)
    Y = X + 1e-3 * rng.standard_normal((inst.n, 10))
    p = rng.standard_normal(inst.m)
    Xe = X.astype(np.float32).astype(np.float64) if prec else X
    rX = O.constraint_map(inst, Xe) - inst.b
    dg, rY, Xe, Ye = run_change(H, inst, X, Y, p, 2.0, rX, prec)
    check(inst, dg, rY, Xe, Ye, p, 2.0, rX, prec)


# ---------------------------------------------------------------------------
# the rank trim
# ---------------------------------------------------------------------------
# The mixed form's Gram runs on the tensor cores: TF32 operand splitting
# (H + L, the L^T L product dropped: relative 2^-22) and FP32 accumulation
# over 1024-row slices, the slices summed in FP64.  Its error is taken as at
# most GRAM_TC_REL * tr(Y^T Y) in norm (a slice of 1024 FP32 additions rounds
# each entry by about sqrt(1024) * 2^-24 relative to its absolute terms);
# eigenvalues then move by at most that much (Weyl) and the kept directions
# by that over the eigengap (Davis-Kahan).
GRAM_TC_REL = 1e-5


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n,r,k", [(777, 3, 1), (777, 12, 5), (777, 33, 32), (777, 90, 89),
                                   (300_000, 33, 32)])
def test_trim_rank_parity(H, n, r, k, prec):
    inst = I.maxcut(n, *I.er_graph(n, min(0.01, 8.0 / n), 2))
    rng = np.random.default_rng(r)
    # distinct column scales: simple, well separated Gram eigenvalues
    Y = rng.standard_normal((n, r)) * np.linspace(2.0, 0.2, r)
    dt = np.float32 if prec else np.float64
    Yc = np.ascontiguousarray(Y.astype(dt))
    Ye = Yc.astype(np.float64)
    out = np.empty((n, k), dtype=dt)
    eigs = np.empty(r)
    with H.create_from_instance(inst, prec) as hd:
        H.hallar_trim_rank(hd.h, Yc, r, k, out, eigs)
    ref = O.trim_rank(Ye, k)
    w_ref = np.sort(np.linalg.eigvalsh(Ye.T @ Ye))[::-1]
    tol = TOL[prec]
    dG = GRAM_TC_REL * w_ref.sum() if prec else 0.0
    gap = w_ref[k - 1] - w_ref[k] if k < r else np.inf
    assert np.all(np.abs(eigs - w_ref) <= tol * w_ref[0] * 10 + dG)
    rot = 4.0 * w_ref[0] * dG / gap
    if n <= 5000:  # the n x n projectors
        Pk = out.astype(np.float64) @ out.astype(np.float64).T
        Pr = ref @ ref.T
        assert np.linalg.norm(Pk - Pr) <= 10 * tol * np.linalg.norm(Pr) + rot
    # the columns are orthogonal with squared norms the k leading eigenvalues
    G = out.astype(np.float64).T @ out.astype(np.float64)
    assert np.linalg.norm(G - np.diag(w_ref[:k])) <= 10 * tol * w_ref[0] + rot


def test_trim_rank_rejects_bad_sizes(H):
    inst = I.maxcut(10, *I.cycle_graph(10))
    Y = np.zeros((10, 4))
    out = np.zeros((10, 5))
    with H.create_from_instance(inst) as hd:
        for r, k in ((4, 5), (4, 0), (91, 3)):
            with pytest.raises(H.HallarError):
                H.hallar_trim_rank(hd.h, Y, r, k, out)


@pytest.mark.parametrize("prec", [0, 1])
def test_solve_with_forced_trims(H, prec):
    # the +-1 torus needs a rank far above 2: with r_cap = 2 every
    # Frank-Wolfe step that appends a column is followed by a trim
    inst = I.maxcut_torus(8, "pm1", seed=2)
    dt = np.float32 if prec else np.float64
    U0 = I.initial_factor(inst.n, 2, 3).astype(dt)
    with H.create_from_instance(inst, prec, r_cap=2, max_outer=8, time_limit_s=30.0) as hd:
        st, res = H.hallar_solve(hd.h, U0, 2)
        rank = H.hallar_get_solution(hd.h)
        U = np.empty((inst.n, rank), dtype=dt)
        H.hallar_get_solution(hd.h, U, rank)
    assert res.trims > 0 and res.rank <= 2 and rank <= 2
    assert np.linalg.norm(U.astype(np.float64)) <= math.sqrt(inst.tau2) * (1 + 1e-6)
    assert np.all(np.isfinite(U))
