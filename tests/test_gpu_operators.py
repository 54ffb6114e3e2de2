"""GPU parity of the operator entry points against the FP64 oracle.

hallar_eval_A, hallar_grad and hallar_min_eig are called through the C ABI
(ctypes) on seeded inputs and compared element by element with the oracle:
FP64 handles to 1e-12 (normwise relative; scalars with cancellation relative
to the sum of the magnitudes of their terms), MIXED handles to 1e-5 against
the oracle run on the same U rounded to float32.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hallar_oracle as O  # noqa: E402
from paper_2505_13719_b300 import instances as I  # noqa: E402
from tests.test_oracle_operators import random_instance  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13719_b300 import hallar
    return hallar


def nrel(a, b):
    d = np.linalg.norm(np.asarray(a, dtype=np.float64) - b)
    s = np.linalg.norm(b)
    return d / s if s > 0 else d


def scalar_scale(inst, U, p, beta):
    """Sum of the magnitudes of the terms of g(U): the scale of its rounding."""
    r = O.constraint_map(inst, U) - inst.b
    a, b, v = O.cost_entries(inst)
    cterm = float(np.sum(np.abs(v) * np.abs(np.einsum("kr,kr->k", U[a], U[b])))) if v.size else 0.0
    cterm += abs(inst.C_J) * float(np.sum(np.abs(U).sum(0) ** 2)) + abs(inst.C_I) * float(np.sum(U * U))
    return cterm + float(np.abs(p * r).sum()) + 0.5 * beta * float(r @ r) + 1.0


def run_grad(H, inst, U, p, beta, prec, host=False):
    dt = np.float32 if prec == H.HALLAR_MIXED else np.float64
    Uc = np.ascontiguousarray(U.astype(dt))
    with H.create_from_instance(inst, prec) as hd:
        if host:
            W = np.empty_like(Uc)
            r = np.empty(inst.m)
            g = H.hallar_grad(hd.h, Uc, U.shape[1], p, beta, W, r)
            return g, W.astype(np.float64), r, Uc.astype(np.float64)
        Ud = torch.from_numpy(Uc).cuda()
        Wd = torch.empty_like(Ud)
        pd = torch.from_numpy(p).cuda()
        rd = torch.empty(inst.m, dtype=torch.float64, device="cuda")
        g = H.hallar_grad(hd.h, Ud, U.shape[1], pd, beta, Wd, rd)
        torch.cuda.synchronize()
        return g, Wd.cpu().numpy().astype(np.float64), rd.cpu().numpy(), Uc.astype(np.float64)


FAMS = [
    ("diag", 0, False, True, 0.0, 0.0),
    ("diag", 0, False, True, -0.5, 0.25),
    ("edge", 0, True, False, -1.0, 0.0),
    ("edge", 0, False, True, 0.3, -0.1),
    ("edge", 0, True, True, -1.0, 0.5),
    ("observed", 400, False, False, 0.0, 0.5),
]
FAM_IDS = [f"{f[0]}-cj{f[4]}-trace{int(f[2])}-c{int(f[3])}" for f in FAMS]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("fam", FAMS, ids=FAM_IDS)
@pytest.mark.parametrize("r", [1, 2, 3, 7, 10, 32, 33, 64])
def test_grad_parity(H, fam, r, prec):
    family, n1, trace, with_c, cj, ci = fam
    n = 1537  # ragged: not a multiple of any tile
    inst = random_instance(family, n, 100 + r, n1=n1, trace=trace, with_c=with_c, cj=cj, ci=ci)
    rng = np.random.default_rng(r)
    U = rng.standard_normal((n, r)) / math.sqrt(r)
    p = rng.standard_normal(inst.m)
    beta = 1.7
    g, W, res, Ueff = run_grad(H, inst, U, p, beta, prec)
    ref = O.al_grad(inst, Ueff, p, beta)
    tol = TOL[prec]
    assert nrel(W, ref.W) <= tol
    # residuals r = A(UU^T) - b: error relative to the scale of A(UU^T)
    assert np.linalg.norm(res - ref.resid) <= tol * (np.linalg.norm(ref.T[1:]) + 1e-300)
    assert abs(g - ref.g) <= tol * scalar_scale(inst, Ueff, p, beta)


@pytest.mark.parametrize("prec", [0, 1])
def test_grad_host_pointers(H, prec):
    inst = random_instance("edge", 900, 5, trace=True, with_c=True, cj=-1.0, ci=0.2)
    rng = np.random.default_rng(1)
    U = rng.standard_normal((900, 5))
    p = rng.standard_normal(inst.m)
    g, W, res, Ueff = run_grad(H, inst, U, p, 0.8, prec, host=True)
    ref = O.al_grad(inst, Ueff, p, 0.8)
    assert nrel(W, ref.W) <= TOL[prec]
    assert np.linalg.norm(res - ref.resid) <= TOL[prec] * np.linalg.norm(ref.T[1:])


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("fam", FAMS, ids=FAM_IDS)
def test_eval_A_parity(H, fam, prec):
    family, n1, trace, with_c, cj, ci = fam
    inst = random_instance(family, 1201, 7, n1=n1, trace=trace, with_c=with_c, cj=cj, ci=ci)
    U = np.random.default_rng(3).standard_normal((1201, 6))
    dt = np.float32 if prec else np.float64
    with H.create_from_instance(inst, prec) as hd:
        Ud = torch.from_numpy(U.astype(dt)).cuda()
        Td = torch.empty(inst.m + 1, dtype=torch.float64, device="cuda")
        H.hallar_eval_A(hd.h, Ud, 6, Td)
        T = Td.cpu().numpy()
    Ueff = U.astype(dt).astype(np.float64)
    ref = O.eval_A_tilde(inst, Ueff)
    assert nrel(T[1:], ref[1:]) <= TOL[prec]
    assert abs(T[0] - ref[0]) <= TOL[prec] * scalar_scale(inst, Ueff, np.zeros(inst.m), 0.0)


def test_full_size_torus_gradient(H):
    # the Max-Cut torus at its full size (n = 1e6, r = 32) in both forms
    inst = I.maxcut_torus(1000, "pm1", seed=2)
    rng = np.random.default_rng(4)
    U = rng.standard_normal((inst.n, 32)) / math.sqrt(32)
    p = rng.standard_normal(inst.m)
    for prec in (0, 1):
        g, W, res, Ueff = run_grad(H, inst, U, p, 2.0, prec)
        ref = O.al_grad(inst, Ueff, p, 2.0)
        assert nrel(W, ref.W) <= TOL[prec]
        assert np.linalg.norm(res - ref.resid) <= TOL[prec] * np.linalg.norm(ref.T[1:])


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_theta_gnm_gradient(H, prec):
    # the Lovasz theta workload at its full size: G(n, M) with n = 1e5 and
    # M = 1e6 distinct edges, the trace row, implicit C = -11^T, r = 64
    inst = I.theta_gnm(100_000, 1_000_000, seed=3)
    rng = np.random.default_rng(6)
    U = rng.standard_normal((inst.n, 64)) / 8.0
    p = rng.standard_normal(inst.m)
    g, W, res, Ueff = run_grad(H, inst, U, p, 2.0, prec)
    ref = O.al_grad(inst, Ueff, p, 2.0)
    tol = TOL[prec]
    assert nrel(W, ref.W) <= tol
    assert np.linalg.norm(res - ref.resid) <= tol * np.linalg.norm(ref.T[1:])
    assert abs(g - ref.g) <= tol * scalar_scale(inst, Ueff, p, 2.0)
    dt = np.float32 if prec else np.float64
    with H.create_from_instance(inst, prec) as hd:
        Td = torch.empty(inst.m + 1, dtype=torch.float64, device="cuda")
        H.hallar_eval_A(hd.h, torch.from_numpy(U.astype(dt)).cuda(), 64, Td)
        T = Td.cpu().numpy()
    assert nrel(T[1:], ref.T[1:]) <= tol
    assert abs(T[0] - ref.T[0]) <= tol * scalar_scale(inst, Ueff, np.zeros(inst.m), 0.0)


def test_empty_rows_and_isolated_vertices(H):
    ei = np.array([0, 5, 9])
    ej = np.array([3, 7, 2])
    inst = I.theta(50, ei, ej)
    U = np.random.default_rng(0).standard_normal((50, 3))
    p = np.random.default_rng(1).standard_normal(inst.m)
    g, W, res, Ueff = run_grad(H, inst, U, p, 2.0, 0)
    ref = O.al_grad(inst, Ueff, p, 2.0)
    assert nrel(W, ref.W) <= 1e-12 and nrel(res, ref.resid) <= 1e-12


def test_invalid_inputs_are_rejected(H):
    inst = I.maxcut(10, *I.cycle_graph(10))
    with pytest.raises(H.HallarError):  # asymmetric C
        H.hallar_create(10, 0, inst.C_rowptr, inst.C_col,
                        inst.C_val * np.linspace(1, 2, inst.C_val.size), 0.0, 0.0, "diag", [], [],
                        0, inst.b, 10.0)
    with pytest.raises(H.HallarError):  # pair index out of range
        H.hallar_create(10, 0, None, None, None, -1.0, 0.0, "edge", [0, 3], [11, 2], 1,
                        np.zeros(3), 1.0)
    bad = inst.b.copy()
    bad[3] = np.nan
    with pytest.raises(H.HallarError):  # NaN in b
        H.hallar_create(10, 0, inst.C_rowptr, inst.C_col, inst.C_val, 0.0, 0.0, "diag", [], [], 0,
                        bad, 10.0)
    with H.create_from_instance(inst) as hd:
        U = torch.zeros((10, 300), dtype=torch.float64, device="cuda")
        with pytest.raises(H.HallarError):  # r out of range
            H.hallar_grad(hd.h, U, 300, torch.zeros(10, dtype=torch.float64, device="cuda"), 1.0, U)


@pytest.mark.parametrize("fam,n,n1", [("diag", 300, 0), ("edge", 400, 0), ("observed", 350, 150)])
def test_min_eig_parity(H, fam, n, n1):
    inst = random_instance(fam, n, 21, n1=n1, trace=True, with_c=True, cj=-0.3, ci=0.1)
    ps = np.random.default_rng(2).standard_normal(inst.m)
    v0 = O.splitmix64_uniform(5, n)
    ref = O.min_eig(inst, ps, tol=1e-10, v0=v0, kmax=n)
    with H.create_from_instance(inst) as hd:
        v = np.empty(n)
        lam, it, res, conv = H.hallar_min_eig(hd.h, ps, 1e-10, 300, v0=v0, v=v)
    assert conv
    assert abs(lam - ref.lam) <= 1e-9 * max(1.0, abs(ref.lam))
    Gv = O.gradient_matrix_apply(inst, ps, v)
    assert np.linalg.norm(Gv - lam * v) <= 2e-10
    assert abs(np.linalg.norm(v) - 1.0) <= 1e-12


def test_min_eig_torus_closed_form(H):
    inst = I.maxcut_torus(200, "unit")
    c = 0.37
    with H.create_from_instance(inst) as hd:
        lam, it, res, conv = H.hallar_min_eig(hd.h, np.full(inst.n, c), 1e-8, 300)
    assert conv
    assert abs(lam - (c - 2.0)) <= 1e-8


def test_splitmix_start_vector_matches_oracle(H):
    # v0 = NULL starts Lanczos from the SplitMix64 vector of the seed: the
    # same run from the oracle's SplitMix64 vector gives the same numbers
    n = 64
    inst = I.maxcut(n, np.zeros(0, int), np.zeros(0, int))
    ps = np.arange(n, dtype=np.float64)
    v0 = O.splitmix64_uniform(0, n)
    with H.create_from_instance(inst, seed=0) as hd:
        lam_a, it_a, _, _ = H.hallar_min_eig(hd.h, ps, 1e-6, 8)
        lam_b, it_b, _, _ = H.hallar_min_eig(hd.h, ps, 1e-6, 8, v0=v0)
    assert lam_a == lam_b and it_a == it_b
