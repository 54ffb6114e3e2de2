"""Batched operators (hallar_batch_*): the fused constraint map + shift + SpMM
of many uneven instances in one launch over a stacked, segmented CSR,
compared instance by instance with the oracle (FP64 to 1e-12, the mixed form
to 1e-5 against the oracle on the same float-rounded factors)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hallar_oracle as O  # noqa: E402
from paper_2505_13719_b300 import instances as I  # noqa: E402
from tests.test_gpu_operators import nrel, scalar_scale  # noqa: E402
from tests.test_oracle_operators import random_instance  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13719_b300 import hallar
    return hallar


def mixed_instances():
    """Uneven sizes and every supported family side by side."""
    return [
        I.maxcut(777, *I.er_graph(777, 0.01, 1)),
        I.completion(40, 55, 3, 900, seed=2),
        random_instance("edge", 300, 3, trace=False, with_c=True, cj=0.0, ci=0.2),
        I.maxcut(33, *I.cycle_graph(33)),
        random_instance("diag", 1500, 4, with_c=True, cj=0.0, ci=-0.3),
        random_instance("observed", 500, 5, n1=200, trace=False, with_c=False, ci=0.5),
        I.maxcut(1, np.zeros(0, int), np.zeros(0, int)),  # a single row, no edges
    ]


def run_batch(H, insts, r, prec, autotune, seed=0, host=False):
    dt = np.float32 if prec else np.float64
    rng = np.random.default_rng(seed)
    with H.Batch(insts, prec, autotune=autotune) as bt:
        U = (rng.standard_normal((bt.n_total, r)) / math.sqrt(r)).astype(dt)
        p = rng.standard_normal(bt.m_total)
        beta = rng.uniform(0.5, 3.0, size=bt.count)
        if host:
            W = np.empty_like(U)
            g = np.empty(bt.count)
            res = np.empty(bt.m_total)
            bt.grad(U, r, p, beta, W, g, res)
        else:
            Ud = torch.from_numpy(U).cuda()
            Wd = torch.empty_like(Ud)
            gd = torch.empty(bt.count, dtype=torch.float64, device="cuda")
            rd = torch.empty(bt.m_total, dtype=torch.float64, device="cuda")
            bt.grad(Ud, r, torch.from_numpy(p).cuda(), torch.from_numpy(beta).cuda(), Wd, gd, rd)
            torch.cuda.synchronize()
            W, g, res = Wd.cpu().numpy(), gd.cpu().numpy(), rd.cpu().numpy()
        shape = bt.shape(r)
        return U.astype(np.float64), p, beta, W.astype(np.float64), g, res, bt.row_off.copy(), \
            bt.cons_off.copy(), shape


def check_against_oracle(insts, U, p, beta, W, g, res, ro, co, tol):
    for k, inst in enumerate(insts):
        Uk = U[ro[k]:ro[k + 1]]
        pk = p[co[k]:co[k + 1]]
        ref = O.al_grad(inst, Uk, pk, beta[k])
        assert nrel(W[ro[k]:ro[k + 1]], ref.W) <= tol, k
        assert np.linalg.norm(res[co[k]:co[k + 1]] - ref.resid) <= \
            tol * (np.linalg.norm(ref.T[1:]) + 1e-300), k
        assert abs(g[k] - ref.g) <= tol * scalar_scale(inst, Uk, pk, beta[k]), k


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("r", [1, 3, 10, 17, 32])
def test_batch_grad_matches_oracle_per_instance(H, r, prec):
    insts = mixed_instances()
    out = run_batch(H, insts, r, prec, autotune=False, seed=r)
    check_against_oracle(insts, *out[:8], TOL[prec])
    assert out[8][2] is False  # the built-in rule, not timed


@pytest.mark.parametrize("prec", [0, 1])
def test_autotuned_shape_matches_oracle(H, prec):
    insts = mixed_instances()
    out = run_batch(H, insts, 10, prec, autotune=True, seed=7)
    check_against_oracle(insts, *out[:8], TOL[prec])
    G, K, tuned = out[8]
    assert tuned and G * K * (4 if prec else 2) >= 10


def test_batch_host_pointers(H):
    insts = mixed_instances()[:3]
    out = run_batch(H, insts, 6, 0, autotune=False, seed=3, host=True)
    check_against_oracle(insts, *out[:8], TOL[0])


def test_batch_rejects_trace_rows_and_C_J(H):
    theta = I.theta(9, *I.cycle_graph(9))  # trace row and C_J = -1
    with pytest.raises(H.HallarError) as e:
        H.Batch([I.maxcut(33, *I.cycle_graph(33)), theta])
    assert e.value.status == H.HALLAR_EINVAL and "instance 1" in str(e.value)
