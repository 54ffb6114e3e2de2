"""GPU consumers of a solved factor against the oracle (not in the paper).

hallar_maxcut_round (Goemans-Williamson hyperplane rounding) takes its sign
decisions and cut sums in double from the stored factor, like the oracle's
maxcut_round on the same factor and normals: the cut values match to 1e-12
and the best sign vector matches exactly except where <U_i, g> is within
rounding of zero.  On the unit-weight torus (bipartite) the solved factor
rounds to the maximum cut, the total edge weight.  hallar_factor_entries
matches the oracle's factor_entries, and on a solved completion problem
its off-diagonal block recovers the rank-2 truth.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hallar_oracle as O  # noqa: E402
from paper_2505_13719_b300 import instances as I  # noqa: E402
from tests.test_gpu_solve import gpu_solve  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13719_b300 import hallar
    return hallar


@pytest.mark.parametrize("prec", [0, 1])
def test_round_matches_oracle_on_a_solved_factor(H, prec):
    inst = I.maxcut(300, *I.er_graph(300, 0.03, 7))
    st, res, U, p = gpu_solve(H, inst, 3, 8, prec=prec)
    assert st == H.HALLAR_OK
    r = U.shape[1]
    G = np.random.default_rng(9).standard_normal((16, r))
    dt = np.float32 if prec else np.float64
    Us = np.ascontiguousarray(U.astype(dt))
    xb = np.empty(inst.n, dtype=np.int8)
    with H.create_from_instance(inst, prec) as hd:
        cuts = H.hallar_maxcut_round(hd.h, Us, r, G, xb)
    ref, X = O.maxcut_round(inst, Us.astype(np.float64), G)
    scale = 1.0 + float(np.abs(inst.C_val).sum())
    assert np.all(np.abs(cuts - ref) <= 1e-12 * scale)
    best = int(np.argmax(ref))
    dots = Us.astype(np.float64) @ G[best]
    tiny = np.abs(dots) <= 1e-12 * (np.abs(Us.astype(np.float64)) @ np.abs(G[best]))
    assert np.array_equal(xb[~tiny], X[best][~tiny].astype(np.int8))
    # the SDP value bounds every cut
    assert cuts.max() <= inst.sense * res.pval * (1 + 1e-5)


def test_round_recovers_the_bipartite_maximum_cut(H):
    inst = I.maxcut_torus(32, "unit")
    st, res, U, p = gpu_solve(H, inst, 2, 7, prec=1)
    assert st == H.HALLAR_OK
    G = np.random.default_rng(1).standard_normal((4, U.shape[1]))
    with H.create_from_instance(inst, 1) as hd:
        cuts = H.hallar_maxcut_round(hd.h, np.ascontiguousarray(U.astype(np.float32)),
                                     U.shape[1], G)
    assert cuts.max() == 2048.0


def test_round_rejects_other_families(H):
    inst = I.theta(9, *I.cycle_graph(9))
    with H.create_from_instance(inst) as hd:
        with pytest.raises(H.HallarError):
            H.hallar_maxcut_round(hd.h, np.zeros((9, 2)), 2, np.ones((1, 2)))


@pytest.mark.parametrize("prec", [0, 1])
def test_factor_entries_recover_the_completion(H, prec):
    inst = I.completion(60, 80, 2, I.completion_sample_count(60, 80, 2), seed=5)
    st, res, U, p = gpu_solve(H, inst, 2, 9, prec=prec)
    assert st == H.HALLAR_OK
    n1, n2 = 60, 80
    ii, jj = np.meshgrid(np.arange(n1), np.arange(n2), indexing="ij")
    a = ii.ravel().astype(np.int32)
    b = (jj.ravel() + n1).astype(np.int32)
    dt = np.float32 if prec else np.float64
    Us = np.ascontiguousarray(U.astype(dt))
    out = np.empty(a.shape[0])
    with H.create_from_instance(inst, prec) as hd:
        H.hallar_factor_entries(hd.h, Us, U.shape[1], a, b, out)
        # device index arrays and output
        od = torch.empty(a.shape[0], dtype=torch.float64, device="cuda")
        H.hallar_factor_entries(hd.h, torch.from_numpy(Us).cuda(), U.shape[1],
                                torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), od)
    ref = O.factor_entries(Us.astype(np.float64), a, b)
    assert np.allclose(out, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert np.array_equal(od.cpu().numpy(), out)
    M = inst.meta["G"] @ inst.meta["H"].T
    assert np.linalg.norm(out.reshape(n1, n2) - M) <= 1e-2 * np.linalg.norm(M)
