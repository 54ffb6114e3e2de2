"""The allocation-free fused gradient, against the regular entry point and the oracle.

hallar_grad_diag_noalloc is for callers that cannot let the library allocate
device memory (applications that serve every device byte from their own pool,
hot paths where an allocation would stall other streams); it keeps its
reduction scratch in a static device array shared by all calls.  Each case
calls it twice in a row through the C ABI, on different inputs, and compares
each result with hallar_grad on the same inputs and with the FP64 oracle's
al_grad, to the FP64 tolerance of the other operator tests (1e-12).  The
cases cover every group width (r = 2, 6, 8, 64; r = 6 leaves lanes of its
group idle), a grid at the 1184-block cap with grid-stride rows (r = 2 on
3.6e5 rows), and resid = NULL.  This file is collected last, so a run that
stops at its first failure has run every other test first.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hallar_oracle as O  # noqa: E402
from paper_2505_13719_b300 import instances as I  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-12


def split_csr(inst):
    """Off-diagonal CSR (int32) and the diagonal of C from an instance."""
    rp = inst.C_rowptr
    rows = np.repeat(np.arange(inst.n), np.diff(rp))
    off = inst.C_col != rows
    diag = np.zeros(inst.n)
    np.add.at(diag, rows[~off], inst.C_val[~off])
    counts = np.bincount(rows[off], minlength=inst.n)
    rowptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    return rowptr, inst.C_col[off].astype(np.int32), inst.C_val[off].copy(), diag + inst.C_I


def g_scale(inst, U, p, beta, resid):
    """Sum of the magnitudes of the terms of g: the scale of its rounding."""
    a, b, v = O.cost_entries(inst)
    cterm = float(np.sum(np.abs(v) * np.abs(np.einsum("kr,kr->k", U[a], U[b]))))
    return cterm + float(np.abs(p * resid).sum()) + 0.5 * beta * float(resid @ resid) + 1.0


CASES = [
    # (torus side, r, write resid)
    (64, 8, True),
    (64, 2, True),
    (64, 6, False),
    (40, 64, True),
    (600, 2, False),   # n = 3.6e5 rows: the 1184-block cap, grid-stride rows
]


@pytest.mark.parametrize("side,r,with_resid", CASES,
                         ids=[f"n{c[0] ** 2}-r{c[1]}-resid{int(c[2])}" for c in CASES])
def test_noalloc_gradient_matches_hallar_grad_and_oracle_twice(side, r, with_resid):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13719_b300 import hallar as H
    inst = I.maxcut_torus(side, "pm1", seed=5)
    n = inst.n
    rowptr, col, cval, cdiag = split_csr(inst)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_rowptr, d_col, d_cval, d_cdiag, d_b = map(dev, (rowptr, col, cval, cdiag, inst.b))
    rng = np.random.default_rng(11 + r)
    stream = torch.cuda.current_stream()
    with H.create_from_instance(inst) as hd:
        for call in range(2):
            U = rng.standard_normal((n, r)) / np.sqrt(r)
            p = rng.standard_normal(n)
            beta = 1.3 + call
            # the existing entry point
            W_ref = np.empty((n, r))
            res_ref = np.empty(n)
            g_ref = H.hallar_grad(hd.h, U, r, p, beta, W_ref, res_ref)
            # the oracle
            ref = O.al_grad(inst, U, p, beta)
            # the allocation-free entry point
            dU, dp = dev(U), dev(p)
            dW = torch.empty_like(dU)
            dres = torch.empty(n, dtype=torch.float64, device="cuda") if with_resid else None
            dg = torch.zeros(1, dtype=torch.float64, device="cuda")
            H.hallar_grad_diag_noalloc(n, r, d_rowptr, d_col, d_cval, d_cdiag, d_b, dp, beta,
                                       dU, dW, dres, dg, stream.cuda_stream)
            torch.cuda.synchronize()
            W = dW.cpu().numpy()
            g = float(dg.cpu().numpy()[0])
            scale = g_scale(inst, U, p, beta, ref.resid)
            for Wr, gr in ((W_ref, g_ref), (ref.W, ref.g)):
                assert np.linalg.norm(W - Wr) <= TOL * np.linalg.norm(Wr)
                assert abs(g - gr) <= TOL * scale
            if with_resid:
                res = dres.cpu().numpy()
                for rr in (res_ref, ref.resid):
                    assert np.linalg.norm(res - rr) <= TOL * np.linalg.norm(ref.T[1:])


def test_noalloc_rejects_sizes_beyond_its_limits():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13719_b300 import hallar as H
    z = torch.zeros(16, dtype=torch.float64, device="cuda")
    zi = torch.zeros(16, dtype=torch.int32, device="cuda")
    for r in (66, 3, 0):
        with pytest.raises(H.HallarError) as ei:
            H.hallar_grad_diag_noalloc(4, r, zi, zi, z, z, z, z, 1.0, z, z, None, z)
        assert "r must be even" in str(ei.value)
