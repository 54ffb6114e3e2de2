"""The allocation-free fused gradient against the regular entry point.

hallar_grad_diag_noalloc is for callers that cannot let the library
allocate device memory (graph capture, caller-managed pools, allocator-free
hot paths); it keeps its reduction scratch in a static device array shared
by all calls.  This test calls it twice in a row through the C ABI, on
different inputs, and compares each result with hallar_grad on the same
inputs, to the FP64 tolerance of the other operator tests (1e-12).  This
file is collected last, so a run that stops at its first failure has run
every other test first.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_13719_b300 import instances as I  # noqa: E402

pytestmark = pytest.mark.gpu


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


def test_noalloc_gradient_matches_hallar_grad_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13719_b300 import hallar as H
    inst = I.maxcut_torus(64, "pm1", seed=5)
    n, r = inst.n, 8
    rowptr, col, cval, cdiag = split_csr(inst)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_rowptr, d_col, d_cval, d_cdiag, d_b = map(dev, (rowptr, col, cval, cdiag, inst.b))
    rng = np.random.default_rng(11)
    stream = torch.cuda.current_stream()
    with H.create_from_instance(inst) as hd:
        for call in range(2):
            U = rng.standard_normal((n, r)) / np.sqrt(r)
            p = rng.standard_normal(n)
            beta = 1.3 + call
            # regular entry point
            W_ref = np.empty((n, r))
            res_ref = np.empty(n)
            g_ref = H.hallar_grad(hd.h, U, r, p, beta, W_ref, res_ref)
            # allocation-free entry point
            dU, dp = dev(U), dev(p)
            dW = torch.empty_like(dU)
            dres = torch.empty(n, dtype=torch.float64, device="cuda")
            dg = torch.zeros(1, dtype=torch.float64, device="cuda")
            H.hallar_grad_diag_noalloc(n, r, d_rowptr, d_col, d_cval, d_cdiag, d_b, dp, beta,
                                       dU, dW, dres, dg, stream.cuda_stream)
            torch.cuda.synchronize()
            W = dW.cpu().numpy()
            assert np.linalg.norm(W - W_ref) <= 1e-12 * np.linalg.norm(W_ref)
            assert np.linalg.norm(dres.cpu().numpy() - res_ref) <= 1e-12 * np.linalg.norm(res_ref)
            g = float(dg.cpu().numpy()[0])
            assert abs(g - g_ref) <= 1e-12 * (abs(g_ref) + np.abs(p * res_ref).sum() + 1.0)


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
