"""Seeded synthetic SDP instances for HALLaR (input data only).

This module builds the problem data of (P) -- min C.X s.t. A(X) = b,
X in the spectraplex {X psd, tr X <= tau^2} (Section 1, eqs. (P), (D) and
Delta Definition) -- for the three constraint families the library supports:

* ``diag``     A_i = e_i e_i^T, one constraint per vertex (Max-Cut SDP).
* ``edge``     A_l = (e_i e_j^T + e_j e_i^T)/2 for a vertex pair (i, j), so
               A_l.X = X_ij, optionally followed by a trace row A = I
               (Lovasz theta SDP, eq. lovasz of Section 5.3).
* ``observed`` the edge family on the off-diagonal block of an
               (n1 + n2) x (n1 + n2) matrix: A_l.X = X_{i, n1+j}
               (matrix completion SDP, eq. matcomp-sdp of Section 5.2).

The cost is C = C_sparse + C_J * 11^T + C_I * I with C_sparse a symmetric
CSR matrix (full pattern, both triangles, diagonal allowed).

Everything here is data preparation: graphs, weights, right-hand sides and
the trace bound.  No operator of the method is evaluated here; the oracle and
the CUDA library both consume these arrays.  All randomness comes from
``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FAMILIES = ("diag", "edge", "observed")
# general problems in HSLR form (Section 3.2, eq. HSLR-rep-body); the oracle
# evaluates them, the device library has no kernels for them yet
GENERAL_FAMILIES = ("hslr", "phase")


@dataclass
class Instance:
    """Problem data of one SDP (P) in the library's input layout.

    Attributes mirror the arguments of ``hallar_create``: a symmetric CSR for
    the sparse part of C, the implicit coefficients C_J (all-ones) and C_I
    (identity), a constraint family, its index pairs, the right-hand side b
    (the trace row, when present, is the last entry) and tau^2, the trace
    bound of the spectraplex.  ``sense`` is -1 for problems that are
    maximisations stated as min (-C).X, so that the user-facing value is
    ``sense * pval``.
    """

    name: str
    family: str
    n: int
    n1: int
    C_rowptr: np.ndarray
    C_col: np.ndarray
    C_val: np.ndarray
    C_J: float
    C_I: float
    cons_i: np.ndarray
    cons_j: np.ndarray
    has_trace_row: bool
    b: np.ndarray
    tau2: float
    sense: float = 1.0
    meta: dict = field(default_factory=dict)
    # family "hslr" only: the sparse parts of A_1..A_m as entries (l, a, b, v)
    # over the full symmetric pattern (both triangles, l zero-based), and the
    # low-rank parts as (l, K_l, D_l) with l = 0 for C
    sp_cons: tuple | None = None
    lr_terms: list = field(default_factory=list)
    # family "phase" only: the K x n complex masks of the coded diffraction
    # measurements (phase retrieval, Section 5.4)
    masks: np.ndarray | None = None

    @property
    def m(self) -> int:
        """Number of constraints (pairs plus the optional trace row, or n)."""
        return int(self.b.shape[0])

    @property
    def m_pairs(self) -> int:
        return int(self.cons_i.shape[0])

    @property
    def tau(self) -> float:
        return math.sqrt(self.tau2)

    def host_bytes(self) -> int:
        """Bytes of the arrays a caller hands to ``hallar_create``."""
        return int(self.C_rowptr.nbytes + self.C_col.nbytes + self.C_val.nbytes
                   + self.cons_i.nbytes + self.cons_j.nbytes + self.b.nbytes)


# ----------------------------------------------------------------------------
# graphs (undirected, simple; edges returned with i < j)
# ----------------------------------------------------------------------------

def _canon(ei, ej):
    ei = np.asarray(ei, dtype=np.int64)
    ej = np.asarray(ej, dtype=np.int64)
    lo = np.minimum(ei, ej)
    hi = np.maximum(ei, ej)
    return lo, hi


def er_graph(n: int, p: float, seed: int):
    """Erdos-Renyi G(n, p): every pair i < j is an edge with probability p.

    For n <= 20000 the pairs are enumerated; beyond that the edge count is
    drawn Binomial(n(n-1)/2, p) and that many distinct pairs are sampled
    (G(n, p) conditioned on its edge count is G(n, M)).
    """
    rng = np.random.default_rng(seed)
    npairs = n * (n - 1) // 2
    if n <= 4000:
        iu, ju = np.triu_indices(n, k=1)
        keep = rng.random(npairs) < p
        return iu[keep].astype(np.int64), ju[keep].astype(np.int64)
    M = int(rng.binomial(npairs, p))
    return _sample_distinct_pairs(n, M, rng)


def _sample_distinct_pairs(n: int, M: int, rng):
    """M distinct uniformly random unordered pairs i != j, returned i < j."""
    if M > n * (n - 1) // 2:
        raise ValueError("more edges than pairs")
    keys = np.empty(0, dtype=np.int64)
    while keys.shape[0] < M:
        need = int((M - keys.shape[0]) * 1.2) + 16
        a = rng.integers(0, n, size=need, dtype=np.int64)
        c = rng.integers(0, n, size=need, dtype=np.int64)
        ok = a != c
        lo, hi = _canon(a[ok], c[ok])
        keys = np.unique(np.concatenate([keys, lo * n + hi]))
    if keys.shape[0] > M:
        keys = np.sort(rng.choice(keys, size=M, replace=False))
    return keys // n, keys % n


def gnm_graph(n: int, M: int, seed: int):
    """G(n, M): M distinct uniform edges without self-loops."""
    rng = np.random.default_rng(seed)
    return _sample_distinct_pairs(n, M, rng)


def torus_graph(N1: int, N2: int):
    """2D toroidal grid N1 x N2: each vertex joins its right and down
    neighbours with wrap-around (2 N1 N2 edges for N1, N2 >= 3)."""
    idx = np.arange(N1 * N2, dtype=np.int64).reshape(N1, N2)
    right = np.roll(idx, -1, axis=1)
    down = np.roll(idx, -1, axis=0)
    ei = np.concatenate([idx.ravel(), idx.ravel()])
    ej = np.concatenate([right.ravel(), down.ravel()])
    return _canon(ei, ej)


def complete_graph(n: int):
    iu, ju = np.triu_indices(n, k=1)
    return iu.astype(np.int64), ju.astype(np.int64)


def cycle_graph(n: int):
    i = np.arange(n, dtype=np.int64)
    return _canon(i, (i + 1) % n)


def hypercube_graph(d: int):
    """Hamming graph H(d, 2) = hypercube Q_d: vertices {0,1}^d, edges at
    Hamming distance one (n = 2^d, |E| = d 2^(d-1))."""
    n = 1 << d
    v = np.arange(n, dtype=np.int64)
    ei, ej = [], []
    for k in range(d):
        nb = v ^ (1 << k)
        keep = v < nb
        ei.append(v[keep])
        ej.append(nb[keep])
    return np.concatenate(ei), np.concatenate(ej)


# ----------------------------------------------------------------------------
# SDP instances
# ----------------------------------------------------------------------------

def _sym_csr(n: int, ei, ej, w, diag=None):
    """Full symmetric CSR (both triangles, sorted columns) of the matrix with
    entries w at (ei, ej) and (ej, ei), plus an optional diagonal."""
    ei = np.asarray(ei, dtype=np.int64)
    ej = np.asarray(ej, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    rows = [ei, ej]
    cols = [ej, ei]
    vals = [w, w]
    if diag is not None:
        d = np.asarray(diag, dtype=np.float64)
        nzd = np.nonzero(d)[0]
        rows.append(nzd)
        cols.append(nzd)
        vals.append(d[nzd])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, c.astype(np.int32), v


def _empty_csr(n: int):
    return (np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32),
            np.zeros(0, dtype=np.float64))


def maxcut(n: int, ei, ej, w=None, name: str = "maxcut") -> Instance:
    """Max-Cut SDP: max (1/4) L.X s.t. diag(X) = 1, X psd, stated as
    min C.X with C = -L/4 (L the weighted Laplacian), b = 1, tau^2 = n
    (trace of any feasible X).  User value = -pval."""
    ei = np.asarray(ei, dtype=np.int64)
    ej = np.asarray(ej, dtype=np.int64)
    w = np.ones(ei.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
    deg = np.zeros(n)
    np.add.at(deg, ei, w)
    np.add.at(deg, ej, w)
    rowptr, col, val = _sym_csr(n, ei, ej, w / 4.0, diag=-deg / 4.0)
    return Instance(name=name, family="diag", n=n, n1=0, C_rowptr=rowptr, C_col=col,
                    C_val=val, C_J=0.0, C_I=0.0, cons_i=np.zeros(0, np.int32),
                    cons_j=np.zeros(0, np.int32), has_trace_row=False,
                    b=np.ones(n), tau2=float(n), sense=-1.0,
                    meta={"edges": int(ei.shape[0]), "total_weight": float(w.sum())})


def theta(n: int, ei, ej, trace_row: bool = True, name: str = "theta") -> Instance:
    """Lovasz theta SDP: max 11^T.X s.t. X_ij = 0 on edges, tr X <= 1 (with
    ``trace_row`` also tr X = 1 as an equality row), stated as min with
    C = -11^T (implicit), tau^2 = 1.  User value = -pval = theta(G)."""
    lo, hi = _canon(ei, ej)
    b = np.zeros(lo.shape[0] + (1 if trace_row else 0))
    if trace_row:
        b[-1] = 1.0
    rowptr, col, val = _empty_csr(n)
    return Instance(name=name, family="edge", n=n, n1=0, C_rowptr=rowptr, C_col=col,
                    C_val=val, C_J=-1.0, C_I=0.0, cons_i=lo.astype(np.int32),
                    cons_j=hi.astype(np.int32), has_trace_row=trace_row, b=b,
                    tau2=1.0, sense=-1.0, meta={"edges": int(lo.shape[0])})


def completion_sample_count(n1: int, n2: int, r: int) -> int:
    """Number of observed entries used in the matrix-completion experiments
    (Section 5.2): ceil(gamma * r * (n1 + n2)) with oversampling
    gamma = r ln(n1 + n2).  The printed formula carries (n1 + n2 - r), but the
    (n1, n2; m) values of Table tab:gpuourmethod_vs_cpu are reproduced by
    (n1 + n2); the table is followed."""
    N = n1 + n2
    return int(math.ceil(r * math.log(N) * r * N))


def completion(n1: int, n2: int, rank: int, m: int, seed: int,
               tau2_slack: float = 1.1, name: str = "completion") -> Instance:
    """Matrix completion SDP (eq. matcomp-sdp): min (1/2) tr X s.t.
    X_{i, n1+j} = M_ij on m uniformly drawn entries, M = G H^T with Gaussian
    n1 x rank and n2 x rank factors.  tau^2 = tau2_slack * 2 ||M||_* (the
    optimal X = [W1 M; M^T W2] has trace 2 ||M||_* under exact recovery)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n1, rank))
    H = rng.standard_normal((n2, rank))
    keys = rng.choice(n1 * n2, size=m, replace=False) if n1 * n2 <= 50_000_000 \
        else _sample_keys(n1 * n2, m, rng)
    keys = np.sort(keys)
    ci = (keys // n2).astype(np.int64)
    cj = (keys % n2).astype(np.int64)
    vals = np.einsum("kr,kr->k", G[ci], H[cj])
    qg, rg = np.linalg.qr(G)
    qh, rh = np.linalg.qr(H)
    nuc = float(np.linalg.svd(rg @ rh.T, compute_uv=False).sum())
    n = n1 + n2
    rowptr, col, val = _empty_csr(n)
    return Instance(name=name, family="observed", n=n, n1=n1, C_rowptr=rowptr,
                    C_col=col, C_val=val, C_J=0.0, C_I=0.5,
                    cons_i=ci.astype(np.int32), cons_j=cj.astype(np.int32),
                    has_trace_row=False, b=vals, tau2=tau2_slack * 2.0 * nuc,
                    sense=1.0, meta={"nuclear_norm": nuc, "rank": rank,
                                     "G": G, "H": H})


def _sample_keys(N: int, m: int, rng):
    keys = np.empty(0, dtype=np.int64)
    while keys.shape[0] < m:
        need = int((m - keys.shape[0]) * 1.1) + 16
        keys = np.unique(np.concatenate([keys, rng.integers(0, N, size=need)]))
    if keys.shape[0] > m:
        keys = rng.choice(keys, size=m, replace=False)
    return keys


def initial_factor(n: int, r: int, seed: int) -> np.ndarray:
    """U_0 with independent standard Gaussian entries (Section 5.1,
    Initialization), n x r row-major float64."""
    return np.random.default_rng(seed).standard_normal((n, r))


# ----------------------------------------------------------------------------
# the named workloads
# ----------------------------------------------------------------------------

def maxcut_er_1000(seed: int = 1) -> Instance:
    """Max-Cut SDP on Erdos-Renyi G(1000, 0.01), unit weights."""
    ei, ej = er_graph(1000, 0.01, seed)
    return maxcut(1000, ei, ej, name="maxcut_er_n1000_p0.01")


def maxcut_torus(N: int = 1000, weights: str = "pm1", seed: int = 2) -> Instance:
    """Max-Cut SDP on the N x N torus with Rademacher +-1 weights (``pm1``)
    or unit weights (``unit``)."""
    ei, ej = torus_graph(N, N)
    if weights == "pm1":
        w = np.random.default_rng(seed).choice([-1.0, 1.0], size=ei.shape[0])
    elif weights == "unit":
        w = np.ones(ei.shape[0])
    else:
        raise ValueError(weights)
    return maxcut(N * N, ei, ej, w, name=f"maxcut_torus_{N}x{N}_{weights}")


def theta_gnm(n: int = 100_000, M: int = 1_000_000, seed: int = 3) -> Instance:
    """Lovasz theta SDP on G(n, M) with the tr X = 1 row."""
    ei, ej = gnm_graph(n, M, seed)
    return theta(n, ei, ej, trace_row=True, name=f"theta_gnm_n{n}_m{M}")


# ----------------------------------------------------------------------------
# general problems in HSLR form
# ----------------------------------------------------------------------------

def _upper_to_full(ell, a, b, v):
    """Entries of symmetric matrices listed by their upper triangle (a <= b)
    -> the full pattern (both triangles; the diagonal once)."""
    ell = np.asarray(ell, dtype=np.int64)
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    v = np.asarray(v, dtype=np.float64)
    if np.any(a > b):
        raise ValueError("entries must be listed by their upper triangle (i <= j)")
    off = a != b
    return (np.concatenate([ell, ell[off]]), np.concatenate([a, b[off]]),
            np.concatenate([b, a[off]]), np.concatenate([v, v[off]]))


def hslr(n: int, sp_upper, lr_terms, b, tau2: float, sense: float = 1.0,
         name: str = "hslr", meta: dict | None = None) -> Instance:
    """A general SDP (P) in Hybrid Sparse Low-Rank form (Section 3.2, eq.
    HSLR-rep-body): A_l = A_l^sp + K_l D_l K_l^T for l = 0..m, C = A_0.

    sp_upper: (l, i, j, v) arrays, the nonzero entries of every A_l^sp on or
        above the diagonal (i <= j), l = 0 for C and 1..m for the constraints.
    lr_terms: a list of (l, K_l, D_l): K_l an n x r_l array, D_l an r_l x r_l
        symmetric array (not necessarily diagonal).
    b: the m right-hand sides; tau2 the trace bound tau^2 of the spectraplex.
    Duplicate (l, i, j) entries are summed.
    """
    ell, a, bb, v = (np.asarray(x) for x in sp_upper)
    b = np.asarray(b, dtype=np.float64)
    m = b.shape[0]
    if ell.size and (ell.min() < 0 or ell.max() > m):
        raise ValueError("matrix index outside 0..m")
    if a.size and (min(a.min(), bb.min()) < 0 or max(a.max(), bb.max()) >= n):
        raise ValueError("entry index outside 0..n-1")
    terms = []
    for l, K, D in lr_terms:
        K = np.asarray(K, dtype=np.float64)
        D = np.asarray(D, dtype=np.float64)
        if K.ndim == 1:
            K = K[:, None]
        D = np.atleast_2d(D)
        if not (0 <= l <= m) or K.shape[0] != n or D.shape != (K.shape[1], K.shape[1]):
            raise ValueError("low-rank term shape")
        if not np.allclose(D, D.T, rtol=0.0, atol=0.0):
            raise ValueError("D_l must be symmetric")
        terms.append((int(l), K, D))
    c0 = ell == 0
    ci, cj, cv = a[c0].astype(np.int64), bb[c0].astype(np.int64), v[c0].astype(np.float64)
    if np.any(ci > cj):
        raise ValueError("entries must be listed by their upper triangle (i <= j)")
    off = ci != cj
    diag = np.zeros(n)
    np.add.at(diag, ci[~off], cv[~off])
    rowptr, col, val = _sym_csr(n, ci[off], cj[off], cv[off], diag=diag)
    # duplicates of one (i, j) in C: _sym_csr keeps them as separate stored
    # entries, which the entry sums treat as their sum
    cons = _upper_to_full(ell[~c0] - 1, a[~c0], bb[~c0], v[~c0])
    return Instance(name=name, family="hslr", n=n, n1=0, C_rowptr=rowptr, C_col=col,
                    C_val=val, C_J=0.0, C_I=0.0, cons_i=np.zeros(0, np.int32),
                    cons_j=np.zeros(0, np.int32), has_trace_row=False, b=b,
                    tau2=float(tau2), sense=float(sense), meta=dict(meta or {}),
                    sp_cons=cons, lr_terms=terms)


# ----------------------------------------------------------------------------
# phase retrieval (Section 5.4)
# ----------------------------------------------------------------------------

def phase_retrieval(n: int, K: int = 12, seed: int = 7, name: str = "phase") -> Instance:
    """The phase retrieval SDP of Section 5.4 (eq. phase retrieval SDP):
    min tr X s.t. <a_i a_i^H, X> = b_i, X Hermitian psd, with tau^2 = |x|^2
    (the paper takes the squared norm of the signal as the trace bound).

    Reading: the paper fixes no measurement ensemble beyond needing an FFT.
    Here the measurements are coded diffraction patterns: K masks d_k with
    entries drawn uniformly from {1, -1, i, -i}, and b_{k,j} = |FFT(d_k * x)_j|^2
    for j = 0..n-1 (numpy's unnormalised forward FFT), so m = K n (the paper's
    instances have m = 12 n).  The signal x has independent standard complex
    Gaussian entries.  Family "phase"; C = I (C_I = 1), n complex dimensions.
    """
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / math.sqrt(2.0)
    masks = np.array([1.0, -1.0, 1j, -1j])[rng.integers(0, 4, size=(K, n))]
    b = (np.abs(np.fft.fft(masks * x[None, :], axis=1)) ** 2).ravel()
    rowptr, col, val = _empty_csr(n)
    return Instance(name=name, family="phase", n=n, n1=0, C_rowptr=rowptr, C_col=col,
                    C_val=val, C_J=0.0, C_I=1.0, cons_i=np.zeros(0, np.int32),
                    cons_j=np.zeros(0, np.int32), has_trace_row=False, b=b,
                    tau2=float(np.vdot(x, x).real), sense=1.0,
                    meta={"signal": x, "K": K}, masks=masks)
