"""HALLaR FP64 CPU oracle -- TEST INFRASTRUCTURE, not product code.

A plain, slow, obviously-correct NumPy implementation of what the hot path of
HALLaR (the hybrid low-rank augmented Lagrangian method) computes:

* the constraint map T = A~(UU^T)                (eq. A tilde operator)
* the adjoint product W = A~*(p~) U              (eq. Adjoint calculation)
* the AL value g(U) = L_beta(UU^T; p) and its U-gradient
                                                 (eqs. AL function, Grad U Space)
* the minimum eigenpair of G = C + A*(p')        (Alg. 1 step 7, eq. Grad X Space)
* ADAP-FISTA, ADAP-AIPP, the HLR loop, the AL outer loop and the relative
  KKT test                                       (Appendix A, A.1; Alg. 1;
                                                  eq. termination2)

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this module.  It shares no code with the CUDA
library: it reads only the plain instance arrays.

Every function states the passage it follows.  Operators are written from
their definitions (sums over the stored entries of each A_l) with a sparse
matrix product as the only library step.  Where the paper is silent the
reading taken is stated in the docstring (``Reading:``) and in the design
notes.

Pins (tests/test_oracle_*.py): operators against dense brute force, the
adjoint identity, finite differences and the Max-Cut cut identity; Lanczos
against dense eigendecomposition and the closed-form torus and hypercube
spectra; the Frank-Wolfe step as an exact line search; ADAP-AIPP's output
invariants; ADAP-FISTA against the closed-form prox point of a quadratic;
the KKT measures at a closed-form optimal primal-dual pair; full solves
against closed-form SDP values with a dense dual certificate;
``splitmix64_uniform`` against the generator's published output words from
state 0; general problems in HSLR form (sparse plus low-rank A_l, Section
3.2) against dense brute force and theta(C_5) with a low-rank cost
(tests/test_oracle_hslr.py); phase retrieval's FFT operators against a
brute-force DFT, its real embedding, and exact recovery of the signal
(tests/test_oracle_phase.py).  Parity unpinned: iteration counts and trajectories (they
follow the readings, not the paper).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

# ----------------------------------------------------------------------------
# the data matrices as entry lists
# ----------------------------------------------------------------------------


def constraint_entries(inst):
    """Stored entries (l, a, b, value) of every constraint matrix A_l.

    Eq. Definition of Linear Operators: [A(X)]_l = A_l . X.  The families:
    diag  A_i = e_i e_i^T                       (one entry per constraint)
    edge  A_l = (e_i e_j^T + e_j e_i^T) / 2     (two entries, 1/2 each)
    trace A = I                                 (last constraint, n entries)
    For ``observed`` the pair is (i, n1 + j).  For ``hslr`` (eq.
    HSLR-rep-body) the sparse parts A_l^sp as given; their low-rank parts
    K_l D_l K_l^T are evaluated separately (``_lr_values``).
    """
    n = inst.n
    if inst.family == "hslr":
        return inst.sp_cons
    if inst.family == "diag":
        idx = np.arange(n, dtype=np.int64)
        return idx, idx, idx, np.ones(n)
    i = inst.cons_i.astype(np.int64)
    j = inst.cons_j.astype(np.int64)
    if inst.family == "observed":
        j = j + inst.n1
    k = np.arange(i.shape[0], dtype=np.int64)
    ls = [k, k]
    as_ = [i, j]
    bs = [j, i]
    vs = [np.full(k.shape[0], 0.5), np.full(k.shape[0], 0.5)]
    if inst.has_trace_row:
        d = np.arange(n, dtype=np.int64)
        ls.append(np.full(n, inst.m - 1, dtype=np.int64))
        as_.append(d)
        bs.append(d)
        vs.append(np.ones(n))
    return (np.concatenate(ls), np.concatenate(as_), np.concatenate(bs),
            np.concatenate(vs))


def cost_entries(inst):
    """Stored entries (a, b, value) of the sparse part of C (CSR expanded);
    C is the cost matrix of (P) (Section 1, eq. P), C_J 11^T and C_I I are
    implicit and handled by the callers."""
    rowptr = inst.C_rowptr.astype(np.int64)
    a = np.repeat(np.arange(inst.n, dtype=np.int64), np.diff(rowptr))
    return a, inst.C_col.astype(np.int64), inst.C_val.astype(np.float64)


def _pair_dots(U, a, b, chunk=1 << 20):
    """B_ab = <U_a,:, U_b,:> for each listed pair (Section 4.1, B = UU^T)."""
    out = np.empty(a.shape[0])
    for s in range(0, a.shape[0], chunk):
        e = min(s + chunk, a.shape[0])
        out[s:e] = np.einsum("kr,kr->k", U[a[s:e]], U[b[s:e]])
    return out


def _lr_values(inst, U):
    """A_l^lr . UU^T = tr(D_l Y_l Y_l^T) with Y_l = K_l^T U for every low-rank
    term (Section 4.1, Alg. 3, written by definition); returns (l, value)
    pairs, l = 0 for C."""
    out = []
    for l, K, D in inst.lr_terms:
        Y = K.T @ U
        out.append((l, float(np.sum(D * (Y @ Y.T)))))
    return out


# ----------------------------------------------------------------------------
# operators (Section 4)
# ----------------------------------------------------------------------------


def cost_dot(inst, U):
    """C . UU^T = sum over the stored entries of C of C_ab <U_a, U_b>
    + C_J ||1^T U||^2 + C_I ||U||_F^2 (T_0 of eq. A tilde operator)."""
    a, b, v = cost_entries(inst)
    val = float(np.dot(v, _pair_dots(U, a, b))) if v.shape[0] else 0.0
    if inst.C_J != 0.0:
        s = U.sum(axis=0)
        val += inst.C_J * float(s @ s)
    if inst.C_I != 0.0:
        val += inst.C_I * float(np.sum(U * U))
    for l, t in _lr_values(inst, U):
        if l == 0:
            val += t
    return val


def constraint_map(inst, U):
    """A(UU^T): T_l = sum_{(a,b) in supp A_l} (A_l)_ab <U_a, U_b>
    (Section 4.1; the sum that Alg. 2 evaluates, written by definition)."""
    ell, a, b, v = constraint_entries(inst)
    # (bincount of no entries is an integer array: force float)
    T = np.bincount(ell, weights=v * _pair_dots(U, a, b), minlength=inst.m).astype(np.float64)
    for l, t in _lr_values(inst, U):
        if l > 0:
            T[l - 1] += t
    return T


def eval_A_tilde(inst, U):
    """T = A~(UU^T) = [C . UU^T ; A(UU^T)] (eq. A tilde operator), m + 1 values."""
    return np.concatenate([[cost_dot(inst, U)], constraint_map(inst, U)])


def adjoint_matrix(inst, ptilde):
    """M = A~*(p~) = p~_0 C_sparse + sum_l p_l A_l as a sparse matrix
    (eq. Adjoint calculation; Alg. 4 forms M on the merged pattern).  The
    implicit C_J 11^T and C_I I parts are returned separately as scaled
    coefficients because 11^T is dense; the low-rank parts K_l D_l K_l^T of
    an ``hslr`` problem are not in M (``adjoint_apply`` applies them,
    ``dense_adjoint`` forms them)."""
    ptilde = np.asarray(ptilde, dtype=np.float64)
    ell, a, b, v = constraint_entries(inst)
    ca, cb, cv = cost_entries(inst)
    rows = np.concatenate([a, ca])
    cols = np.concatenate([b, cb])
    vals = np.concatenate([v * ptilde[1 + ell], cv * ptilde[0]])
    M = sp.coo_matrix((vals, (rows, cols)), shape=(inst.n, inst.n)).tocsr()
    return M, ptilde[0] * inst.C_J, ptilde[0] * inst.C_I


def adjoint_apply(inst, ptilde, U):
    """W = A~*(p~) U = (p~_0 C + A*(p)) U (eq. Adjoint calculation)."""
    M, cj, ci = adjoint_matrix(inst, ptilde)
    U2 = U if U.ndim == 2 else U[:, None]
    W = M @ U2
    if cj != 0.0:
        W = W + cj * np.ones((inst.n, 1)) * U2.sum(axis=0, keepdims=True)
    if ci != 0.0:
        W = W + ci * U2
    for l, K, D in inst.lr_terms:  # Alg. 5: + p~_l K_l (D_l (K_l^T U))
        if ptilde[l] != 0.0:
            W = W + ptilde[l] * (K @ (D @ (K.T @ U2)))
    return W if U.ndim == 2 else W[:, 0]


def dense_adjoint(inst, ptilde):
    """A~*(p~) = sum_l p~_l A_l as a dense n x n array, low-rank parts
    included (small instances: certificates and brute-force pins)."""
    ptilde = np.asarray(ptilde, dtype=np.float64)
    M, cj, ci = adjoint_matrix(inst, ptilde)
    G = M.toarray() + cj * np.ones((inst.n, inst.n)) + ci * np.eye(inst.n)
    for l, K, D in inst.lr_terms:
        G = G + ptilde[l] * (K @ D @ K.T)
    return G


@dataclass
class GradResult:
    g: float            # g(U) = L_beta(UU^T; p)
    W: np.ndarray       # (C + A*(p')) U; the U-gradient is 2W
    resid: np.ndarray   # r = A(UU^T) - b
    pshift: np.ndarray  # p' = p + beta r
    T: np.ndarray       # A~(UU^T)
    mag: float = 0.0    # sum |p'_l| |T_l| + sum |C terms|: the scale of g's rounding


def al_grad(inst, U, p, beta):
    """g(U) = C.UU^T + p^T r + (beta/2) ||r||^2 with r = A(UU^T) - b
    (eq. AL function) and W with grad g(U) = 2 W,
    W = [C + A*(p + beta r)] U (eq. Grad U Space)."""
    T = eval_A_tilde(inst, U)
    r = T[1:] - inst.b
    g = T[0] + float(p @ r) + 0.5 * beta * float(r @ r)
    ps = p + beta * r
    W = adjoint_apply(inst, np.concatenate([[1.0], ps]), U)
    return GradResult(g=g, W=W, resid=r, pshift=ps, T=T, mag=_magnitude(inst, U, ps, T))


def _magnitude(inst, U, ps, T):
    """sum_l |p'_l| |A_l.UU^T| plus the absolute values of the terms of
    C.UU^T: the size of the terms whose rounding perturbs g.  Not in the
    paper: it scales the rounding allowance of the ADAP-FISTA and ADAP-AIPP
    step-2 tests (a floating-point reading)."""
    a, b, v = cost_entries(inst)
    mag = float(np.abs(ps) @ np.abs(T[1:]))
    if v.shape[0]:
        mag += float(np.abs(v) @ np.abs(_pair_dots(U, a, b)))
    if inst.C_J != 0.0:
        s = U.sum(axis=0)
        mag += abs(inst.C_J) * float(s @ s)
    if inst.C_I != 0.0:
        mag += abs(inst.C_I) * float(np.sum(U * U))
    for l, K, D in inst.lr_terms:
        if l == 0:
            Y = K.T @ U
            mag += float(np.sum(np.abs(D) * np.abs(Y @ Y.T)))
    return mag


# unit roundoff of float64 and the multiple of it that the ADAP-FISTA and
# ADAP-AIPP step-2 tests allow (times lambda and the magnitude of g's terms)
UNIT_ROUNDOFF = 2.0 ** -53
ROUND_SLACK = 16.0


def al_value(inst, U, p, beta):
    """g(U) alone (eq. AL function)."""
    T = eval_A_tilde(inst, U)
    r = T[1:] - inst.b
    return T[0] + float(p @ r) + 0.5 * beta * float(r @ r)


def _pair_change(X, Y, D, a, b):
    """<Y_a, Y_b> - <X_a, X_b> for listed pairs, as <D_a, Y_b> + <X_a, D_b>
    with D = Y - X (an exact identity that avoids cancellation)."""
    return _pair_dots_mixed(D, Y, a, b) + _pair_dots_mixed(X, D, a, b)


def _pair_dots_mixed(P, Q, a, b, chunk=1 << 20):
    """<P_a,:, Q_b,:> for each listed pair (the pair products of Section 4.1
    with two different factors)."""
    out = np.empty(a.shape[0])
    for s in range(0, a.shape[0], chunk):
        e = min(s + chunk, a.shape[0])
        out[s:e] = np.einsum("kr,kr->k", P[a[s:e]], Q[b[s:e]])
    return out


def al_value_change(inst, X, Y, p, beta, rX=None):
    """g(Y) - g(X) for g(U) = L_beta(UU^T; p) (eq. AL function).

    Written through the differences of the pair products,
    <Y_a,Y_b> - <X_a,X_b> = <D_a,Y_b> + <X_a,D_b>, so that the result carries
    relative (not absolute) rounding error.  This is the quantity the
    descent test of ADAP-FISTA step 2 and the inequality of ADAP-AIPP
    step 2 compare; evaluating g(Y) and g(X) separately and subtracting
    loses all accuracy once the steps become small.
    Returns (dg, rY) with rY = A(YY^T) - b.
    """
    D = Y - X
    ell, a, b, v = constraint_entries(inst)
    dT = np.bincount(ell, weights=v * _pair_change(X, Y, D, a, b),
                     minlength=inst.m).astype(np.float64)
    ca, cb, cv = cost_entries(inst)
    dT0 = float(np.dot(cv, _pair_change(X, Y, D, ca, cb))) if cv.shape[0] else 0.0
    if inst.C_J != 0.0:
        sd = D.sum(axis=0)
        dT0 += inst.C_J * float(sd @ (Y.sum(axis=0) + X.sum(axis=0)))
    if inst.C_I != 0.0:
        dT0 += inst.C_I * float(np.sum(D * (Y + X)))
    for l, K, Dl in inst.lr_terms:
        # tr(D_l (Q Q^T - P P^T)) = tr(D_l (Delta Q^T + P Delta^T)),
        # P = K^T X, Q = K^T Y, Delta = K^T D (no cancellation)
        P = K.T @ X
        Dlt = K.T @ D
        ch = float(np.sum(Dl * (Dlt @ (P + Dlt).T + P @ Dlt.T)))
        if l == 0:
            dT0 += ch
        else:
            dT[l - 1] += ch
    if rX is None:
        rX = constraint_map(inst, X) - inst.b
    dg = dT0 + float(p @ dT) + 0.5 * beta * float(dT @ (2.0 * rX + dT))
    return dg, rX + dT


def gradient_matrix_apply(inst, pshift, v):
    """G v with G = C + A*(p') (eq. Grad X Space)."""
    return adjoint_apply(inst, np.concatenate([[1.0], pshift]), v)


# ----------------------------------------------------------------------------
# phase retrieval (Section 5.4): complex factors, FFT operators
# ----------------------------------------------------------------------------


def phase_map(inst, U):
    """[A(UU^H)]_{k,j} = sum_s |FFT(d_k * U_s)_j|^2 for the coded diffraction
    measurements a_{k,j}^H x = FFT(d_k * x)_j of a ``phase`` instance (eq.
    phase retrieval SDP; the FFT is the only library step).  U: n x r
    complex; returns the m = K n values, k-major."""
    U = np.asarray(U, dtype=np.complex128)
    U2 = U if U.ndim == 2 else U[:, None]
    out = np.empty((inst.masks.shape[0], inst.n))
    for k, d in enumerate(inst.masks):
        Y = np.fft.fft(d[:, None] * U2, axis=0)
        out[k] = np.sum(np.abs(Y) ** 2, axis=1)
    return out.ravel()


def phase_adjoint(inst, p, U):
    """A*(p) U = sum_{k,j} p_{k,j} a_{k,j} a_{k,j}^H U for the same
    measurements: sum_k conj(d_k) * F^H (p_k * F (d_k * U)), F^H y = n ifft(y)."""
    U = np.asarray(U, dtype=np.complex128)
    U2 = U if U.ndim == 2 else U[:, None]
    p = np.asarray(p, dtype=np.float64).reshape(inst.masks.shape)
    W = np.zeros_like(U2)
    for k, d in enumerate(inst.masks):
        Y = np.fft.fft(d[:, None] * U2, axis=0) * p[k][:, None]
        W += np.conj(d)[:, None] * (inst.n * np.fft.ifft(Y, axis=0))
    return W if U.ndim == 2 else W[:, 0]


def phase_vectors(inst):
    """The measurement vectors as an m x n array of rows a_i^H (row k n + j
    is the j-th DFT row times diag(d_k)); small instances, brute force."""
    n = inst.n
    t = np.arange(n)
    F = np.exp(-2j * np.pi * np.outer(t, t) / n)
    return np.concatenate([F * d[None, :] for d in inst.masks])


def embed_factor(U):
    """The real factor of the real embedding of a complex factor:
    [[Re U, -Im U], [Im U, Re U]] (2n x 2r), whose Gram is the real form
    [[Re X, -Im X], [Im X, Re X]] of X = UU^H."""
    U = np.asarray(U, dtype=np.complex128)
    return np.block([[U.real, -U.imag], [U.imag, U.real]])


def phase_to_hslr(inst):
    """The phase retrieval SDP as a real SDP on 2n in HSLR form (Section 3.2).
    A Hermitian X is psd iff its real form X_R is, tr X_R = 2 tr X, and
    <a a^H, X> = <(v1 v1^T + v2 v2^T)/2, X_R> with v1 = [Re a; Im a],
    v2 = [-Im a; Re a]; the J-invariant A_R keeps the real relaxation's value
    equal to the complex one.  So C_R = I/2, A_R = K D K^T with K = [v1 v2],
    D = I/2, b unchanged, tau_R^2 = 2 tau^2."""
    from paper_2505_13719_b300 import instances as _I
    n = inst.n
    Ah = phase_vectors(inst)          # rows a^H
    a = np.conj(Ah)                   # rows a
    terms = []
    for i in range(a.shape[0]):
        v1 = np.concatenate([a[i].real, a[i].imag])
        v2 = np.concatenate([-a[i].imag, a[i].real])
        terms.append((i + 1, np.stack([v1, v2], axis=1), 0.5 * np.eye(2)))
    d = np.arange(2 * n)
    sp_upper = (np.zeros(2 * n, np.int64), d, d, np.full(2 * n, 0.5))
    return _I.hslr(2 * n, sp_upper, terms, inst.b, 2.0 * inst.tau2, sense=1.0,
                   name=inst.name + "_real")


# ----------------------------------------------------------------------------
# minimum eigenpair (Alg. 1 step 7; the eigensolver is not specified)
# ----------------------------------------------------------------------------


def splitmix64_uniform(seed: int, count: int) -> np.ndarray:
    """Uniform [-1, 1) doubles from the SplitMix64 generator (Steele, Lea and
    Flood, 2014): state_k = seed + k * 0x9E3779B97F4A7C15, then the
    published 64-bit finaliser; the top 53 bits give u in [0, 1) and the
    value is 2u - 1.  Both the oracle and the library draw Lanczos start
    vectors this way, so a given seed gives the same start vector."""
    M = (1 << 64) - 1
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (np.uint64(seed & M) + k * np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


@dataclass
class EigResult:
    lam: float
    v: np.ndarray
    iters: int
    resid: float
    converged: bool


def lanczos_min_eig(apply_G, n, v0, tol, kmax=300, max_restarts=20):
    """lambda_min(G) and a unit eigenvector (Alg. 1 step 7).

    Reading: the paper does not name its eigensolver.  Lanczos with full
    reorthogonalisation (classical Gram-Schmidt applied twice), started from
    v0; every iteration the k x k tridiagonal is diagonalised and the loop
    stops when the Ritz residual |beta_k s_k| = ||G v - lambda v|| <= tol.
    When kmax steps do not converge, Lanczos restarts from the Ritz vector.
    """
    v = np.asarray(v0, dtype=np.float64).copy()
    total = 0
    lam, res = math.inf, math.inf
    for _restart in range(max_restarts + 1):
        nv = np.linalg.norm(v)
        if nv == 0.0:
            v = np.ones(n)
            nv = math.sqrt(n)
        Q = np.zeros((kmax, n))
        Q[0] = v / nv
        alph, bet = [], []
        done = False
        for k in range(kmax):
            w = apply_G(Q[k])
            total += 1
            a = float(Q[k] @ w)
            w = w - a * Q[k]
            if k > 0:
                w = w - bet[-1] * Q[k - 1]
            for _ in range(2):
                w = w - Q[:k + 1].T @ (Q[:k + 1] @ w)
            bnorm = float(np.linalg.norm(w))
            alph.append(a)
            bet.append(bnorm)
            Tk = np.diag(alph) + np.diag(bet[:-1], 1) + np.diag(bet[:-1], -1)
            evals, evecs = np.linalg.eigh(Tk)
            lam = float(evals[0])
            s = evecs[:, 0]
            res = abs(bnorm * s[-1])
            if res <= tol or bnorm <= 1e-300 or k + 1 == n:
                done = True
                break
            if k + 1 < kmax:
                Q[k + 1] = w / bnorm
        v = Q[:len(alph)].T @ s
        v /= np.linalg.norm(v)
        if done:
            break
    return EigResult(lam=lam, v=v, iters=total, resid=res, converged=res <= tol)


def min_eig(inst, pshift, tol, v0=None, seed=0, kmax=300):
    """Minimum eigenpair of G = C + A*(p') (eq. Grad X Space)."""
    if v0 is None:
        v0 = splitmix64_uniform(seed, inst.n)
    return lanczos_min_eig(lambda x: gradient_matrix_apply(inst, pshift, x),
                           inst.n, v0, tol, kmax=kmax)


# ----------------------------------------------------------------------------
# Frobenius-ball projection
# ----------------------------------------------------------------------------


def project_ball(U, tau):
    """Projection onto B_tau^s = {U : ||U||_F <= tau} (eq. dimensional ball).

    ||U||_F is formed with an exactly rounded sum of the squares
    (math.fsum): a projected point then lies on the sphere to a few units
    of roundoff.  A BLAS dot product of a few 10^5 entries is off by about
    1e-14, and the step-2 tests see that radial error times the radial
    gradient (2n on the theta SDP) as a change of g."""
    nrm = math.sqrt(math.fsum(np.square(U).ravel()))
    return U if nrm <= tau else U * (tau / nrm)


# ----------------------------------------------------------------------------
# ADAP-FISTA (Appendix A.1) and ADAP-AIPP (Appendix A)
# ----------------------------------------------------------------------------


@dataclass
class Options:
    """Parameters of the method.  Reading: sigma, chi, lambda_0, beta_0 and the
    epsilon_t / beta_t schedules are not given in the paper; the defaults
    below are this implementation's choices."""
    tol: float = 1e-5
    sigma: float = 0.3
    chi: float = 0.5
    lambda0: float = 1.0
    # > 0: every ADAP-AIPP call starts at lambda_kappa / beta_t instead of
    # the carried lambda (0: carried, the default reading)
    lambda_kappa: float = 0.0
    beta0: float = 1.0
    beta_max: float = 1e8
    eps_decay: float = 0.5
    eps1_rel: float = 1e-2
    max_outer: int = 300
    max_hlr: int = 100
    max_aipp: int = 20000
    max_fista: int = 400
    lanczos_kmax: int = 300
    lanczos_tol_rel: float = 0.5
    r_cap: int = 64
    seed: int = 0
    time_limit_s: float = 3600.0


@dataclass
class Counters:
    grads: int = 0
    values: int = 0
    fista_iters: int = 0
    aipp_iters: int = 0
    fista_fail: int = 0
    hlr_iters: int = 0
    lanczos_iters: int = 0
    fw_steps: int = 0
    outer: int = 0


class _Subproblem:
    """g_t(U) = L_beta(UU^T; p) on the ball B_tau^s (eq. Lr / g func).

    ``observer`` (None by default) is called as observer(event, data) when a
    step-2 test of ADAP-FISTA or ADAP-AIPP accepts; it only reads, so the
    tests can recheck each accepted inequality in exact arithmetic."""

    def __init__(self, inst, p, beta, cnt, observer=None):
        self.inst, self.p, self.beta, self.cnt = inst, p, beta, cnt
        self.observer = observer

    def grad(self, U):
        self.cnt.grads += 1
        return al_grad(self.inst, U, self.p, self.beta)

    def value(self, U):
        self.cnt.values += 1
        return al_value(self.inst, U, self.p, self.beta)

    def change(self, X, Y, rX):
        self.cnt.values += 1
        return al_value_change(self.inst, X, Y, self.p, self.beta, rX)


def adap_fista(sub, lam, center, mu, L0, opt, tau):
    """ADAP-FISTA (Appendix A.1) on psi_s(u) = lam g(u) + 1/2 ||u - center||^2
    with psi_n = lam * indicator of the ball, started at x0 = center (ADAP-AIPP
    step 1 passes x_0 = W_{j-1}, the prox centre).

    Returns (status, y, L, V, dg) with status "success" or "failure" and
    dg = g(y) - g(center).
    Reading: l_psi(u; x~) is the linearisation psi_s(x~) + <grad psi_s(x~), u - x~>,
    so the step-2 test reads
    psi_s(y) - psi_s(x~) <= <grad psi_s(x~), y - x~> + (1 - chi) L/4 ||y - x~||^2,
    with the left side formed as a difference (al_value_change).
    Reading: V = grad psi_s(y) - grad psi_s(x~) + L (x~ - y); the y-step's
    optimality gives L (x~ - y) - grad psi_s(x~) in N_B(y), so V lies in
    grad psi_s(y) + N_B(y), which is what ADAP-AIPP's R_j needs.
    Reading: more than max_fista iterations count as failure.
    Floating point: when the accepted y equals x_0 within rounding
    (|y - x_0| <= ROUND_SLACK * UNIT_ROUNDOFF * |x_0|), step 4 is not taken
    and the call succeeds: both sides of step 4's inequality are then
    rounding-level numbers, and a "failure" decided by them would halve
    ADAP-AIPP's lambda for nothing (it never grows back).
    """
    cnt = sub.cnt
    x0 = center
    x = x0.copy()
    y = x0.copy()
    A = 0.0
    tk = 1.0
    L = L0
    for _i in range(opt.max_fista):
        cnt.fista_iters += 1
        Ln = L                                                   # step 1
        while True:                                              # step 2
            a = (tk + math.sqrt(tk * tk + 4.0 * tk * A * (Ln - mu))) / (2.0 * (Ln - mu))
            xt = (A * y + a * x) / (A + a)
            gr = sub.grad(xt)
            dpsi_xt = lam * 2.0 * gr.W + (xt - center)
            ynew = project_ball(xt - dpsi_xt / Ln, tau)
            d = ynew - xt
            dg, _ry = sub.change(xt, ynew, gr.resid)
            dpsi = lam * dg + float(np.sum(d * (0.5 * (ynew + xt) - center)))
            slack = ROUND_SLACK * UNIT_ROUNDOFF * lam * gr.mag
            if float(np.sum(dpsi_xt * d)) + (1.0 - opt.chi) * Ln / 4.0 * float(np.sum(d * d)) \
                    >= dpsi - slack:
                if sub.observer is not None:
                    sub.observer("fista_step2", dict(xt=xt, y=ynew, center=center, lam=lam,
                                                     L=Ln, chi=opt.chi, slack=slack,
                                                     mag=gr.mag))
                break
            Ln *= 2.0
            if Ln > 1e30:
                cnt.fista_fail += 1
                return "failure", None, Ln, None, None
        A_new = A + a                                            # step 3
        tk_new = tk + a * mu
        s = (Ln - mu) * (xt - ynew)
        x = (mu * a * ynew + tk * x - a * s) / tk_new
        dy0 = float(np.sum((ynew - x0) ** 2))
        # y equal to x_0 within rounding: x_0 is the prox point to working
        # precision, and step 4 would compare two rounding-level numbers
        at_x0 = dy0 <= (ROUND_SLACK * UNIT_ROUNDOFF) ** 2 * float(np.sum(x0 * x0))
        if not at_x0 and dy0 < opt.chi * A_new * Ln * float(np.sum((ynew - xt) ** 2)):  # step 4
            cnt.fista_fail += 1
            return "failure", None, Ln, None, None
        if at_x0 or math.sqrt(float(np.sum(s * s))) <= opt.sigma * math.sqrt(dy0):  # step 5
            gy = sub.grad(ynew)
            dpsi_y = lam * 2.0 * gy.W + (ynew - center)
            V = dpsi_y - dpsi_xt + Ln * (xt - ynew)
            dg0, _ = sub.change(center, ynew, None)
            return "success", ynew, Ln, V, (dg0, gy.mag)
        y, A, tk, L = ynew, A_new, tk_new, Ln
    cnt.fista_fail += 1
    return "failure", None, L, None, None


@dataclass
class AippState:
    lam: float
    Mbar: float = 1.0


def adap_aipp(sub, W0, rho, state, opt, tau):
    """ADAP-AIPP (Appendix A): find (W, R) with R in grad g(W) + N_B(W),
    ||R||_F <= rho and g(W) <= g(W0).

    Reading: M_j = max(1, Mbar_{j-1} / 2) within the allowed [1, Mbar_{j-1}];
    lambda carries over between calls (it only ever halves, step 2).
    Floating point: the step-2 inequality (and ADAP-FISTA's step-2 test)
    accepts a violation up to ROUND_SLACK * UNIT_ROUNDOFF * lam * (sum of
    the magnitudes of g's terms), the size of rounding in g; a prox step that
    leaves W unchanged ends the method (no further progress is possible).
    The step-2 inequality lam g(W_{j-1}) - [lam g(W) + 1/2 ||W - W_{j-1}||^2]
    >= V . (W_{j-1} - W) is evaluated with g(W) - g(W_{j-1}) formed as a
    difference (al_value_change).
    """
    cnt = sub.cnt
    Wprev = W0
    R = np.zeros_like(W0)
    for _j in range(opt.max_aipp):
        cnt.aipp_iters += 1
        stalled = False
        while True:
            Mlow = max(1.0, state.Mbar / 2.0)                          # step 1
            st, W, L, V, dgm = adap_fista(sub, state.lam, Wprev, 0.5, Mlow, opt, tau)
            if st == "success":
                dg, mag = dgm
                D = W - Wprev
                d2 = float(np.sum(D * D))
                stalled = d2 == 0.0
                lhs = -state.lam * dg - 0.5 * d2
                slack = ROUND_SLACK * UNIT_ROUNDOFF * state.lam * mag
                if stalled or lhs >= -float(np.sum(V * D)) - slack:     # step 2
                    if sub.observer is not None:
                        sub.observer("aipp_step2", dict(Wprev=Wprev, W=W, V=V, lam=state.lam,
                                                        stalled=stalled, slack=slack, mag=mag))
                    break
            state.lam /= 2.0
            if state.lam < 1e-30:
                raise RuntimeError("ADAP-AIPP: prox stepsize underflow")
        state.Mbar = L
        R = (V + Wprev - W) / state.lam                                 # eq. Rj def
        if math.sqrt(float(np.sum(R * R))) <= rho or stalled:           # step 3
            return W, R
        Wprev = W                                                       # step 4
    return Wprev, R


# ----------------------------------------------------------------------------
# HLR and the AL outer loop (Alg. 1)
# ----------------------------------------------------------------------------


@dataclass
class SolveResult:
    U: np.ndarray
    p: np.ndarray
    theta: float
    pval: float
    dval: float
    user_value: float
    rel_primal: float
    rel_gap: float
    rel_dual: float
    kkt: float
    lam_min_S: float
    rank: int
    converged: bool
    counters: Counters
    seconds: float
    history: list = field(default_factory=list)


def fw_step(inst, Y, y, theta, gap, beta, tau2):
    """Frank-Wolfe step of HLR (eqs. FW stepsize and tilde Y).

    alpha = min{ (G.YY^T + tau^2 theta) / (beta ||A(YY^T) - A(tau^2 yy^T)||^2), 1 }
    Y~ = tau y if alpha = 1, else [sqrt(1 - alpha) Y, sqrt(alpha) tau y].
    Reading: the garbled 'tau yy^T' of the X-space remark is tau^2 yy^T, as
    in eq. FW stepsize.  Reading: when theta = 0 (y = 0) no zero column is
    appended; Y is only scaled by sqrt(1 - alpha) (or set to 0 if alpha = 1).
    """
    tau = math.sqrt(tau2)
    AY = constraint_map(inst, Y)
    Ay = constraint_map(inst, y[:, None]) * tau2
    diff = AY - Ay
    denom = beta * float(diff @ diff)
    alpha = 1.0 if denom <= 0.0 else min(gap / denom, 1.0)
    if theta > 0.0:
        if alpha >= 1.0:
            return tau * y[:, None], alpha
        return np.hstack([math.sqrt(1.0 - alpha) * Y, math.sqrt(alpha) * tau * y[:, None]]), alpha
    if alpha >= 1.0:
        return np.zeros((inst.n, 1)), alpha
    return math.sqrt(1.0 - alpha) * Y, alpha


def c_norm1(inst):
    """Induced 1-norm of C = C_sparse + C_J 11^T + C_I I (largest absolute
    column sum).  Reading: eq. termination2's ||C||_1 is taken as the
    induced norm."""
    n = inst.n
    if any(l == 0 for l, _K, _D in inst.lr_terms):
        # a low-rank part in C: the induced norm of the dense matrix
        # (small problems only: n^2 entries)
        if n > 20000:
            raise ValueError("||C||_1 with a low-rank C is formed densely: n too large")
        G = dense_adjoint(inst, np.concatenate([[1.0], np.zeros(inst.m)]))
        return float(np.abs(G).sum(axis=0).max()) if n else 0.0
    a, b, v = cost_entries(inst)
    M = sp.coo_matrix((v, (a, b)), shape=(n, n)).tocsc()
    M.sum_duplicates()
    rows = M.indices.astype(np.int64)
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(M.indptr))
    on_diag = rows == cols
    absval = np.abs(M.data + inst.C_J + np.where(on_diag, inst.C_I, 0.0))
    col = np.bincount(cols, weights=absval, minlength=n).astype(np.float64)
    stored = np.diff(M.indptr).astype(np.float64)
    diag_in = np.bincount(cols[on_diag], minlength=n) > 0
    # entries outside the stored pattern hold C_J (+ C_I on the diagonal)
    col += abs(inst.C_J) * (n - stored - np.where(diag_in, 0.0, 1.0))
    col += np.where(diag_in, 0.0, abs(inst.C_J + inst.C_I))
    return float(col.max()) if n else 0.0


def kkt_measures(inst, U, p, theta, lam_min_S, cnorm):
    """Relative KKT residuals of eq. termination2:
    max{ ||A X - b|| / (1 + ||b||_1),
         |pval - dval| / (1 + |pval| + |dval|),
         max(0, -lambda_min(S)) / (1 + ||C||_1) },
    pval = C.X, dval = -b^T p - tau^2 theta, S = C + A*p + theta I."""
    T = eval_A_tilde(inst, U)
    r = T[1:] - inst.b
    pval = T[0]
    dval = -float(inst.b @ p) - inst.tau2 * theta
    rp = float(np.linalg.norm(r)) / (1.0 + float(np.abs(inst.b).sum()))
    rg = abs(pval - dval) / (1.0 + abs(pval) + abs(dval))
    rd = max(0.0, -lam_min_S) / (1.0 + cnorm)
    return pval, dval, rp, rg, rd


def hallar_solve(inst, U0, p0=None, opt: Options | None = None, log=None):
    """HALLaR (Alg. 1): inexact AL on (P) with the HLR inner method.

    Readings (the paper leaves these open):
    * epsilon_t = max(eps_floor, eps_1 * eps_decay^(t-1)) with
      eps_1 = eps1_rel (1 + tau^2 ||C||_1) (a bound on |C.X| over the
      spectraplex) and eps_floor = tol/2 (1 + |pval|);
      the nonconvex solver gets rho_t = epsilon_t / tau so that
      <R, Y> <= epsilon_t on the ball (Alg. 1 step 6 passes epsilon_t).
    * beta_t: start at beta0; after each dual update, double beta (capped at
      beta_max (1 + ||C||_1)) when ||r_t|| > ||r_{t-1}|| / 4 while the
      relative primal infeasibility is still above tol (a LANCELOT-style
      test: the penalty grows only while infeasibility is the obstacle).
      The cap is in units of 1 + ||C||_1: scaling C by s leaves the AL
      iterates unchanged when beta and p scale by s too, so an absolute cap
      would stop the theta SDP (||C||_1 = n) before its multipliers reach
      their optimal size, which grows like n / degree.
    * termination: eq. termination2 at relative tolerance tol.
    * U0 outside the ball is projected onto it.
    """
    opt = opt or Options()
    t0 = time.perf_counter()
    cnt = Counters()
    tau2 = inst.tau2
    tau = math.sqrt(tau2)
    U = project_ball(np.asarray(U0, dtype=np.float64), tau)
    p = np.zeros(inst.m) if p0 is None else np.asarray(p0, dtype=np.float64).copy()
    beta = opt.beta0
    aipp = AippState(lam=opt.lambda0)
    cnorm = c_norm1(inst)
    eps1 = opt.eps1_rel * (1.0 + tau2 * cnorm)
    prev_rnorm = math.inf
    v_prev = None
    history = []
    theta = 0.0
    lam_min_S = 0.0
    res = None
    for t in range(1, opt.max_outer + 1):
        cnt.outer += 1
        pval_now = cost_dot(inst, U)
        eps_floor = 0.5 * opt.tol * (1.0 + abs(pval_now))
        eps_t = max(eps_floor, eps1 * opt.eps_decay ** (t - 1))
        rho_t = eps_t / max(tau, 1e-300)
        sub = _Subproblem(inst, p, beta, cnt)
        Yt = U
        for _h in range(opt.max_hlr):                                   # HLR
            cnt.hlr_iters += 1
            if opt.lambda_kappa > 0.0:
                aipp.lam = opt.lambda_kappa / beta
            Y, _R = adap_aipp(sub, Yt, rho_t, aipp, opt, tau)      # step 6
            gr = al_grad(inst, Y, p, beta)                               # step 7
            GdotX = float(np.sum(gr.W * Y))
            eig_tol = opt.lanczos_tol_rel * eps_t / tau2
            v0 = splitmix64_uniform(opt.seed + 7919 * cnt.hlr_iters, inst.n)
            if v_prev is not None:
                v0 = v_prev + 0.1 * v0 / math.sqrt(inst.n)
            er = min_eig(inst, gr.pshift, eig_tol, v0=v0, kmax=opt.lanczos_kmax)
            cnt.lanczos_iters += er.iters
            v_prev = er.v
            theta = max(-er.lam, 0.0)                                    # eq. FW subproblem
            y = er.v if theta > 0.0 else np.zeros(inst.n)
            gap = GdotX + tau2 * theta
            lam_min_S = er.lam + theta
            if gap <= eps_t:                                             # step 8
                break
            Yt, _alpha = fw_step(inst, Y, y, theta, gap, beta, tau2)     # step 11
            cnt.fw_steps += 1
            if Yt.shape[1] > opt.r_cap:
                Yt = trim_rank(Yt, opt.r_cap)
        U = Y                                                            # step 13
        r = constraint_map(inst, U) - inst.b
        p = p + beta * r                                                 # step 14
        pval, dval, rp, rg, rd = kkt_measures(inst, U, p, theta, lam_min_S, cnorm)
        kkt = max(rp, rg, rd)
        history.append(dict(t=t, rank=U.shape[1], beta=beta, eps=eps_t, pval=pval,
                            dval=dval, rp=rp, rg=rg, rd=rd,
                            grads=cnt.grads, lanczos=cnt.lanczos_iters))
        if log:
            log(history[-1])
        if kkt <= opt.tol:                                               # step 15
            res = (pval, dval, rp, rg, rd, True)
            break
        rnorm = float(np.linalg.norm(r))
        if rp > opt.tol and rnorm > 0.25 * prev_rnorm:
            beta = min(2.0 * beta, opt.beta_max * (1.0 + cnorm))
        prev_rnorm = rnorm
        if time.perf_counter() - t0 > opt.time_limit_s:
            break
    if res is None:
        res = (pval, dval, rp, rg, rd, False)
    pval, dval, rp, rg, rd, conv = res
    return SolveResult(U=U, p=p, theta=theta, pval=pval, dval=dval,
                       user_value=inst.sense * pval, rel_primal=rp, rel_gap=rg,
                       rel_dual=rd, kkt=max(rp, rg, rd), lam_min_S=lam_min_S,
                       rank=U.shape[1], converged=conv, counters=cnt,
                       seconds=time.perf_counter() - t0, history=history)


def trim_rank(Y, r_cap):
    """Reading (not in the paper): when the factor would exceed r_cap columns,
    keep the r_cap leading directions of YY^T (eigenvectors of the Gram
    Y^T Y), i.e. Y <- Y Q_k for the top-k eigenvectors Q_k."""
    Gm = Y.T @ Y
    w, Q = np.linalg.eigh(Gm)
    return Y @ Q[:, ::-1][:, :r_cap]


# ----------------------------------------------------------------------------
# consumers of a solved factor (not in the paper)
# ----------------------------------------------------------------------------


def maxcut_round(inst, U, G):
    """Goemans-Williamson hyperplane rounding of a Max-Cut factor (not in the
    paper, which stops at the SDP solution).  For each normal g (a row of
    G): x = sign(U g) with sign(0) = +1, and its cut value -x^T C x, which is
    (1/4) x^T L x, the weight of the edges x cuts, for C = -L/4.
    Returns (cuts [trials], X [trials x n] of +-1)."""
    U = np.asarray(U, dtype=np.float64)
    G = np.atleast_2d(np.asarray(G, dtype=np.float64))
    X = np.where(U @ G.T < 0.0, -1.0, 1.0).T
    cuts = np.array([-cost_dot(inst, x[:, None]) for x in X])
    return cuts, X


def factor_entries(U, a, b):
    """X_ab = <U_a, U_b> for listed index pairs (X = UU^T); for matrix
    completion (eq. matcomp-sdp) the recovered matrix is M^_ij = X_{i, n1+j}."""
    U = np.asarray(U, dtype=np.float64)
    return _pair_dots_mixed(U, U, np.asarray(a, dtype=np.int64), np.asarray(b, dtype=np.int64))
