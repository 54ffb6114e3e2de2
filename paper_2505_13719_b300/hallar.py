"""Thin ctypes binding of the C ABI in include/hallar.h (argument marshalling only).

Every function keeps the C name.  Arrays may be NumPy arrays (host memory)
or CUDA torch tensors (device memory); the library tells them apart.  Factor
arrays hold float64 for HALLAR_FP64 handles and float32 for HALLAR_MIXED.
There is no CPU fallback: if ``libhallar.so`` is missing or fails to load,
importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhallar.so")

HALLAR_OK, HALLAR_EINVAL, HALLAR_ENOMEM, HALLAR_ECUDA = 0, 1, 2, 3
HALLAR_ENOTCONV, HALLAR_ETIMEOUT, HALLAR_ERANK, HALLAR_ENUMERIC = 4, 5, 6, 7
HALLAR_DIAG, HALLAR_EDGE, HALLAR_OBSERVED = 0, 1, 2
HALLAR_FP64, HALLAR_MIXED = 0, 1
FAMILY = {"diag": HALLAR_DIAG, "edge": HALLAR_EDGE, "observed": HALLAR_OBSERVED}


def _family_code(family):
    """hallar_family of a family name; general HSLR problems (family
    "hslr") have no device kernels yet and are refused here."""
    if not isinstance(family, str):
        return int(family)
    if family not in FAMILY:
        raise ValueError(f"family {family!r}: the device library implements "
                         f"{', '.join(FAMILY)} only")
    return FAMILY[family]

EXPORTED = ("hallar_default_options", "hallar_create", "hallar_eval_A", "hallar_grad",
            "hallar_value_change", "hallar_trim_rank", "hallar_maxcut_round",
            "hallar_factor_entries", "hallar_min_eig", "hallar_solve", "hallar_get_solution", "hallar_get_sizes",
            "hallar_destroy", "hallar_last_error", "hallar_status_string", "hallar_profile",
            "hallar_profile_sampling", "hallar_grad_diag_noalloc", "hallar_solve_footprint", "hallar_server_create",
            "hallar_server_submit", "hallar_server_wait", "hallar_server_get_stats",
            "hallar_server_destroy", "hallar_server_last_error", "hallar_batch_create",
            "hallar_batch_layout", "hallar_batch_grad", "hallar_batch_shape",
            "hallar_batch_destroy", "hallar_batch_last_error", "hallar_check_problem",
            "hallar_merge_general")


class hallar_options(C.Structure):
    _fields_ = [("tol", C.c_double), ("sigma", C.c_double), ("chi", C.c_double),
                ("lambda0", C.c_double), ("beta0", C.c_double), ("beta_max", C.c_double),
                ("eps_decay", C.c_double), ("eps1_rel", C.c_double),
                ("lanczos_tol_rel", C.c_double), ("time_limit_s", C.c_double),
                ("lambda_kappa", C.c_double),
                ("r_cap", C.c_int32), ("max_outer", C.c_int32), ("max_hlr", C.c_int32),
                ("max_aipp", C.c_int32), ("max_fista", C.c_int32),
                ("lanczos_kmax", C.c_int32), ("precision", C.c_int32),
                ("verbose", C.c_int32), ("promote", C.c_int32), ("seed", C.c_uint64), ("stream", C.c_void_p)]


class hallar_result(C.Structure):
    _fields_ = [("pval", C.c_double), ("dval", C.c_double), ("theta", C.c_double),
                ("lam_min_S", C.c_double), ("rel_primal", C.c_double),
                ("rel_gap", C.c_double), ("rel_dual", C.c_double), ("kkt", C.c_double),
                ("beta", C.c_double), ("seconds", C.c_double), ("rank", C.c_int32),
                ("converged", C.c_int32), ("outer_iters", C.c_int32),
                ("hlr_iters", C.c_int32), ("aipp_iters", C.c_int32),
                ("fista_iters", C.c_int32), ("fista_failures", C.c_int32),
                ("lanczos_iters", C.c_int32), ("fw_steps", C.c_int32), ("trims", C.c_int32),
                ("promoted_at", C.c_int32), ("grad_evals", C.c_int64), ("value_evals", C.c_int64),
                ("kernel_launches", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class hallar_server_options(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_double), ("max_inflight", C.c_int32),
                ("device", C.c_int32)]


class hallar_request(C.Structure):
    _fields_ = [("n", C.c_int64), ("n1", C.c_int64), ("C_rowptr", C.c_void_p),
                ("C_col", C.c_void_p), ("C_val", C.c_void_p), ("C_nnz", C.c_int64),
                ("C_J", C.c_double), ("C_I", C.c_double), ("family", C.c_int32),
                ("m_pairs", C.c_int64), ("cons_i", C.c_void_p), ("cons_j", C.c_void_p),
                ("has_trace_row", C.c_int32), ("b", C.c_void_p), ("tau2", C.c_double),
                ("U0", C.c_void_p), ("r0", C.c_int32), ("opt", hallar_options)]


class hallar_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("failed", C.c_int64), ("queued", C.c_int64), ("inflight", C.c_int64),
                ("max_inflight_seen", C.c_int64), ("bytes_inflight", C.c_double),
                ("peak_bytes_inflight", C.c_double), ("p50_latency_s", C.c_double),
                ("p99_latency_s", C.c_double), ("mean_latency_s", C.c_double),
                ("max_latency_s", C.c_double), ("first_submit_to_last_done_s", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhallar.so not built ({LIB_PATH}); run "
                          "python -m paper_2505_13719_b300.build")
    lib = C.CDLL(LIB_PATH)
    P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    sig = {
        "hallar_default_options": ([P], C.c_int),
        "hallar_create": ([I64, I64, P, P, P, D, D, I32, I64, P, P, I32, P, D, P,
                           C.POINTER(C.c_void_p)], C.c_int),
        "hallar_eval_A": ([P, P, I32, P], C.c_int),
        "hallar_grad": ([P, P, I32, P, D, P, P, P], C.c_int),
        "hallar_value_change": ([P, P, P, I32, P, D, P, P, P], C.c_int),
        "hallar_trim_rank": ([P, P, I32, I32, P, P], C.c_int),
        "hallar_maxcut_round": ([P, P, I32, P, I32, P, P], C.c_int),
        "hallar_factor_entries": ([P, P, I32, P, P, I64, P], C.c_int),
        "hallar_min_eig": ([P, P, D, I32, P, P, P, P, P], C.c_int),
        "hallar_solve": ([P, P, I32, P, P], C.c_int),
        "hallar_get_solution": ([P, P, I32, P, P], C.c_int),
        "hallar_get_sizes": ([P, P, P, P, P], C.c_int),
        "hallar_profile": ([P, I32, P, P, P, P], C.c_int),
        "hallar_profile_sampling": ([P, I32], C.c_int),
        "hallar_grad_diag_noalloc": ([I64, I32, P, P, P, P, P, P, D, P, P, P, P, P, C.c_char_p,
                                      I32], C.c_int),
        "hallar_solve_footprint": ([P], I64),
        "hallar_server_create": ([P, C.POINTER(C.c_void_p)], C.c_int),
        "hallar_server_submit": ([P, P, C.POINTER(I64)], C.c_int),
        "hallar_server_wait": ([P, I64, D, P, P, I32, P, P, P], C.c_int),
        "hallar_server_get_stats": ([P, P], C.c_int),
        "hallar_server_destroy": ([P], None),
        "hallar_server_last_error": ([P], C.c_char_p),
        "hallar_merge_general": ([I64, I64, I64, P, P, P, P, P, P, P, P, P, P, P], I32),
        "hallar_check_problem": ([I64, I64, P, P, P, D, D, I32, I64, P, P, I32, P, D, P, P, P],
                                 C.c_int),
        "hallar_batch_create": ([I32, P, I32, I32, P, C.POINTER(C.c_void_p)], C.c_int),
        "hallar_batch_layout": ([P, P, P, P, P], C.c_int),
        "hallar_batch_grad": ([P, P, I32, P, P, P, P, P], C.c_int),
        "hallar_batch_shape": ([P, I32, P, P, P], C.c_int),
        "hallar_batch_destroy": ([P], None),
        "hallar_batch_last_error": ([P], C.c_char_p),
        "hallar_destroy": ([P], None),
        "hallar_last_error": ([P], C.c_char_p),
        "hallar_status_string": ([C.c_int], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


class HallarError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_lib.hallar_status_string(status).decode()}: {msg}")
        self.status = status


def _ptr(a):
    """Address of a NumPy array or torch tensor (None for None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data if a.size else None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _check(status, h=None, allow=()):
    if status != HALLAR_OK and status not in allow:
        raise HallarError(status, _lib.hallar_last_error(h).decode())
    return status


def hallar_default_options(**overrides) -> hallar_options:
    o = hallar_options()
    _check(_lib.hallar_default_options(C.byref(o)))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def hallar_create(n, n1, C_rowptr, C_col, C_val, C_J, C_I, family, cons_i, cons_j,
                  has_trace_row, b, tau2, opt: hallar_options | None = None):
    """Create a handle from host arrays (see hallar_create in hallar.h)."""
    fam = _family_code(family)
    rp = None if C_rowptr is None else np.ascontiguousarray(C_rowptr, dtype=np.int64)
    ci = np.ascontiguousarray([] if C_col is None else C_col, dtype=np.int32)
    cv = np.ascontiguousarray([] if C_val is None else C_val, dtype=np.float64)
    pi = np.ascontiguousarray(cons_i, dtype=np.int32)
    pj = np.ascontiguousarray(cons_j, dtype=np.int32)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    m_pairs = 0 if fam == HALLAR_DIAG else int(pi.shape[0])
    h = C.c_void_p()
    st = _lib.hallar_create(int(n), int(n1), _ptr(rp), _ptr(ci), _ptr(cv), float(C_J),
                            float(C_I), fam, m_pairs, _ptr(pi), _ptr(pj),
                            int(bool(has_trace_row)), _ptr(bb), float(tau2),
                            C.byref(opt) if opt is not None else None, C.byref(h))
    _check(st, None)
    return h


def hallar_check_problem(n, n1, C_rowptr, C_col, C_val, C_J, C_I, family, cons_i, cons_j,
                         has_trace_row, b, tau2):
    """Host-only validation and merge (see hallar.h): (m, nnz_merged, c_norm1)."""
    fam = _family_code(family)
    rp = None if C_rowptr is None else np.ascontiguousarray(C_rowptr, dtype=np.int64)
    ci = np.ascontiguousarray([] if C_col is None else C_col, dtype=np.int32)
    cv = np.ascontiguousarray([] if C_val is None else C_val, dtype=np.float64)
    pi = np.ascontiguousarray(cons_i, dtype=np.int32)
    pj = np.ascontiguousarray(cons_j, dtype=np.int32)
    bb = np.ascontiguousarray(b, dtype=np.float64)
    m_pairs = 0 if fam == HALLAR_DIAG else int(pi.shape[0])
    m, nnz, cn = C.c_int64(), C.c_int64(), C.c_double()
    st = _lib.hallar_check_problem(int(n), int(n1), _ptr(rp), _ptr(ci), _ptr(cv), float(C_J),
                                   float(C_I), fam, m_pairs, _ptr(pi), _ptr(pj),
                                   int(bool(has_trace_row)), _ptr(bb), float(tau2),
                                   C.byref(m), C.byref(nnz), C.byref(cn))
    _check(st, None)
    return m.value, nnz.value, cn.value


def hallar_merge_general(n, m, ell, ii, jj, val):
    """Merged support of general sparse data matrices (see hallar.h):
    (rowptr, col, lptr, lidx, lval), the pattern S as CSR over both triangles
    and, per stored entry, its list L_ij of (matrix, value).  Entries are
    (ell, ii, jj, val) with ii <= jj (upper triangles), ell = 0 for C."""
    el = np.ascontiguousarray(ell, dtype=np.int32)
    ia = np.ascontiguousarray(ii, dtype=np.int32)
    ja = np.ascontiguousarray(jj, dtype=np.int32)
    va = np.ascontiguousarray(val, dtype=np.float64)
    k = int(el.shape[0])
    if not (ia.shape[0] == ja.shape[0] == va.shape[0] == k):
        raise ValueError("entry arrays differ in length")
    ns, nl = C.c_int64(), C.c_int64()
    st = _lib.hallar_merge_general(int(n), int(m), k, _ptr(el), _ptr(ia), _ptr(ja), _ptr(va),
                                   C.byref(ns), C.byref(nl), None, None, None, None, None)
    _check(st, None)
    if ns.value == 0:  # nothing stored: the empty pattern
        return (np.zeros(int(n) + 1, dtype=np.int64), np.zeros(0, np.int32),
                np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float64))
    rowptr = np.empty(int(n) + 1, dtype=np.int64)
    col = np.empty(ns.value, dtype=np.int32)
    lptr = np.empty(ns.value + 1, dtype=np.int64)
    lidx = np.empty(nl.value, dtype=np.int32)
    lval = np.empty(nl.value, dtype=np.float64)
    st = _lib.hallar_merge_general(int(n), int(m), k, _ptr(el), _ptr(ia), _ptr(ja), _ptr(va),
                                   None, None, _ptr(rowptr), _ptr(col), _ptr(lptr), _ptr(lidx),
                                   _ptr(lval))
    _check(st, None)
    return rowptr, col, lptr, lidx, lval


def check_instance(inst):
    return hallar_check_problem(inst.n, inst.n1, inst.C_rowptr, inst.C_col, inst.C_val,
                                inst.C_J, inst.C_I, inst.family, inst.cons_i, inst.cons_j,
                                inst.has_trace_row, inst.b, inst.tau2)


def hallar_eval_A(h, U, r, T):
    return _check(_lib.hallar_eval_A(h, _ptr(U), int(r), _ptr(T)), h)


def hallar_grad(h, U, r, p, beta, W, resid=None):
    """Returns g(U); W (and resid) are written in place."""
    g = C.c_double()
    _check(_lib.hallar_grad(h, _ptr(U), int(r), _ptr(p), float(beta), _ptr(W), C.byref(g),
                            _ptr(resid)), h)
    return g.value


def hallar_value_change(h, X, Y, r, p, beta, rX=None, rY=None):
    """Returns g(Y) - g(X); rY (if given) receives A(YY^T) - b."""
    dg = C.c_double()
    _check(_lib.hallar_value_change(h, _ptr(X), _ptr(Y), int(r), _ptr(p), float(beta), _ptr(rX),
                                    C.byref(dg), _ptr(rY)), h)
    return dg.value


def hallar_trim_rank(h, Y, r, k, Yout, eigs=None):
    """Yout = Y Q_k (k leading Gram eigenvectors); eigs (host float64 [r]) optional."""
    return _check(_lib.hallar_trim_rank(h, _ptr(Y), int(r), int(k), _ptr(Yout), _ptr(eigs)), h)


def hallar_maxcut_round(h, U, r, G, x_best=None):
    """Hyperplane rounding with the normals G [trials x r]; returns the
    per-trial cut values (x_best, int8 [n], receives the best signs)."""
    G = np.ascontiguousarray(G, dtype=np.float64) if isinstance(G, np.ndarray) else G
    trials = int(G.shape[0])
    cuts = np.empty(trials)
    _check(_lib.hallar_maxcut_round(h, _ptr(U), int(r), _ptr(G), trials, _ptr(x_best),
                                    _ptr(cuts)), h)
    return cuts


def hallar_factor_entries(h, U, r, a, b, out):
    """out[t] = <U_a[t], U_b[t]> (int32 index arrays, host or device)."""
    return _check(_lib.hallar_factor_entries(h, _ptr(U), int(r), _ptr(a), _ptr(b),
                                             int(len(a)), _ptr(out)), h)


def hallar_min_eig(h, pshift, tol, kmax, v0=None, v=None):
    """Returns (lambda_min, iterations, residual, converged)."""
    lam = C.c_double()
    it = C.c_int32()
    res = C.c_double()
    st = _lib.hallar_min_eig(h, _ptr(pshift), float(tol), int(kmax), _ptr(v0), C.byref(lam),
                             _ptr(v), C.byref(it), C.byref(res))
    _check(st, h, allow=(HALLAR_ENOTCONV,))
    return lam.value, it.value, res.value, st == HALLAR_OK


def hallar_solve(h, U0, r0, p0=None):
    """Returns (status, hallar_result); HALLAR_ENOTCONV / HALLAR_ETIMEOUT do not raise."""
    res = hallar_result()
    st = _lib.hallar_solve(h, _ptr(U0), int(r0), _ptr(p0), C.byref(res))
    _check(st, h, allow=(HALLAR_ENOTCONV, HALLAR_ETIMEOUT))
    return st, res


def hallar_get_solution(h, U=None, r_capacity=0, p=None):
    """Copies the last solution out; returns its rank."""
    rank = C.c_int32()
    _check(_lib.hallar_get_solution(h, _ptr(U), int(r_capacity), _ptr(p), C.byref(rank)), h)
    return rank.value


def hallar_get_sizes(h):
    n, m, nnz = C.c_int64(), C.c_int64(), C.c_int64()
    prec = C.c_int32()
    _check(_lib.hallar_get_sizes(h, C.byref(n), C.byref(m), C.byref(nnz), C.byref(prec)), h)
    return n.value, m.value, nnz.value, prec.value


def hallar_profile(h, op, padded=False):
    """op 1: clear and start kernel timing, 2: stop, 0: read.  Returns
    (ms[3], launches[3], bytes[3]) for the fused operator, value-change and
    Lanczos kernel classes, plus bytes_padded[3] when padded is true."""
    ms = (C.c_double * 3)()
    nl = (C.c_int64 * 3)()
    by = (C.c_double * 3)()
    bp = (C.c_double * 3)()
    _check(_lib.hallar_profile(h, int(op), ms, nl, by, bp), h)
    if padded:
        return list(ms), list(nl), list(by), list(bp)
    return list(ms), list(nl), list(by)


def hallar_profile_sampling(h, every):
    """Time only every `every`-th launch of each kernel class."""
    return _check(_lib.hallar_profile_sampling(h, int(every)), h)


def hallar_grad_diag_noalloc(n, r, rowptr, col, cval, cdiag, b, p, beta, U, W, resid, g_out,
                             stream=None):
    """Allocation-free fused gradient of a diagonal-family problem from
    caller-owned device arrays (see hallar.h); enqueues on `stream` (a
    cudaStream_t as an int, or None) and returns without synchronising."""
    err = C.create_string_buffer(256)
    st = _lib.hallar_grad_diag_noalloc(int(n), int(r), _ptr(rowptr), _ptr(col), _ptr(cval),
                                       _ptr(cdiag), _ptr(b), _ptr(p), float(beta), _ptr(U),
                                       _ptr(W), _ptr(resid), _ptr(g_out), stream, err, 256)
    if st != HALLAR_OK:
        raise HallarError(st, err.value.decode())
    return st


def hallar_destroy(h):
    if h is not None:
        _lib.hallar_destroy(h)


def hallar_last_error(h=None) -> str:
    return _lib.hallar_last_error(h).decode()


# ---------------------------------------------------------------------------
# convenience: a handle built from an instances.Instance
# ---------------------------------------------------------------------------
@dataclass
class Handle:
    h: object
    n: int
    m: int
    precision: int

    @property
    def dtype(self):
        return np.float32 if self.precision == HALLAR_MIXED else np.float64

    def close(self):
        if self.h is not None:
            hallar_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def create_from_instance(inst, precision=HALLAR_FP64, **options) -> Handle:
    opt = hallar_default_options(precision=precision, **options)
    h = hallar_create(inst.n, inst.n1, inst.C_rowptr, inst.C_col, inst.C_val, inst.C_J,
                      inst.C_I, inst.family, inst.cons_i, inst.cons_j, inst.has_trace_row,
                      inst.b, inst.tau2, opt)
    return Handle(h=h, n=inst.n, m=inst.m, precision=precision)


# ---------------------------------------------------------------------------
# serving engine
# ---------------------------------------------------------------------------
def request_from_instance(inst, U0, precision=HALLAR_FP64, **options):
    """A hallar_request for an instances.Instance and a host start factor.
    Returns (request, keep): `keep` holds the arrays the request points to;
    it must stay alive until hallar_server_submit returns."""
    opt = hallar_default_options(precision=precision, **options)
    fam = _family_code(inst.family)
    dt = np.float32 if precision == HALLAR_MIXED else np.float64
    keep = {
        "rp": None if inst.C_rowptr is None else np.ascontiguousarray(inst.C_rowptr, np.int64),
        "ci": np.ascontiguousarray([] if inst.C_col is None else inst.C_col, np.int32),
        "cv": np.ascontiguousarray([] if inst.C_val is None else inst.C_val, np.float64),
        "pi": np.ascontiguousarray(inst.cons_i, np.int32),
        "pj": np.ascontiguousarray(inst.cons_j, np.int32),
        "b": np.ascontiguousarray(inst.b, np.float64),
        "U0": np.ascontiguousarray(U0, dt),
    }
    q = hallar_request()
    q.n, q.n1 = int(inst.n), int(inst.n1)
    q.C_rowptr = _ptr(keep["rp"])
    q.C_col, q.C_val = _ptr(keep["ci"]), _ptr(keep["cv"])
    q.C_nnz = 0 if keep["rp"] is None else int(keep["rp"][-1])
    q.C_J, q.C_I = float(inst.C_J), float(inst.C_I)
    q.family = fam
    q.m_pairs = 0 if fam == HALLAR_DIAG else int(keep["pi"].shape[0])
    q.cons_i, q.cons_j = _ptr(keep["pi"]), _ptr(keep["pj"])
    q.has_trace_row = int(bool(inst.has_trace_row))
    q.b = _ptr(keep["b"])
    q.tau2 = float(inst.tau2)
    q.U0 = _ptr(keep["U0"])
    q.r0 = int(keep["U0"].shape[1])
    q.opt = opt
    return q, keep


def hallar_solve_footprint(req) -> int:
    return int(_lib.hallar_solve_footprint(C.byref(req)))


def _scheck(status, s, allow=()):
    if status != HALLAR_OK and status not in allow:
        raise HallarError(status, _lib.hallar_server_last_error(s).decode())
    return status


def hallar_server_create(hbm_budget_bytes, max_inflight, device=0):
    o = hallar_server_options(float(hbm_budget_bytes), int(max_inflight), int(device))
    s = C.c_void_p()
    st = _lib.hallar_server_create(C.byref(o), C.byref(s))
    if st != HALLAR_OK:
        raise HallarError(st, "hallar_server_create failed")
    return s


def hallar_server_submit(s, req) -> int:
    t = C.c_int64()
    _scheck(_lib.hallar_server_submit(s, C.byref(req), C.byref(t)), s)
    return t.value


def hallar_server_wait(s, ticket, timeout_s=-1.0, U=None, U_capacity=0, p=None):
    """Returns (status, hallar_result, rank, latency_s); U / p filled when given."""
    res = hallar_result()
    rank = C.c_int32()
    lat = C.c_double()
    st = _lib.hallar_server_wait(s, int(ticket), float(timeout_s), C.byref(res), _ptr(U),
                                 int(U_capacity), _ptr(p), C.byref(rank), C.byref(lat))
    if lat.value < 0.0 and st != HALLAR_ETIMEOUT:
        _scheck(st, s)  # the call itself failed (unknown ticket, capacity)
    return st, res, rank.value, lat.value


def hallar_server_get_stats(s) -> dict:
    st = hallar_server_stats()
    _scheck(_lib.hallar_server_get_stats(s, C.byref(st)), s)
    return st.as_dict()


def hallar_server_destroy(s):
    _lib.hallar_server_destroy(s)


def hallar_server_last_error(s) -> str:
    return _lib.hallar_server_last_error(s).decode()


class Server:
    """hallar_server_* wrapper: submit instances, wait for solutions."""

    def __init__(self, hbm_budget_bytes, max_inflight, device=0):
        self.s = hallar_server_create(hbm_budget_bytes, max_inflight, device)
        self.meta = {}

    def submit(self, inst, U0, precision=HALLAR_FP64, **options) -> int:
        q, keep = request_from_instance(inst, U0, precision, **options)
        t = hallar_server_submit(self.s, q)
        del keep
        self.meta[t] = (inst.n, inst.m, precision, int(options.get("r_cap", 32)))
        return t

    def wait(self, ticket, timeout_s=-1.0):
        """(status, result, U [n x rank], p [m], latency_s) of a ticket."""
        n, m, precision, r_cap = self.meta[ticket]
        dt = np.float32 if precision == HALLAR_MIXED else np.float64
        cap = r_cap + 1
        U = np.empty((n, cap), dtype=dt)
        p = np.empty(m)
        st, res, rank, lat = hallar_server_wait(self.s, ticket, timeout_s, U, cap, p)
        if st == HALLAR_ETIMEOUT and lat < 0.0:  # still queued or running
            return st, None, None, None, None
        del self.meta[ticket]
        return st, res, np.ascontiguousarray(U[:, :rank]), p, lat

    def stats(self) -> dict:
        return hallar_server_get_stats(self.s)

    def close(self):
        if self.s is not None:
            hallar_server_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---------------------------------------------------------------------------
# batched operators over a segmented CSR
# ---------------------------------------------------------------------------
def _bcheck(status, b):
    if status != HALLAR_OK:
        raise HallarError(status, _lib.hallar_batch_last_error(b).decode())
    return status


class Batch:
    """hallar_batch_*: many instances stacked into one segmented problem."""

    def __init__(self, instances, precision=HALLAR_FP64, autotune=False, stream=None):
        reqs, keep = [], []
        for inst in instances:
            q, k = request_from_instance(inst, np.zeros((inst.n, 1)), precision)
            reqs.append(q)
            keep.append(k)
        arr = (hallar_request * len(reqs))(*reqs)
        self.b = C.c_void_p()
        _bcheck(_lib.hallar_batch_create(len(reqs), arr, int(precision), int(bool(autotune)),
                                         stream, C.byref(self.b)), None)
        del keep
        self.count = len(reqs)
        self.precision = precision
        self.row_off = np.empty(self.count + 1, np.int64)
        self.cons_off = np.empty(self.count + 1, np.int64)
        nt, mt = C.c_int64(), C.c_int64()
        _bcheck(_lib.hallar_batch_layout(self.b, _ptr(self.row_off), _ptr(self.cons_off),
                                         C.byref(nt), C.byref(mt)), self.b)
        self.n_total, self.m_total = nt.value, mt.value

    def grad(self, U, r, p, beta, W, g, resid=None):
        return _bcheck(_lib.hallar_batch_grad(self.b, _ptr(U), int(r), _ptr(p), _ptr(beta),
                                              _ptr(W), _ptr(g), _ptr(resid)), self.b)

    def shape(self, r):
        G, K, t = C.c_int32(), C.c_int32(), C.c_int32()
        _bcheck(_lib.hallar_batch_shape(self.b, int(r), C.byref(G), C.byref(K), C.byref(t)),
                self.b)
        return G.value, K.value, bool(t.value)

    def close(self):
        if self.b is not None:
            _lib.hallar_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
