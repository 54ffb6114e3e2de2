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

EXPORTED = ("hallar_default_options", "hallar_create", "hallar_eval_A", "hallar_grad",
            "hallar_min_eig", "hallar_solve", "hallar_get_solution", "hallar_get_sizes",
            "hallar_destroy", "hallar_last_error", "hallar_status_string", "hallar_profile",
            "hallar_grad_diag_noalloc")


class hallar_options(C.Structure):
    _fields_ = [("tol", C.c_double), ("sigma", C.c_double), ("chi", C.c_double),
                ("lambda0", C.c_double), ("beta0", C.c_double), ("beta_max", C.c_double),
                ("eps_decay", C.c_double), ("eps1_rel", C.c_double),
                ("lanczos_tol_rel", C.c_double), ("time_limit_s", C.c_double),
                ("r_cap", C.c_int32), ("max_outer", C.c_int32), ("max_hlr", C.c_int32),
                ("max_aipp", C.c_int32), ("max_fista", C.c_int32),
                ("lanczos_kmax", C.c_int32), ("precision", C.c_int32),
                ("verbose", C.c_int32), ("seed", C.c_uint64), ("stream", C.c_void_p)]


class hallar_result(C.Structure):
    _fields_ = [("pval", C.c_double), ("dval", C.c_double), ("theta", C.c_double),
                ("lam_min_S", C.c_double), ("rel_primal", C.c_double),
                ("rel_gap", C.c_double), ("rel_dual", C.c_double), ("kkt", C.c_double),
                ("beta", C.c_double), ("seconds", C.c_double), ("rank", C.c_int32),
                ("converged", C.c_int32), ("outer_iters", C.c_int32),
                ("hlr_iters", C.c_int32), ("aipp_iters", C.c_int32),
                ("fista_iters", C.c_int32), ("fista_failures", C.c_int32),
                ("lanczos_iters", C.c_int32), ("fw_steps", C.c_int32), ("trims", C.c_int32),
                ("grad_evals", C.c_int64), ("value_evals", C.c_int64),
                ("kernel_launches", C.c_int64)]

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
        "hallar_min_eig": ([P, P, D, I32, P, P, P, P, P], C.c_int),
        "hallar_solve": ([P, P, I32, P, P], C.c_int),
        "hallar_get_solution": ([P, P, I32, P, P], C.c_int),
        "hallar_get_sizes": ([P, P, P, P, P], C.c_int),
        "hallar_profile": ([P, I32, P, P, P], C.c_int),
        "hallar_grad_diag_noalloc": ([I64, I32, P, P, P, P, P, P, D, P, P, P, P, P, C.c_char_p,
                                      I32], C.c_int),
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
    fam = FAMILY[family] if isinstance(family, str) else int(family)
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


def hallar_eval_A(h, U, r, T):
    return _check(_lib.hallar_eval_A(h, _ptr(U), int(r), _ptr(T)), h)


def hallar_grad(h, U, r, p, beta, W, resid=None):
    """Returns g(U); W (and resid) are written in place."""
    g = C.c_double()
    _check(_lib.hallar_grad(h, _ptr(U), int(r), _ptr(p), float(beta), _ptr(W), C.byref(g),
                            _ptr(resid)), h)
    return g.value


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


def hallar_profile(h, op):
    """op 1: clear and start kernel timing, 2: stop, 0: read.  Returns
    (ms[3], launches[3], bytes[3]) for the fused operator, value-change and
    Lanczos kernel classes."""
    ms = (C.c_double * 3)()
    nl = (C.c_int64 * 3)()
    by = (C.c_double * 3)()
    _check(_lib.hallar_profile(h, int(op), ms, nl, by), h)
    return list(ms), list(nl), list(by)


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
