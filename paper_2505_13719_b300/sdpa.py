"""Reader for SDP data in sparse SDPA format (Section 3.2, "SDPA format";
Section 4.3, eq. constraint matrix density).  Host-side data loading only:
it builds an ``instances.Instance`` of family ``hslr`` (Section 3.2, eq.
HSLR-rep-body) with every matrix in its sparse part and no low-rank terms.

SDPA describes the pair
    min  sum_i c_i x_i   s.t.  sum_i F_i x_i - F_0 psd
    max  F_0 . Y         s.t.  F_i . Y = c_i (i = 1..m),  Y psd,
and the second of these is (P) as this library states it, a minimisation:
C = -F_0, A_i = F_i, b = c, with ``sense = -1`` so that the user value
``sense * pval`` is the SDPA maximum.  The trace bound tau^2 of the
spectraplex is not part of the format; the caller supplies it.

Layout of a file: comment lines (starting with '"' or '*'), then m, the
number of blocks, the block sizes, the m values c_i, and one line per
nonzero entry "matno blkno i j value" (1-based, i <= j: each symmetric
matrix is listed by its upper triangle).  Separators ',', '{', '}', '(' and
')' count as blanks.  One positive semidefinite block is supported.

Each matrix gets its density d_l = nnz(A_l) / n^2 over the full symmetric
pattern (eq. constraint matrix density); matrices with d_l > 0.1 are
marked dense (``meta["dense"]``), the split the paper's SDPA kernels use.
"""
from __future__ import annotations

import numpy as np

from . import instances as I

DENSE_THRESHOLD = 0.1


def _tokens(text):
    for line in text.splitlines():
        s = line.strip()
        if not s or s[0] in "\"*":
            continue
        for ch in ",{}()":
            s = s.replace(ch, " ")
        yield s.split()


def parse(text: str, tau2: float, name: str = "sdpa") -> I.Instance:
    """The SDP of an SDPA-sparse text as an ``hslr`` Instance (see the module
    docstring).  Raises ValueError for malformed input, more than one block,
    a diagonal (LP) block, an index out of range or an entry below the
    diagonal."""
    if not (tau2 > 0.0):
        raise ValueError("tau2 must be positive")
    lines = list(_tokens(text))

    def num(tok):
        return float(tok.replace("D", "E").replace("d", "e"))

    def leading_numbers(ln):
        # the numbers at the start of a header line; what follows the first
        # non-number ("7 = mDIM") is a comment
        out = []
        for t in ln:
            try:
                out.append(num(t))
            except ValueError:
                break
        return out

    k = 0
    try:
        m = int(leading_numbers(lines[0])[0])
        nblocks = int(leading_numbers(lines[1])[0])
        k = 2
    except (IndexError, ValueError):
        raise ValueError("SDPA header: m and the number of blocks") from None
    if m < 0:
        raise ValueError("SDPA header: m < 0")
    if nblocks != 1:
        raise ValueError("SDPA: exactly one block is supported")
    sizes = leading_numbers(lines[k]) if k < len(lines) else []
    if not sizes:
        raise ValueError("SDPA header: block sizes")
    n = int(sizes[0])
    k += 1
    if n <= 0:
        raise ValueError("SDPA: the block must be a positive (psd) block")
    cvals = []
    while len(cvals) < m:
        if k >= len(lines):
            raise ValueError("SDPA header: fewer than m values of c")
        got = leading_numbers(lines[k])
        if not got:
            raise ValueError("SDPA header: the values of c")
        cvals.extend(got)
        k += 1
    if len(cvals) != m:
        raise ValueError("SDPA header: more than m values of c on a line")
    c = np.array(cvals)
    used = k
    ells, ii, jj, vv = [], [], [], []
    for ln in lines[used:]:
        if len(ln) != 5:
            raise ValueError(f"SDPA entry line: {' '.join(ln)!r}")
        l, blk, i, j = (int(x) for x in ln[:4])
        v = num(ln[4])
        if blk != 1 or not (0 <= l <= m) or not (1 <= i <= n) or not (1 <= j <= n):
            raise ValueError(f"SDPA entry out of range: {' '.join(ln)!r}")
        if i > j:
            raise ValueError(f"SDPA entry below the diagonal: {' '.join(ln)!r}")
        if v == 0.0:
            continue
        ells.append(l)
        ii.append(i - 1)
        jj.append(j - 1)
        vv.append(v)
    ell = np.array(ells, dtype=np.int64)
    a = np.array(ii, dtype=np.int64)
    b = np.array(jj, dtype=np.int64)
    v = np.array(vv, dtype=np.float64)
    v = np.where(ell == 0, -v, v)  # C = -F_0
    # density over the full symmetric pattern of each matrix (duplicates once)
    key = (ell * n + a) * n + b
    uniq, first = np.unique(key, return_index=True)
    ul, ua, ub = ell[first], a[first], b[first]
    nnz = np.bincount(ul, weights=np.where(ua == ub, 1.0, 2.0), minlength=m + 1)
    density = nnz / float(n) ** 2
    meta = {"density": density, "dense": density > DENSE_THRESHOLD,
            "format": "sdpa", "entries": int(ell.shape[0])}
    return I.hslr(n, (ell, a, b, v), [], c, tau2, sense=-1.0, name=name, meta=meta)


def read(path: str, tau2: float) -> I.Instance:
    """``parse`` of a file."""
    with open(path) as f:
        return parse(f.read(), tau2, name=path.rsplit("/", 1)[-1])


def write(inst: I.Instance) -> str:
    """The SDPA-sparse text of an ``hslr`` Instance without low-rank terms
    (the inverse of ``parse``; F_0 = -C)."""
    if inst.family != "hslr" or inst.lr_terms:
        raise ValueError("only hslr instances without low-rank terms")
    n, m = inst.n, inst.m
    out = [f"{m}", "1", f"{n}", " ".join(repr(float(x)) for x in inst.b)]
    rowptr = inst.C_rowptr
    for i in range(n):
        for e in range(int(rowptr[i]), int(rowptr[i + 1])):
            j = int(inst.C_col[e])
            if i <= j:
                out.append(f"0 1 {i + 1} {j + 1} {repr(-float(inst.C_val[e]))}")
    ell, a, b, v = inst.sp_cons
    for k in range(ell.shape[0]):
        if a[k] <= b[k]:
            out.append(f"{int(ell[k]) + 1} 1 {int(a[k]) + 1} {int(b[k]) + 1} {repr(float(v[k]))}")
    return "\n".join(out) + "\n"
