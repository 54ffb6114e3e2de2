"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/hallar.h declares (host-only calls; no device work)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hallar.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hallar_[a-z_A-Z0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_13719_b300.build import build_library
    path = build_library()
    from paper_2505_13719_b300 import hallar as H
    return path, H


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hallar_create", "hallar_eval_A", "hallar_grad", "hallar_min_eig",
                     "hallar_solve", "hallar_destroy", "hallar_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    path, H = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (hallar_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        assert hasattr(H._lib, f)


def test_build_targets_sm_103a(lib):
    from paper_2505_13719_b300 import build as B
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.getmtime(lib[0]) >= max(os.path.getmtime(f) for f in B.sources())


def test_host_only_entry_points(lib):
    _, H = lib
    o = H.hallar_default_options()
    assert o.tol == 1e-5 and o.r_cap == 32 and o.precision == H.HALLAR_FP64
    assert H._lib.hallar_status_string(H.HALLAR_EINVAL) == b"HALLAR_EINVAL"
    assert H._lib.hallar_default_options(None) == H.HALLAR_EINVAL
    assert H._lib.hallar_eval_A(None, None, 1, None) == H.HALLAR_EINVAL
    assert H._lib.hallar_get_sizes(None, None, None, None, None) == H.HALLAR_EINVAL
    H._lib.hallar_destroy(None)  # no-op


def test_binding_names_match_c_names(lib):
    _, H = lib
    for f in declared_functions():
        assert f in H.EXPORTED
