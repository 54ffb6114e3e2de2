"""Host-side parts of the serving engine that need no GPU: the footprint
estimate that admission charges, and option validation."""
import pytest

from paper_2505_13719_b300 import instances as I


@pytest.fixture(scope="module")
def H():
    from paper_2505_13719_b300.build import build_library
    build_library()
    from paper_2505_13719_b300 import hallar
    return hallar


def footprint(H, inst, prec=0, **opts):
    q, keep = H.request_from_instance(inst, I.initial_factor(inst.n, 2, 1), prec, **opts)
    return H.hallar_solve_footprint(q)


def test_footprint_covers_the_dominant_buffers(H):
    inst = I.maxcut_torus(100, "unit")  # n = 1e4
    n = inst.n
    fp = footprint(H, inst, 0, r_cap=32, lanczos_kmax=300)
    # at least the Lanczos basis (n x 300 doubles) and ten factor buffers
    # (n x 34 doubles each: r_cap + 1 padded to an even width)
    assert fp >= n * 300 * 8 + 10 * n * 34 * 8
    # and not absurdly more (allocator slack is 5 % + 64 MB)
    assert fp <= 2 * (n * 300 * 8 + 10 * n * 34 * 8) + (80 << 20)


def test_footprint_grows_with_size_rank_and_precision(H):
    small, big = I.maxcut_torus(50, "unit"), I.maxcut_torus(100, "unit")
    assert footprint(H, big) > footprint(H, small)
    assert footprint(H, big, r_cap=64) > footprint(H, big, r_cap=8)
    # float factors are half the size, unless the solve may go on in FP64
    assert footprint(H, big, 0) > footprint(H, big, 1, promote=0)
    n, ld = big.n, 36  # r_cap 32 + 1 padded to 4 floats
    assert footprint(H, big, 1, promote=1) - footprint(H, big, 1, promote=0) \
        >= 10 * n * ld * 4


def test_server_options_are_validated(H):
    with pytest.raises(H.HallarError) as e:
        H.hallar_server_create(0.0, 2)
    assert e.value.status == H.HALLAR_EINVAL
    with pytest.raises(H.HallarError) as e:
        H.hallar_server_create(1e9, 0)
    assert e.value.status == H.HALLAR_EINVAL


def test_options_layout_matches_the_header(H):
    # hallar_default_options fills the struct in C; reading every field back
    # through the ctypes mirror pins the two layouts to each other (a shifted
    # field would misread all that follow it)
    o = H.hallar_default_options()
    want = dict(tol=1e-5, sigma=0.3, chi=0.5, lambda0=1.0, beta0=1.0, beta_max=1e8,
                eps_decay=0.5, eps1_rel=1e-2, lanczos_tol_rel=0.5, time_limit_s=3600.0,
                lambda_kappa=0.0, r_cap=32, max_outer=300, max_hlr=100, max_aipp=20000,
                max_fista=400, lanczos_kmax=300, precision=0, verbose=0, promote=1, seed=0)
    for k, v in want.items():
        assert getattr(o, k) == v, k
    assert o.stream is None
