"""Serving engine (hallar_server_*): continuous batching of whole solves.

Each request is solved alone (one solve in flight) and again inside a mix
of requests that overlap on the device; the results must be identical, bit
for bit, since every kernel is deterministic and handles share no device
state.  Served results are also pinned to closed forms, admission is checked
against the HBM budget, and malformed requests are rejected."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2505_13719_b300 import instances as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_13719_b300 import hallar
    return hallar


def requests():
    """(name, instance, r0, U0 seed, precision, options, closed form or None)."""
    return [
        ("maxcut C101 fp64", I.maxcut(101, *I.cycle_graph(101)), 2, 11, 0, {},
         50.5 * (1 + math.cos(math.pi / 101))),
        ("maxcut ER300 mixed", I.maxcut(300, *I.er_graph(300, 0.03, 12)), 4, 12, 1, {}, None),
        ("theta C9 fp64", I.theta(9, *I.cycle_graph(9)), 2, 13, 0, {},
         9 * math.cos(math.pi / 9) / (1 + math.cos(math.pi / 9))),
        ("maxcut torus 16 unit mixed", I.maxcut_torus(16, "unit"), 3, 14, 1, {}, 512.0),
        ("completion 60x80 fp64",
         I.completion(60, 80, 2, I.completion_sample_count(60, 80, 2), seed=5), 2, 15, 0, {},
         None),
        ("theta H(6,2) mixed", I.theta(64, *I.hypercube_graph(6)), 2, 16, 1, {}, 32.0),
    ]


TOL = {0: 1e-6, 1: 5e-6}


def submit_all(H, srv, reqs):
    tickets = []
    for name, inst, r0, seed, prec, opts, _ in reqs:
        U0 = I.initial_factor(inst.n, r0, seed)
        tickets.append(srv.submit(inst, U0, prec, tol=TOL[prec], time_limit_s=120.0, **opts))
    return tickets


def test_results_same_alone_and_in_the_mix(H):
    reqs = requests()
    budget = 8e9
    alone = []
    with H.Server(budget, 1) as srv:
        for req in reqs:
            (t,) = submit_all(H, srv, [req])
            alone.append(srv.wait(t))
        st1 = srv.stats()
    assert st1["max_inflight_seen"] == 1
    with H.Server(budget, 4) as srv:
        tickets = submit_all(H, srv, reqs)
        mixed = [srv.wait(t) for t in tickets]
        st4 = srv.stats()
    assert st4["completed"] == len(reqs)
    assert st4["max_inflight_seen"] >= 2  # the solves did overlap
    for (name, inst, *_), a, b in zip(reqs, alone, mixed):
        st_a, res_a, U_a, p_a, _ = a
        st_b, res_b, U_b, p_b, _ = b
        assert st_a == H.HALLAR_OK, (name, res_a.as_dict())
        assert st_b == st_a, name
        assert res_b.pval == res_a.pval, name
        assert res_b.kkt == res_a.kkt, name
        assert U_b.shape == U_a.shape and np.array_equal(U_b, U_a), name
        assert np.array_equal(p_b, p_a), name


def test_served_results_meet_closed_forms(H):
    reqs = [r for r in requests() if r[6] is not None]
    with H.Server(8e9, 4) as srv:
        tickets = submit_all(H, srv, reqs)
        for (name, inst, r0, seed, prec, opts, ref), t in zip(reqs, tickets):
            st, res, U, p, lat = srv.wait(t)
            assert st == H.HALLAR_OK, name
            assert res.kkt <= TOL[prec], name
            assert abs(inst.sense * res.pval - ref) <= 1e-5 * abs(ref), (name, res.pval, ref)
            assert lat > 0.0
        stats = srv.stats()
    assert stats["p99_latency_s"] >= stats["p50_latency_s"] > 0.0


def test_admission_respects_the_budget(H):
    reqs = requests()[:4]
    fps = []
    for name, inst, r0, seed, prec, opts, _ in reqs:
        q, keep = H.request_from_instance(inst, I.initial_factor(inst.n, r0, seed), prec)
        fps.append(H.hallar_solve_footprint(q))
    # room for the largest request but not for any two of them
    budget = max(fps) + 0.5 * min(fps)
    with H.Server(budget, 4) as srv:
        tickets = submit_all(H, srv, reqs)
        for t in tickets:
            assert srv.wait(t)[0] == H.HALLAR_OK
        st = srv.stats()
    assert st["max_inflight_seen"] == 1
    assert st["peak_bytes_inflight"] <= budget


def test_rejections_and_failed_requests(H):
    inst = I.maxcut(50, *I.cycle_graph(50))
    U0 = I.initial_factor(inst.n, 2, 1)
    with H.Server(1e6, 2) as srv:  # 1 MB: below any footprint
        with pytest.raises(H.HallarError) as e:
            srv.submit(inst, U0)
        assert e.value.status == H.HALLAR_ENOMEM
    with H.Server(4e9, 2) as srv:
        q, keep = H.request_from_instance(inst, U0)
        q.b = None
        with pytest.raises(H.HallarError) as e:
            H.hallar_server_submit(srv.s, q)
        assert e.value.status == H.HALLAR_EINVAL
        with pytest.raises(H.HallarError):
            H.hallar_server_wait(srv.s, 12345)
        # a problem only hallar_create rejects (tau^2 <= 0) completes with EINVAL
        bad = I.maxcut(50, *I.cycle_graph(50))
        bad.tau2 = -1.0
        t = srv.submit(bad, U0)
        st, res, U, p, lat = srv.wait(t)
        assert st == H.HALLAR_EINVAL
        assert srv.stats()["failed"] == 1


def test_wait_with_timeout_keeps_the_ticket(H):
    inst = I.maxcut_torus(64, "unit")
    with H.Server(8e9, 1) as srv:
        t = srv.submit(inst, I.initial_factor(inst.n, 4, 3), 0, tol=1e-6, time_limit_s=60.0)
        st, res, *_ = srv.wait(t, timeout_s=1e-3)
        if st == H.HALLAR_ETIMEOUT and res is None:
            st, res, *_ = srv.wait(t)
        assert st == H.HALLAR_OK
