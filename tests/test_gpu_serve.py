"""Continuous batching: each request's result is the same served alone and in a mix."""
import pytest

from paper_2212_09782_b300 import serve

pytestmark = pytest.mark.gpu


def _mix():
    return [serve.Request(0, 12, 3, 16, 1.5, 6, arrival=0.0),
            serve.Request(1, 10, 4, 12, 0.8, 4, arrival=0.0),
            serve.Request(2, 16, 2, 8, 1.2, 5, arrival=0.05),
            serve.Request(3, 8, 5, 20, 2.0, 3, arrival=0.1)]


def _copy(r):
    return serve.Request(r.rid, r.L, r.d, r.chi_max, r.g, r.steps, r.dt, 0.0)


def test_results_same_alone_and_in_mix():
    srv = serve.QuenchServer(precision="c64_3xtf32", reserve_bytes=0)
    for r in _mix():
        srv.submit(r)
    m = srv.run()
    assert m["requests_done"] == 4 and m["requests_rejected"] == 0
    mixed = {r.rid: r for r in srv.done}
    for r in _mix():
        solo = serve.QuenchServer(precision="c64_3xtf32", reserve_bytes=0)
        solo.submit(_copy(r))
        solo.run()
        a = solo.done[0]
        b = mixed[r.rid]
        assert len(a.z_mid) == len(b.z_mid) == r.steps
        # deterministic kernels and reduction orders: identical, not merely close
        assert a.z_mid == b.z_mid
        assert a.bond_dims == b.bond_dims and a.eps == b.eps
    assert m["p99_step_latency_ms"] >= m["p50_step_latency_ms"] > 0


def test_memory_budget_queues_requests():
    # a budget that fits one request at a time: everyone finishes, one after another
    reqs = _mix()[:3]
    one = max(serve.QuenchServer(reserve_bytes=0).footprint(r) for r in reqs)
    state = {"used": 0}
    srv = serve.QuenchServer(precision="c64_3xtf32", reserve_bytes=0,
                             mem_free=lambda: one + 1024 - 0 * state["used"],
                             mem_total=lambda: 10 * one, max_active=1)
    for r in reqs:
        srv.submit(r)
    m = srv.run()
    assert m["requests_done"] == 3
    starts = sorted(r.admitted_at for r in srv.done)
    ends = sorted(r.finished_at for r in srv.done)
    assert starts[1] >= ends[0] - 1e-6 and starts[2] >= ends[1] - 1e-6
