"""Host-side pieces of the quench server: footprints, admission decisions, request mix."""
import numpy as np

from paper_2212_09782_b300 import serve


def test_state_bytes_scale_with_caps():
    small = serve.Request(0, 32, 3, 128, 1.0, 5)
    big = serve.Request(1, 128, 5, 1024, 1.0, 5)
    a = serve.state_bytes(small, "c64_3xtf32")
    b = serve.state_bytes(big, "c64_3xtf32")
    assert b > 100 * a
    # complex128 doubles the tensor bytes
    assert serve.state_bytes(big, "c128") > 1.9 * b
    caps = serve.chain_caps(8, 3, 10)
    assert caps == [1, 3, 9, 10, 10, 10, 9, 3, 1]


def test_admission_waits_then_rejects_what_never_fits():
    free = {"v": 0}
    srv = serve.QuenchServer(mem_free=lambda: free["v"], mem_total=lambda: 40 << 30,
                             reserve_bytes=0)
    req = serve.Request(0, 64, 4, 512, 1.0, 5)
    need = srv.footprint(req)
    free["v"] = need - 1
    ok, ever = srv._fits(req)
    assert not ok and ever
    free["v"] = need
    ok, ever = srv._fits(req)
    assert ok and ever
    huge = serve.Request(1, 128, 5, 1 << 16, 1.0, 5)
    ok, ever = srv._fits(huge)
    assert not ever


def test_poisson_mix_is_seeded():
    a = serve.poisson_mix(16, 4.0, seed=5)
    b = serve.poisson_mix(16, 4.0, seed=5)
    assert [(r.L, r.d, r.chi_max, r.g, r.arrival) for r in a] == \
           [(r.L, r.d, r.chi_max, r.g, r.arrival) for r in b]
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert np.all(gaps > 0)
    assert {r.L for r in a} <= {32, 64, 128} and {r.d for r in a} <= {3, 4, 5}


def test_admission_reserves_one_workspace_per_executor_worker():
    from paper_2212_09782_b300 import lib as L
    nw = L.layer_workers()
    assert nw >= 1
    srv = serve.QuenchServer(mem_free=lambda: 1 << 40, mem_total=lambda: 1 << 40, reserve_bytes=0)
    assert srv.workers == nw
    req = serve.Request(0, 32, 3, 128, 1.0, 2)
    assert srv.footprint(req) == serve.state_bytes(req, srv.precision) + nw * serve.workspace_bytes(req, srv.precision)


def test_big_bonds_hold_only_the_big_workers_workspaces():
    # a chi = 1024, d = 5 request: its bonds need more than the big-bond threshold, so the
    # executor holds LAYER_BIG_WORKERS of its workspaces and threshold-sized ones elsewhere
    srv = serve.QuenchServer(mem_free=lambda: 1 << 40, mem_total=lambda: 1 << 40, reserve_bytes=0)
    big = serve.Request(0, 128, 5, 1024, 1.0, 2)
    ws = serve.workspace_bytes(big, srv.precision)
    assert ws > serve.LAYER_BIG_BOND_BYTES
    expect = (serve.LAYER_BIG_WORKERS * ws +
              (srv.workers - serve.LAYER_BIG_WORKERS) * serve.LAYER_BIG_BOND_BYTES)
    assert srv.footprint(big) == serve.state_bytes(big, srv.precision) + expect
    assert expect < srv.workers * ws


def test_header_constants_mirrored():
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                            "qrtebd.h")).read()
    assert re.search(r"#define QRTEBD_LAYER_BIG_BOND_BYTES \(1024ull << 20\)", hdr)
    assert serve.LAYER_BIG_BOND_BYTES == 1024 << 20
    assert re.search(r"#define QRTEBD_LAYER_BIG_WORKERS (\d+)", hdr).group(1) == str(serve.LAYER_BIG_WORKERS)
