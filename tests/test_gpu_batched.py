"""Batched layers (all bonds of a parity of several states at once, on worker streams,
graph-captured in steady state) against the same layers applied state by state."""
import numpy as np
import pytest

from oracle import clock

pytestmark = pytest.mark.gpu


def _states(Lb, prec):
    specs = [(8, 3, 9, 1.5), (10, 2, 8, 1.0), (6, 4, 16, 0.7)]
    out = []
    for L, d, chi, g in specs:
        out.append((Lb.MPS(L, d, chi, precision=prec), Lb.MPS(L, d, chi, precision=prec),
                    Lb.clock_layer_gates(L, d, g, 0.025), Lb.clock_layer_gates(L, d, g, 0.05), d))
    return out


@pytest.mark.parametrize("prec", ["c128", "c64_3xtf32"])
@pytest.mark.parametrize("scheme", ["plain", "cbe"])
def test_batched_equals_sequential(prec, scheme):
    from paper_2212_09782_b300 import lib as Lb
    tr = Lb.trunc_default(Lb.CBE if scheme == "cbe" else Lb.PLAIN, 16, dchi_min=8)
    sts = _states(Lb, prec)
    batched = [a for a, _, _, _, _ in sts]
    for step in range(6):  # long enough to saturate, capture a graph and replay it
        Lb.tebd_step_batched(batched, [h for _, _, h, _, _ in sts], [f for _, _, _, f, _ in sts], tr)
        for _, single, h, f, _ in sts:
            Lb.tebd_step(single, h, f, tr)
    for a, b, _, _, d in sts:
        a.sync(); b.sync()
        Z, _ = clock.clock_operators(d)
        za = [a.expectation(m, Z) for m in range(a.L)]
        zb = [b.expectation(m, Z) for m in range(b.L)]
        assert za == zb  # same kernels, same reduction order: bit for bit
        assert a.bond_dims() == b.bond_dims()
        assert a.truncation_error(-1) == b.truncation_error(-1)


def test_set_site_and_bond_roundtrip():
    from paper_2212_09782_b300 import lib as Lb
    from paper_2212_09782_b300 import workloads as W
    L, d, chi = 6, 3, 9
    dims, B, Xi = W.random_right_canonical_mps(L, d, chi, seed=3)
    s = Lb.MPS(L, d, chi, precision="c128")
    for m in range(L):
        s.set_site(m, B[m])
    for b in range(L + 1):
        s.set_bond(b, Xi[b], diagonal=True)
    assert s.bond_dims() == dims
    # <1> from every site equals ||Xi[m] B[m]||^2 = ||Xi[m]||^2 = 1 (right isometry)
    for m in range(L):
        assert abs(s.expectation(m, np.eye(d)) - 1) < 1e-12
    assert np.allclose(s.schmidt(3), np.sort(np.abs(Xi[3]))[::-1], atol=1e-12)


def test_batched_layer_sweeps_is_part_of_the_replayed_shape():
    # a plain layer is captured as a graph on its second sighting; the same shapes with a
    # different number of ALS sweeps must not replay it
    import numpy as np
    from paper_2212_09782_b300 import lib as L
    Lc, d, chi = 8, 3, 9
    runs = {}
    for sweeps in (1, 1, 1, 3):
        s = L.MPS(Lc, d, chi, precision="c128")
        U = np.linalg.qr(np.random.default_rng(5).normal(size=(9, 9)) + 1j * np.random.default_rng(6).normal(size=(9, 9)))[0]
        gates = np.stack([U] * (Lc - 1))
        tr = L.trunc_default(L.PLAIN, chi, sweeps=sweeps)
        for _ in range(3):
            L.apply_layer_batched([s], 0, [gates], tr)
            L.apply_layer_batched([s], 1, [gates], tr)
        s.sync()
        runs.setdefault(sweeps, []).append(s.truncation_error(-1))
        s.close()
    # identical runs agree (graph replay included); three sweeps truncate less
    assert np.allclose(runs[1], runs[1][0], rtol=1e-12, atol=0)
    assert runs[3][0] < runs[1][0]


@pytest.mark.parametrize("prec,tol", [("c128", 1e-10), ("c64_3xtf32", 1e-5)])
@pytest.mark.parametrize("scheme", ["plain", "cbe"])
def test_batched_against_oracle(prec, tol, scheme):
    # several states of different L, d and chi_max evolved by batched layers (CBE cuts kept
    # on the device and read back once per layer; repeated shapes replayed as graphs) against
    # the oracle's TEBD of each
    from oracle import mps as omps
    from paper_2212_09782_b300 import lib as Lb
    specs = [(8, 3, 9, 1.5), (6, 4, 16, 0.7), (10, 2, 8, 1.0)]
    dt, steps = 0.05, 8
    kw = dict(dchi_min=8) if scheme == "cbe" else {}
    states, orcs, halves, fulls = [], [], [], []
    for L, d, chi, g in specs:
        states.append(Lb.MPS(L, d, chi, precision=prec))
        orcs.append((omps.product_state(L, d, 0, True), omps.strang_gates(L, d, g, dt, True), chi))
        halves.append(Lb.clock_layer_gates(L, d, g, dt / 2))
        fulls.append(Lb.clock_layer_gates(L, d, g, dt))
    tr = Lb.trunc_default(Lb.CBE if scheme == "cbe" else Lb.PLAIN, 1 << 20, **kw)
    for _ in range(steps):
        Lb.tebd_step_batched(states, halves, fulls, tr)
        for o, (half, full), chi in orcs:
            omps.tebd_step(o, half, full, scheme=scheme, chi_max=chi, **kw)
    for s, (o, _g, _chi), (L, d, _c, _gg) in zip(states, orcs, specs):
        s.sync()
        Z, _ = clock.clock_operators(d)
        zg = np.array([s.expectation(m, Z) for m in range(L)])
        zo = np.array([omps.expectation_1site(o, m, Z) for m in range(L)])
        assert np.abs(zg - zo).max() < tol, (L, d, np.abs(zg - zo).max())
        if scheme == "plain":
            assert s.bond_dims() == o.bond_dims()
        s.close()
