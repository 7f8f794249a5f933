"""C3 at reduced steps against the oracle: the uniform two-site cell with CBE (d = 5, g = 2,
dt = 0.02, chi_max = 1024) for its first 80 steps, in which chi grows from 1 to ~650, run
through the library and compared every 5 steps with the oracle's trace of the same run
(tests/golden/c3_oracle_trace.json, written by tests/golden/make_c3_trace.py from the
oracle alone).

complex128: <Z> to 1e-9 and the bond dimensions to within 1 % (a Schmidt value at the
svd_min = 1e-14 threshold may fall either side of it in the last bits). complex64 3xTF32:
<Z> to 2e-5; its Schmidt values below ~1e-7 of the largest are rounding noise, so its bond
dimensions are not compared."""
import json
import os

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("prec", ["c128", "c64_3xtf32"])
def test_c3_first_80_steps_match_oracle(prec):
    from paper_2212_09782_b300 import lib as L
    with open(os.path.join(HERE, "golden", "c3_oracle_trace.json")) as f:
        ref = {r["step"]: r for r in json.load(f)["trace"]}
    Lc, d, g, dt = 2, 5, 2.0, 0.02
    tr = L.trunc_default(L.CBE, 1024)
    half = L.clock_layer_gates(Lc, d, g, dt / 2, infinite=True)
    full = L.clock_layer_gates(Lc, d, g, dt, infinite=True)
    s = L.MPS(Lc, d, 1024, precision=prec, infinite=True)
    Z = np.diag(np.exp(2j * np.pi * np.arange(d) / d))
    worst = 0.0
    try:
        for k in range(1, 81):
            L.tebd_step(s, half, full, tr)
            if k in ref:
                z = s.expectation(0, Z)
                zr = complex(*ref[k]["z"])
                worst = max(worst, abs(z - zr))
                assert abs(z - zr) <= (1e-9 if prec == "c128" else 2e-5), (k, z, zr)
                if prec == "c128":
                    for a, b in zip(s.bond_dims(), ref[k]["chi"]):
                        assert abs(a - b) <= max(1, 0.01 * b), (k, s.bond_dims(), ref[k]["chi"])
        L.stream_check()
    finally:
        s.close()
    print(prec, "max |<Z> - <Z>_oracle| over 16 checkpoints:", worst)
