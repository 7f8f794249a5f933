"""Writes c3_oracle_trace.json: the oracle's run of the C3 workload (uniform two-site cell,
d = 5, g = 2.0, |00>, Strang dt = 0.02, CBE with dchi = max(100, ceil(0.1 chi)), chi_max =
1024, svd_min = 1e-14; Sec. III, Fig. 4 parameters) for its first 80 steps, in which chi
grows from 1 to ~650. Every 5 steps: <Z> on site 0 (Eq. 3's Z), both bond dimensions and
the accumulated eps. Calls only the oracle.

    python tests/golden/make_c3_trace.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import clock, mps  # noqa: E402

STEPS, EVERY = 80, 5
L, D, G, DT = 2, 5, 2.0, 0.02


def main():
    st = mps.product_state(L, D, 0, finite=False)
    half = clock.layer_gates(L, D, G, DT / 2, finite=False)
    full = clock.layer_gates(L, D, G, DT, finite=False)
    Z, _ = clock.clock_operators(D)
    rows = []
    for k in range(1, STEPS + 1):
        mps.tebd_step(st, half, full, scheme="cbe", chi_max=1024, dchi_min=100, dchi_frac=0.1,
                      svd_min=1e-14)
        if k % EVERY == 0:
            z = mps.expectation_1site(st, 0, Z)
            rows.append({"step": k, "z": [z.real, z.imag], "chi": st.bond_dims(), "eps_sum": st.eps_sum})
    out = {"workload": "C3: uniform two-site cell, d=5, g=2, |00>, dt=0.02, CBE dchi_min=100 "
                       "dchi_frac=0.1, chi_max=1024, svd_min=1e-14 (oracle, complex128)",
           "steps": STEPS, "trace": rows}
    with open(os.path.join(HERE, "c3_oracle_trace.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
