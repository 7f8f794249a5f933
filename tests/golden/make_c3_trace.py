"""Writes c3_oracle_trace.json: the oracle's run of the C3 workload (uniform two-site cell,
d = 5, g = 2.0, |00>, Strang dt = 0.02, CBE with dchi = max(100, ceil(0.1 chi)), chi_max =
1024, svd_min = 1e-14; Sec. III, Fig. 4 parameters) for its first 80 steps, in which chi
grows from 1 to ~650. Every 5 steps: <Z> on site 0 (Eq. 3's Z), both bond dimensions, the
number of Schmidt values above 1e-6 and above 1e-5 of the largest on each bond, and the
accumulated eps.
The oracle takes step (iv) as the paper states it, the eigenvalues of L^dag L, whose
absolute error ~1e-16 S_1^2 leaves every Schmidt value below ~1e-8 S_1 at rounding noise:
the bond dimension at svd_min = 1e-14 counts noise, the counts above 1e-6 S_1 (relative
error of the oracle's values there ~5e-5) and 1e-5 S_1 do not.
Calls only the oracle.

    python tests/golden/make_c3_trace.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import bond, clock, mps  # noqa: E402

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
            svs = [bond.schmidt_values(x) for x in st.Xi]
            rows.append({"step": k, "z": [z.real, z.imag], "chi": st.bond_dims(),
                         "n_above_1e-6": [int(np.sum(sv > 1e-6 * sv[0])) for sv in svs],
                         "n_above_1e-5": [int(np.sum(sv > 1e-5 * sv[0])) for sv in svs],
                         "eps_sum": st.eps_sum})
    out = {"workload": "C3: uniform two-site cell, d=5, g=2, |00>, dt=0.02, CBE dchi_min=100 "
                       "dchi_frac=0.1, chi_max=1024, svd_min=1e-14 (oracle, complex128)",
           "steps": STEPS, "trace": rows}
    with open(os.path.join(HERE, "c3_oracle_trace.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
