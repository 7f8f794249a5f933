"""Pins for the oracle's entanglement entropy (Fig. 4 plots S_vN on the central bond).

S_vN = -sum_k p_k ln p_k with p_k = S_k^2 / sum S^2, the Schmidt values S_k of the bond
matrix. The pins do not retype that formula: they fix the log base and the squaring by
closed forms, and tie the bond matrices of a TEBD run to the reduced density matrix of the
exact state vector, which is built without the MPS at all.
"""
import numpy as np
import pytest

from oracle import bond, exact, mps

from test_oracle_tebd import run_finite


def test_bell_pair_is_ln2():
    # two equal Schmidt values: S_vN = ln 2 (natural log; log2 would give 1)
    Xi = np.diag([1 / np.sqrt(2), 1 / np.sqrt(2)]).astype(np.complex128)
    assert abs(bond.entropy(Xi) - np.log(2)) < 1e-15


def test_maximally_entangled_d_levels_is_ln_d():
    # d equal Schmidt values in any basis (a unitary on either side): S_vN = ln d
    rng = np.random.default_rng(5)
    for d in (3, 5, 8):
        Ua, _ = np.linalg.qr(rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d)))
        Ub, _ = np.linalg.qr(rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d)))
        assert abs(bond.entropy(3.7 * Ua @ Ub) - np.log(d)) < 1e-13


def test_product_state_is_zero():
    assert bond.entropy(np.ones((1, 1), np.complex128)) == 0.0
    # one nonzero Schmidt value among zeros (a product state at a larger bond dimension)
    assert bond.entropy(np.diag([0.0, 2.0, 0.0]).astype(np.complex128)) == 0.0
    st = mps.product_state(6, 3)
    assert all(s == 0.0 for s in mps.entropies(st))


def test_two_values_closed_form():
    # S = (cos a, sin a): S_vN = -c^2 ln c^2 - s^2 ln s^2; a missing square (p = S) or a
    # missing normalisation (an unnormalised Xi) would change it
    for a in (0.1, 0.4, 0.7):
        c2, s2 = np.cos(a) ** 2, np.sin(a) ** 2
        Xi = 2.5 * np.array([[np.cos(a), 0], [0, np.sin(a)]], np.complex128)
        assert abs(bond.entropy(Xi) - (-c2 * np.log(c2) - s2 * np.log(s2))) < 1e-14


@pytest.mark.parametrize("scheme", ["plain", "cbe"])
def test_matches_reduced_density_matrix(scheme):
    # L = 6, d = 3, no truncation: the bond matrix of every bond carries the Schmidt
    # spectrum of the bipartition of the exact Trotterised state; its entropy must equal
    # -tr(rho ln rho) for the reduced density matrix of the left sites
    L, d, g, dt, steps = 6, 3, 1.5, 0.05, 8
    st = run_finite(L, d, g, dt, steps, chi_max=27, scheme=scheme, dchi_min=100)
    psi = exact.trotter_statevector(exact.product_vector(L, d), L, d, g, dt, steps)
    ent = mps.entropies(st)
    assert len(ent) == L + 1
    assert ent[0] == 0.0 and ent[L] == 0.0
    for b in range(1, L):
        M = psi.reshape(d ** b, d ** (L - b))
        rho = M @ M.conj().T
        w = np.linalg.eigvalsh(rho)
        w = w[w > 1e-300]
        s_ref = float(-(w * np.log(w)).sum())
        assert abs(ent[b] - s_ref) < 1e-11, (b, ent[b], s_ref)
    # the quench entangles every inner bond
    assert min(ent[1:L]) > 1e-3
