"""Host side of the charge-sector CBE entry point (no GPU): the charge-basis clock gate
against the oracle's, the workspace query and the refusals it makes before any device work."""
import ctypes as C

import numpy as np
import pytest

from oracle import symmetric as sym


@pytest.fixture(scope="module")
def L():
    from paper_2212_09782_b300 import lib
    return lib


@pytest.mark.parametrize("d,g,wl,wr,tau", [(2, 1.0, 0.5, 0.5, 0.1), (3, 1.5, 1.0, 0.5, 0.025),
                                           (5, 2.0, 0.5, 1.0, 0.01), (4, 0.7, 0.5, 0.5, -0.05j)])
def test_charge_gate_matches_oracle(L, d, g, wl, wr, tau):
    U = L.clock_bond_gate_charge(d, g, wl, wr, tau)
    assert np.max(np.abs(U - sym.clock_gate_charge_basis(d, g, tau, wl, wr))) < 1e-13
    # entries that change the pair charge are exact zeros
    assert np.all(U[~sym.pair_charge_mask(d)] == 0)


def test_workspace_and_eta_sum(L):
    d, chi = 5, 50
    c = np.arange(chi) % d
    t = L.trunc_default(L.CBE, 1000, dchi_min=3)
    nb, eta_sum = L.sym_bond_workspace_size("c64_3xtf32", chi, d, chi, chi, c, c, c, t)
    # every block is chi_l x chi_r (each left state gives one row to every block);
    # eta_q = min(chi_q + max(3, ceil(0.1 chi_q)), chi_l, chi_r) with chi_q = 10
    assert eta_sum == d * 13 and nb > 0
    nb2, _ = L.sym_bond_workspace_size("c64_3xtf32", chi, d, chi, chi, c, c, c, t, theta_given=False)
    assert nb2 > nb  # theta' = B^m B^n needs its own buffer


@pytest.mark.parametrize("case", ["plain", "eta", "charge", "d", "xi_dense"])
def test_refusals(L, case):
    d, chi = 3, 12
    c = np.arange(chi) % d
    t = L.trunc_default(L.PLAIN if case == "plain" else L.CBE, 24)
    if case == "eta":
        t.eta = 5
    cl = c.copy()
    if case == "charge":
        cl[3] = d
    dd = 17 if case == "d" else d
    xk = 1 if case == "xi_dense" else 2
    with pytest.raises(L.QrtebdError) as e:
        L.sym_bond_workspace_size("c128", chi, dd, chi, chi, cl, c, c, t, xi_kind=xk)
    assert e.value.status == L.ERR_INVALID_ARG


def test_update_refuses_a_short_workspace_before_any_launch(L):
    d, chi = 3, 12
    c = np.arange(chi) % d
    t = L.trunc_default(L.CBE, 24)
    nb, _ = L.sym_bond_workspace_size("c128", chi, d, chi, chi, c, c, c, t, xi_kind=0)
    io = L.SymBondIO()
    io.precision, io.chi_l, io.d, io.chi_m, io.chi_r = L.C128, chi, d, chi, chi
    keep = [np.ascontiguousarray(c, np.int32) for _ in range(3)]
    io.charge_l, io.charge_m, io.charge_r = (k.ctypes.data_as(C.POINTER(C.c_int)) for k in keep)
    io.xi_kind = 0
    fake = 1 << 40  # never dereferenced: the refusal comes first
    io.theta, io.gate, io.bm_out, io.xi_out, io.bn_out = fake, fake, fake, fake, fake
    out = np.zeros(64, np.int32)
    io.charge_out = out.ctypes.data_as(C.POINTER(C.c_int))
    io.workspace, io.workspace_bytes = fake, nb - 1
    info = L.BondInfo()
    st = L.raw().qrtebd_sym_bond_update(C.byref(io), C.byref(t), None, C.byref(info))
    assert st == L.ERR_OOM
    assert b"workspace too small" in L.raw().qrtebd_last_error_message()
