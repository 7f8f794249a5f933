"""The C-ABI library loads and exports every symbol include/qrtebd.h declares (no GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import clock

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "qrtebd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qrtebd_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2212_09782_b300 import lib
    return lib


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 8
    so = ctypes.CDLL(L.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_version_and_strerror(L):
    assert "qrtebd" in L.version()
    assert L.strerror(0) == "ok"
    assert L.strerror(L.ERR_TIMEOUT) == "bounded wait expired"


def test_trunc_defaults(L):
    t = L.trunc_default(L.CBE, 1024)
    assert (t.scheme, t.chi_max, t.eta, t.dchi_min) == (L.CBE, 1024, 0, 100)
    assert t.dchi_frac == 0.1 and t.svd_min == 1e-14
    assert t.eps_target == 0.0 and t.reorth == -1   # re-orthogonalisation: per precision


def test_reorth_pass_workspace(L):
    # the pass takes D (eta x eta) and a second isometry buffer (d chi_r x eta): by default
    # on the 1xTF32 precision only, and nothing when it is off
    args = (1024, 5, 1024, 1024)
    for prec, auto_on in ((L.C64_TF32, True), (L.C64_3XTF32, False)):
        auto = L.bond_workspace_size(prec, *args, L.trunc_default(L.PLAIN, 1024), xi_kind=0,
                                     theta_given=True)
        on = L.bond_workspace_size(prec, *args, L.trunc_default(L.PLAIN, 1024, reorth=1),
                                   xi_kind=0, theta_given=True)
        off = L.bond_workspace_size(prec, *args, L.trunc_default(L.PLAIN, 1024, reorth=0),
                                    xi_kind=0, theta_given=True)
        assert on - off >= (1024 * 1024 + 5120 * 1024) * 8
        assert auto == (on if auto_on else off)
    c128 = L.trunc_default(L.PLAIN, 1024)
    assert (L.bond_workspace_size(L.C128, *args, c128, xi_kind=0, theta_given=True) ==
            L.bond_workspace_size(L.C128, *args, L.trunc_default(L.PLAIN, 1024, reorth=0),
                                  xi_kind=0, theta_given=True))


def test_workspace_size_query_needs_no_gpu(L):
    t = L.trunc_default(L.PLAIN, 1024)
    n64 = L.bond_workspace_size(L.C64_3XTF32, 1024, 5, 1024, 1024, t, xi_kind=0, theta_given=True)
    n128 = L.bond_workspace_size(L.C128, 1024, 5, 1024, 1024, t, xi_kind=0, theta_given=True)
    assert n64 > 5120 * 5120 * 8 and n128 > 5120 * 5120 * 16
    with pytest.raises(L.QrtebdError):  # eta larger than d * chi
        L.bond_workspace_size(L.C128, 2, 2, 2, 2, L.trunc_default(L.PLAIN, 100, eta=50))


@pytest.mark.parametrize("d,g,wl,wr,tau", [(2, 1.0, 0.5, 0.5, 0.05), (3, 1.5, 1.0, 0.5, 0.025),
                                           (5, 2.0, 0.5, 1.0, 0.01), (4, 0.7, 0.5, 0.5, -0.3j)])
def test_clock_gate_matches_oracle(L, d, g, wl, wr, tau):
    U = L.clock_bond_gate(d, g, wl, wr, tau)
    Uo = clock.trotter_gate(clock.bond_hamiltonian(d, g, wl, wr), tau)
    assert np.abs(U - Uo).max() < 1e-12


def test_invalid_arguments_rejected(L):
    with pytest.raises(L.QrtebdError):
        L.clock_bond_gate(1, 1.0, 0.5, 0.5, 0.1)


def test_autotune_table_host(L):
    # the autotuner's table on the host: insert, replace, order, validation (no GPU work)
    import ctypes as C
    raw = L.raw()
    L.autotune_clear()
    try:
        assert raw.qrtebd_autotune_count() == 0
        L.autotune_set((512, 256, 1024, 1), (128, 4, 0))
        L.autotune_set((512, 256, 1024, 0), (256, 0, 1))
        L.autotune_set((512, 256, 1024, 1), (256, 2, 0))  # replaces the first
        e = L.autotune_entries()
        assert [x["shape"] for x in e] == [(512, 256, 1024, 0), (512, 256, 1024, 1)]
        assert e[1]["config"] == (256, 2, 0) and e[1]["ms_tuned"] == 0.0
        for bad in [((256, 512, 1024, 1), (128, 1, 0)),   # M < N: not a swapped shape
                    ((512, 256, 1024, 1), (64, 1, 0)),    # no such tile width
                    ((512, 256, 1024, 1), (128, 33, 0))]: # more K-splits than allowed
            with pytest.raises(L.QrtebdError):
                L.autotune_set(*bad)
        # precisions without tensor-core products tune nothing and touch no GPU
        n = C.c_int(-1)
        t = L.trunc_default(L.PLAIN, 64)
        assert raw.qrtebd_autotune_bond(L.C128, 64, 3, 64, 64, 0, 1, C.byref(t), None, C.byref(n)) == 0
        assert n.value == 0
    finally:
        L.autotune_clear()


def test_autotune_table_save_load(L, tmp_path):
    # a table saved as JSON and loaded again gives the same shapes and configurations
    L.autotune_clear()
    try:
        L.autotune_set((1024, 128, 5120, 1), (128, 8, 0))
        L.autotune_set((4992, 896, 128, 1), (256, 1, 0))
        path = str(tmp_path / "tune.json")
        L.autotune_save(path)
        before = [(e["shape"], e["config"]) for e in L.autotune_entries()]
        L.autotune_clear()
        assert L.autotune_load(path) == 2
        assert [(e["shape"], e["config"]) for e in L.autotune_entries()] == before
    finally:
        L.autotune_clear()


def test_binding_refuses_strided_tensors(L):
    # the C ABI reads dense row-major data: a transposed or permuted view would be read in
    # the wrong order, so the binding refuses it instead of passing its base pointer
    import torch
    t = torch.zeros(4, 6, dtype=torch.complex64)
    assert L._ptr(t) is not None
    with pytest.raises(ValueError):
        L._ptr(t.t())
    with pytest.raises(ValueError):
        L._ptr(torch.zeros(3, 4, 5, dtype=torch.complex64).permute(0, 2, 1))
    # a row-strided block (leading dimension > width) is fine where the ABI takes it
    big = torch.zeros(8, 8, dtype=torch.complex64)
    assert L._ptr_rows(big[:4, :4]) is not None
    with pytest.raises(ValueError):
        L._ptr_rows(big.t())


def test_workload_arrays_are_row_major():
    from paper_2212_09782_b300 import workloads as W
    wl = W.bond_microbench(16, 3)
    for k in ("theta", "U", "Bn"):
        assert wl[k].flags["C_CONTIGUOUS"], k
    r = W.rng(1)
    assert W.random_right_isometry(r, 5, 3, 4).flags["C_CONTIGUOUS"]
