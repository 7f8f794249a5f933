"""GPU parity of the charge-sector CBE update (Sec. III with Z_d charges) against the oracle.

Same seeded inputs on both sides. The new bond's charges, the block dimensions chi~_q and
chi~ are integers and must agree exactly (the seeds have clean gaps at every cut); Schmidt
values and eps at the precision's tolerance; the kept subspace (projector, B~^m B~^n, Gram
matrix) at the Davis-Kahan tolerance of the merged spectrum's gap at the cut. Entries the
charge rule forbids must be exact zeros."""
import numpy as np
import pytest

from oracle import symmetric as sym
from paper_2212_09782_b300 import workloads as W
from tests.gpu_helpers import TOL, compare, host, rounded, subspace_tol, to_dev

pytestmark = pytest.mark.gpu

# name: chi_l, chi_m, chi_r, d, chi_max, dchi_min, seed, diagonal Xi
CASES = {
    "small_full": (12, 10, 14, 3, 1000, 100, 1, True),
    "cut": (60, 40, 52, 3, 45, 8, 2, True),
    "tiles_d5": (160, 150, 170, 5, 200, 20, 3, False),
    "ragged_d4": (97, 61, 75, 4, 90, 12, 5, True),
}


def _inputs(chi_l, chi_m, chi_r, d, seed, diag_xi, one_sector=False):
    r = W.rng(seed)
    cl, cm, cr = (W.random_charges(r, n, d) for n in (chi_l, chi_m, chi_r))
    if one_sector:
        cm = np.zeros(chi_m, int)
    th = W.symmetric_theta(r, cl, cr, d)
    xi = (np.sort(r.random(chi_l))[::-1] + 0.1) if diag_xi else None
    if xi is not None:
        xi = xi / np.linalg.norm(xi)
    U = W.charge_conserving_unitary(r, d)
    return cl, cm, cr, th, xi, U


def _run(prec, cl, cm, cr, th, xi, U, tr, bm=None, bn=None):
    import torch
    from paper_2212_09782_b300 import lib as L
    d = th.shape[1] if th is not None else bm.shape[1]
    up = L.SymBondUpdater(prec, d, cl, cm, cr, tr, xi_kind=2 if xi is not None else 0,
                          theta_given=th is not None)
    gate = torch.from_numpy(np.ascontiguousarray(U, np.complex128)).cuda()
    xi_dev = to_dev(xi.astype(np.complex128), prec) if xi is not None else None
    info = up.run(gate, theta=to_dev(th, prec) if th is not None else None, xi=xi_dev,
                  bm=to_dev(bm, prec) if bm is not None else None,
                  bn=to_dev(bn, prec) if bn is not None else None)
    L.stream_check()
    Bm, x, Bn, ch, st = up.outputs()
    return {"Bm_new": host(Bm), "Xi_new": np.diag(host(x)), "Bn_new": host(Bn), "charges": ch,
            "chi_sector": up.chi_sector.copy(), "eps": float(st[0].item()),
            "chi_new": info.chi_new, "eta_sum": info.eta}


def _check(gpu, orc, prec, cl, cr, d):
    assert gpu["chi_new"] == orc["chi_new"]
    assert np.array_equal(gpu["chi_sector"], orc["chi_sector"])
    assert np.array_equal(gpu["charges"], orc["charge_new"])
    assert gpu["eta_sum"] == sum(b["eta"] for b in orc["blocks"] if b is not None)
    o = {"Bm_new": orc["Bm_new"], "Xi_new": np.diag(orc["xi_new"]).astype(np.complex128),
         "Bn_new": orc["Bn_new"], "eps": orc["eps"]}
    tol = TOL[prec]
    errs = compare(gpu, o, tol, sub_tol=subspace_tol(tol, prec, orc["S"], orc["chi_new"]))
    # Schmidt values block by block (each block descending)
    sg, so = np.real(np.diag(gpu["Xi_new"])), orc["xi_new"]
    for q in range(d):
        a, b = sg[orc["charge_new"] == q], so[orc["charge_new"] == q]
        if len(b):
            assert np.max(np.abs(a - b)) <= tol * max(b[0], 1e-300) * 10, (q, a[:4], b[:4])
    # the charge rule: exact zeros outside it
    cn = orc["charge_new"]
    assert np.all(gpu["Bm_new"][~sym.allowed_site(cl, cn, d)] == 0)
    assert np.all(gpu["Bn_new"][~sym.allowed_site(cn, cr, d)] == 0)
    return errs


@pytest.mark.parametrize("prec", ["c128", "c64_3xtf32", "c64_fp32", "c64_tf32"])
@pytest.mark.parametrize("case", list(CASES))
def test_sym_update_matches_oracle(prec, case):
    from paper_2212_09782_b300 import lib as L
    chi_l, chi_m, chi_r, d, chi_max, dchi, seed, dx = CASES[case]
    cl, cm, cr, th, xi, U = _inputs(chi_l, chi_m, chi_r, d, seed, dx)
    th = rounded(th, prec)
    xi = None if xi is None else np.real(rounded(xi.astype(np.complex128), prec))
    tr = L.trunc_default(L.CBE, chi_max, dchi_min=dchi)
    orc = sym.sym_qr_update(th, xi, U, cl, cm, cr, chi_max=chi_max, dchi_min=dchi)
    gpu = _run(prec, cl, cm, cr, th, xi, U, tr)
    _check(gpu, orc, prec, cl, cr, d)


@pytest.mark.parametrize("prec", ["c128", "c64_3xtf32"])
def test_empty_middle_blocks_grow(prec):
    # the old middle bond has charge 0 only: every other block starts at chi_q = 0 and is
    # expanded by dchi_q = dchi_min; the cut hands states to every block
    from paper_2212_09782_b300 import lib as L
    cl, cm, cr, th, xi, U = _inputs(40, 12, 44, 3, 4, True, one_sector=True)
    th = rounded(th, prec)
    xi = np.real(rounded(xi.astype(np.complex128), prec))
    tr = L.trunc_default(L.CBE, 60, dchi_min=10)
    orc = sym.sym_qr_update(th, xi, U, cl, cm, cr, chi_max=60, dchi_min=10)
    gpu = _run(prec, cl, cm, cr, th, xi, U, tr)
    _check(gpu, orc, prec, cl, cr, 3)
    assert np.count_nonzero(gpu["chi_sector"]) == 3


@pytest.mark.parametrize("prec", ["c128", "c64_3xtf32"])
def test_from_site_tensors(prec):
    # theta' = B^m B^n formed in the library from charge-respecting site tensors
    from paper_2212_09782_b300 import lib as L
    r = W.rng(77)
    d, chi_l, chi_m, chi_r = 3, 30, 36, 33
    cl, cm, cr = (W.random_charges(r, n, d) for n in (chi_l, chi_m, chi_r))
    Bm = W.complex_gaussian(r, (chi_l, d, chi_m)) * sym.allowed_site(cl, cm, d)
    Bn = W.complex_gaussian(r, (chi_m, d, chi_r)) * sym.allowed_site(cm, cr, d)
    Bm, Bn = rounded(Bm / np.linalg.norm(Bm), prec), rounded(Bn, prec)
    U = W.charge_conserving_unitary(r, d)
    tr = L.trunc_default(L.CBE, 50, dchi_min=6)
    th = np.tensordot(Bm, Bn, axes=(2, 0))
    orc = sym.sym_qr_update(th, None, U, cl, cm, cr, chi_max=50, dchi_min=6)
    gpu = _run(prec, cl, cm, cr, None, None, U, tr, bm=Bm, bn=Bn)
    _check(gpu, orc, prec, cl, cr, d)


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["c64_3xtf32", "c128"])
def test_full_size_chi1024_d5(prec):
    # the C2 shape with Z_5 charges: chi = 1024, d = 5, charges spread over all sectors;
    # five 1024 x 1024 blocks, eta_q = chi_q + 100
    from paper_2212_09782_b300 import lib as L
    chi, d = 1024, 5
    r = W.rng(2212)
    cl, cm, cr = (W.random_charges(r, chi, d) for _ in range(3))
    th = rounded(W.symmetric_theta(r, cl, cr, d), prec)
    U = W.charge_conserving_unitary(r, d)
    tr = L.trunc_default(L.CBE, chi)
    orc = sym.sym_qr_update(th, None, U, cl, cm, cr, chi_max=chi)
    gpu = _run(prec, cl, cm, cr, th, None, U, tr)
    _check(gpu, orc, prec, cl, cr, d)


def test_chain_matches_oracle_chain():
    # L = 6, d = 3 clock chain from |0~ 0~ ...> in the charge basis, no truncation: every
    # bond update through the library; the state after 4 Strang steps equals the oracle's
    import torch
    from paper_2212_09782_b300 import lib as L
    Ls, d, g, dt, steps = 6, 3, 1.5, 0.05, 4
    prec = "c128"
    wts = [(1.0 if b == 0 else 0.5, 1.0 if b == Ls - 2 else 0.5) for b in range(Ls - 1)]
    half = [torch.from_numpy(L.clock_bond_gate_charge(d, g, wl, wr, dt / 2)).cuda() for wl, wr in wts]
    full = [torch.from_numpy(L.clock_bond_gate_charge(d, g, wl, wr, dt)).cuda() for wl, wr in wts]
    B = []
    for _ in range(Ls):
        b = np.zeros((1, d, 1), np.complex128)
        b[0, 0, 0] = 1
        B.append(to_dev(b, prec))
    xi = [to_dev(np.ones(1, np.complex128), prec) for _ in range(Ls + 1)]
    ch = [np.zeros(1, int) for _ in range(Ls + 1)]
    tr = L.trunc_default(L.CBE, 27, dchi_min=100, svd_min=0.0)
    for _ in range(steps):
        for gates, parity in ((half, 0), (full, 1), (half, 0)):
            for m in range(parity, Ls - 1, 2):
                up = L.SymBondUpdater(prec, d, ch[m], ch[m + 1], ch[m + 2], tr, xi_kind=2,
                                      theta_given=False)
                up.run(gates[m], xi=xi[m], bm=B[m], bn=B[m + 1])
                L.stream_check()
                bm, x, bn, c, _ = up.outputs()
                B[m], B[m + 1], xi[m + 1], ch[m + 1] = bm.clone(), bn.clone(), x.clone(), c
    st = sym.product_state(Ls, d, 0)
    oh = sym.layer_gates_charge_basis(Ls, d, g, dt / 2)
    of = sym.layer_gates_charge_basis(Ls, d, g, dt)
    for _ in range(steps):
        sym.tebd_step(st, oh, of, chi_max=27, dchi_min=100, svd_min=0.0)
    for b in range(Ls + 1):
        assert np.array_equal(ch[b], st.charges[b])
        assert np.allclose(np.real(host(xi[b])), st.xi[b], atol=1e-12)
    v = host(xi[0])[:, None, None] * host(B[0])
    for m in range(1, Ls):
        v = np.tensordot(v, host(B[m]), axes=(v.ndim - 1, 0))
    assert np.max(np.abs(v.reshape(-1) - sym.to_statevector(st))) < 1e-12
