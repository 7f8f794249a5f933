"""Pins for the oracle's charge-sector CBE (Sec. III, closing paragraphs: with symmetries the
blocks expand one by one and one cut over all blocks picks their dimensions).

Nothing here retypes the block algorithm. The pins are:
  * the Fourier basis diagonalises X and turns Z into a charge raise (Eq. 3), and the clock
    gates conserve the pair charge to rounding (the symmetry the blocks rest on);
  * with every block fully expanded the update reproduces theta~' exactly and its Schmidt
    values are the singular values of the dense theta~ (LAPACK SVD of the whole matrix);
  * truncated, it keeps the chi largest dense singular values (Eckart-Young), its eps is the
    dense discarded weight, and each block's dimension equals the number of those dense
    singular vectors that live in the block: the per-block dimensions the paper says CBE
    picks;
  * the outputs obey the charge rule, and blocks that were empty acquire states;
  * a chain evolved by the block update equals the exact Trotterised state vector (no
    truncation), and, truncated, matches the dense CBE oracle run on the same chain.
"""
import numpy as np
import pytest

from oracle import bond, clock, exact, mps
from oracle import symmetric as sym
from paper_2212_09782_b300 import workloads as W


def _inputs(seed, chi_l=7, d=3, chi_m=5, chi_r=8):
    r = W.rng(seed)
    cl, cm, cr = (W.random_charges(r, n, d) for n in (chi_l, chi_m, chi_r))
    th = W.symmetric_theta(r, cl, cr, d)
    xi = np.sort(r.random(chi_l))[::-1] + 0.1
    U = W.charge_conserving_unitary(r, d)
    return cl, cm, cr, th, xi, U


def _dense_T(th, xi, U):
    chiL, d, _, chiR = th.shape
    tp = bond.apply_gate(U, th)
    return tp.reshape(chiL * d, d * chiR), (xi[:, None, None, None] * tp).reshape(chiL * d, d * chiR)


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_fourier_basis_and_charge(d):
    F = sym.fourier_basis(d)
    Z, X = clock.clock_operators(d)
    w = np.exp(2j * np.pi / d)
    assert np.allclose(F.conj().T @ F, np.eye(d), atol=1e-14)
    assert np.allclose(F.conj().T @ X @ F, np.diag(w ** np.arange(d)), atol=1e-14)
    # Z raises the charge by one (cyclically)
    Zc = F.conj().T @ Z @ F
    raise_ = np.zeros((d, d))
    for k in range(d):
        raise_[(k + 1) % d, k] = 1.0
    assert np.allclose(Zc, raise_, atol=1e-14)


@pytest.mark.parametrize("d", [2, 3, 5])
def test_clock_gate_conserves_pair_charge(d):
    U = clock.trotter_gate(clock.bond_hamiltonian(d, 1.3, 0.5, 1.0), 0.07)
    Uc = sym.to_charge_basis(U, d)
    mask = sym.pair_charge_mask(d)
    assert np.max(np.abs(Uc[~mask])) < 1e-14
    Ug = sym.clock_gate_charge_basis(d, 1.3, 0.07, 0.5, 1.0)
    assert np.allclose(Ug.conj().T @ Ug, np.eye(d * d), atol=1e-13)
    F2 = np.kron(sym.fourier_basis(d), sym.fourier_basis(d))
    assert np.allclose(F2 @ Ug @ F2.conj().T, U, atol=1e-13)


def test_sectors_partition_theta():
    cl, cm, cr, th, xi, U = _inputs(11)
    d = th.shape[1]
    rows, cols = sym.sector_rows(cl, d), sym.sector_cols(cr, d)
    assert sorted(np.concatenate(rows)) == list(range(len(cl) * d))
    assert sorted(np.concatenate(cols)) == list(range(len(cr) * d))
    mask = sym.allowed_theta(cl, cr, d).reshape(len(cl) * d, d * len(cr))
    blocks = np.zeros_like(mask)
    for q in range(d):
        blocks[np.ix_(rows[q], cols[q])] = True
    assert np.array_equal(mask, blocks)
    # the gate keeps theta~' inside the blocks
    Tp, _ = _dense_T(th, xi, U)
    assert np.max(np.abs(Tp[~mask])) < 1e-15


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_full_expansion_is_exact(seed):
    cl, cm, cr, th, xi, U = _inputs(seed)
    d = th.shape[1]
    res = sym.sym_qr_update(th, xi, U, cl, cm, cr, chi_max=1000, dchi_min=1000, svd_min=0.0)
    Tp, T = _dense_T(th, xi, U)
    rec = np.tensordot(res["Bm_new"], res["Bn_new"], axes=(2, 0)).reshape(Tp.shape)
    assert np.max(np.abs(rec - Tp)) < 1e-13
    Bn = res["Bn_new"].reshape(res["chi_new"], -1)
    assert np.allclose(Bn @ Bn.conj().T, np.eye(res["chi_new"]), atol=1e-13)
    sv = np.linalg.svd(T, compute_uv=False)
    n = min(len(sv), len(res["S"]))
    assert np.allclose(res["S"][:n], sv[:n], atol=1e-13)
    assert res["eps"] < 1e-26 and abs(res["eps_kept"]) < 1e-14
    assert abs(np.sum(res["xi_new"] ** 2) - 1) < 1e-14


@pytest.mark.parametrize("seed,k", [(4, 5), (5, 9), (6, 3)])
def test_truncation_is_eckart_young_with_block_dims(seed, k):
    cl, cm, cr, th, xi, U = _inputs(seed, chi_l=9, chi_r=9)
    d = th.shape[1]
    res = sym.sym_qr_update(th, xi, U, cl, cm, cr, chi_max=k, dchi_min=1000, tie_tol=0.0)
    _, T = _dense_T(th, xi, U)
    _, sv, Vh = np.linalg.svd(T)
    assert sv[k - 1] - sv[k] > 1e-6  # a clean gap at the cut
    assert res["chi_new"] == k
    # the kept values are the k largest dense singular values, renormalised
    kept = np.sort(res["xi_new"])[::-1]
    assert np.allclose(kept, sv[:k] / np.linalg.norm(sv[:k]), atol=1e-13)
    tail = np.sum(sv[k:] ** 2) / np.sum(sv ** 2)
    assert abs(res["eps"] - tail) < 1e-13 and abs(res["eps_kept"] - tail) < 1e-13
    # block dimensions: how many of the k dominant dense singular vectors each block holds
    cols = sym.sector_cols(cr, d)
    want = np.zeros(d, int)
    for v in Vh[:k]:
        want[int(np.argmax([np.linalg.norm(v[c]) for c in cols]))] += 1
    assert np.array_equal(res["chi_sector"], want)


def test_outputs_obey_charge_rule_and_order():
    cl, cm, cr, th, xi, U = _inputs(7)
    d = th.shape[1]
    res = sym.sym_qr_update(th, xi, U, cl, cm, cr, chi_max=10, dchi_min=2)
    cn = res["charge_new"]
    assert np.all(np.diff(cn) >= 0)  # blocks in increasing charge
    for q in range(d):  # descending inside each block
        assert np.all(np.diff(res["xi_new"][cn == q]) <= 0)
    assert np.all(res["Bm_new"][~sym.allowed_site(cl, cn, d)] == 0)
    assert np.all(res["Bn_new"][~sym.allowed_site(cn, cr, d)] == 0)
    assert np.array_equal(np.bincount(cn, minlength=d), res["chi_sector"])


def test_empty_blocks_acquire_states():
    # the old middle bond has charge 0 only; theta~ has weight in every block, and the
    # expansion gives every block dchi states to offer to the cut
    r = W.rng(21)
    d = 3
    cl, cr = W.random_charges(r, 6, d), W.random_charges(r, 6, d)
    cm = np.zeros(2, int)
    th = W.symmetric_theta(r, cl, cr, d)
    U = W.charge_conserving_unitary(r, d)
    res = sym.sym_qr_update(th, None, U, cl, cm, cr, chi_max=12, dchi_min=4)
    assert np.count_nonzero(res["chi_sector"]) == d
    etas = [b["eta"] for b in res["blocks"] if b is not None]
    assert etas[1] == min(4, len(sym.sector_rows(cl, d)[1]), len(sym.sector_cols(cr, d)[1]))


def _sym_chain(L, d, g, dt, steps, **tr):
    st = sym.product_state(L, d, 0)
    half = sym.layer_gates_charge_basis(L, d, g, dt / 2)
    full = sym.layer_gates_charge_basis(L, d, g, dt)
    for _ in range(steps):
        sym.tebd_step(st, half, full, **tr)
    return st


def test_chain_equals_trotterised_statevector():
    L, d, g, dt, steps = 6, 3, 1.5, 0.05, 6
    # svd_min = 0: nothing is cut (the default 1e-14 drops weight ~1e-21, amplitudes ~1e-11)
    st = _sym_chain(L, d, g, dt, steps, chi_max=27, dchi_min=100, svd_min=0.0)
    v = sym.statevector_to_clock_basis(sym.to_statevector(st), L, d)
    # |0~>^L in the clock basis: the uniform superposition on every site
    psi0 = np.ones(d ** L, np.complex128) / np.sqrt(d ** L)
    psi = exact.trotter_statevector(psi0, L, d, g, dt, steps)
    assert np.max(np.abs(v - psi)) < 1e-13
    assert st.eps_sum < 1e-26
    # the charge-0 product state spreads over every charge of the central bond
    assert len(set(st.charges[L // 2].tolist())) == d


def test_truncated_chain_matches_dense_cbe():
    # with every block fully expanded the block update is the SVD cut of the whole theta~,
    # as is the dense CBE with eta = d chi: both chains keep the same Schmidt values
    # dt = 0.2: the cut is active (eps ~ 2e-2) and, at chi = 8, falls inside a charge-conjugate
    # pair on two bonds, which both chains then keep whole (bond dimension 7)
    L, d, g, dt, steps, chi = 8, 3, 1.5, 0.2, 6, 8
    st = _sym_chain(L, d, g, dt, steps, chi_max=chi, dchi_min=1000)
    dn = mps.product_state(L, d, 0, True)
    half = sym.layer_gates_charge_basis(L, d, g, dt / 2)
    full = sym.layer_gates_charge_basis(L, d, g, dt)
    for _ in range(steps):
        mps.tebd_step(dn, half, full, scheme="cbe", chi_max=chi, dchi_min=1000)
    assert st.eps_sum > 1e-3  # the cut is active
    assert 7 in st.bond_dims()
    assert abs(st.eps_sum - dn.eps_sum) < 1e-12
    for b in range(1, L):
        s_sym = np.sort(st.xi[b])[::-1]
        s_den = bond.schmidt_values(dn.Xi[b])
        assert len(s_sym) == len(s_den)
        assert np.allclose(s_sym, s_den, atol=1e-11)
    Xd = np.diag(2 * np.cos(2 * np.pi * np.arange(d) / d)).astype(np.complex128)
    for m in range(L):
        C = st.xi[m][:, None, None] * st.B[m]
        xs = np.einsum("aib,ij,ajb->", C.conj(), Xd, C)
        assert abs(xs - mps.expectation_1site(dn, m, Xd)) < 1e-11
