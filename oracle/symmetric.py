"""Oracle (test infrastructure): controlled bond expansion with Z_d charge sectors.

Sec. III (closing paragraphs): with a global symmetry the bond indices carry charges and
every tensor is block-sparse. CBE lets the block dimensions chi_q change from update to
update: each block is expanded on its own (chi_q -> chi_q + dchi_q) and one cut over the
Schmidt values of all blocks together keeps the dominant ones, so that the blocks end up
with the dimensions an SVD truncation of the whole theta~ would give.

The clock model (Eqs. 2-3) has the Z_d symmetry generated by prod_n X_n. In the basis that
diagonalises X (the Fourier basis of each site) the label k of a site state is its charge:
X|k> = w^k |k>, Z raises k by one, so Z x Z^dag conserves k1 + k2 mod d.

Conventions (readings where the paper is silent; each is listed in the design notes):
  * charges are integers mod d; a bond index alpha carries c(alpha). A site tensor
    B^i_{alpha beta} is nonzero only when c_left(alpha) + i = c_right(beta) (mod d), so a
    charge flows left to right and the last bond carries the total charge.
  * theta'^{ij}_{alpha delta} = B^m B^n is nonzero only when c_l(alpha) + i + j = c_r(delta).
  * the central bond sector q holds the rows (alpha, i) of theta~ with c_l(alpha) + i = q and
    the columns (j, delta) with c_r(delta) - j = q, both in the dense order (row alpha*d + i,
    column j*chi_r + delta); theta~ has no entries outside these blocks.
  * per block: eta_q = min(chi_q + dchi_q, |rows_q|, |cols_q|) with chi_q the number of old
    middle-bond states of charge q and dchi_q = max(dchi_min, ceil(dchi_frac chi_q)) (the
    dense CBE policy applied block by block); Y0_q = the first eta_q rows of theta~_q.
  * the cut: the Schmidt values of all blocks in one list, in descending order with equal
    values ordered by (charge, position in the block); the dense rule (``bond.cbe_cut``:
    svd_min relative to the norm of all values, chi_max, eps_target, never inside a
    multiplet) picks how many to keep; chi~_q counts the kept values of block q.
  * the new middle bond lists the kept states block by block in increasing charge, each
    block in descending Schmidt order; Xi~ is diagonal with unit norm over all blocks.
"""
import numpy as np

from . import bond as _bond
from . import clock as _clock


# ------------------------------------------------------------------ basis and gates
def fourier_basis(d):
    """F (d x d, unitary): column k is the eigenvector of X (Eq. 3) with eigenvalue w^k."""
    n = np.arange(d)
    return np.exp(2j * np.pi * np.outer(n, n) / d) / np.sqrt(d)


def to_charge_basis(U, d):
    """A two-site operator in the Fourier basis of both sites: (F x F)^dag U (F x F)."""
    F2 = np.kron(fourier_basis(d), fourier_basis(d))
    return F2.conj().T @ U @ F2


def pair_charge_mask(d):
    """Boolean d^2 x d^2 mask of the entries (i j),(i' j') with i + j = i' + j' (mod d)."""
    t = np.add.outer(np.arange(d), np.arange(d)).reshape(-1) % d
    return t[:, None] == t[None, :]


def clock_gate_charge_basis(d, g, tau, wl=0.5, wr=0.5):
    """exp(-i tau h_b) of the clock model in the charge basis, with the entries that the
    symmetry forbids set to zero (they are rounding noise of the basis change)."""
    Uc = to_charge_basis(_clock.trotter_gate(_clock.bond_hamiltonian(d, g, wl, wr), tau), d)
    return np.where(pair_charge_mask(d), Uc, 0.0)


def layer_gates_charge_basis(L, d, g, tau):
    """Gates for every bond of a finite chain, in the charge basis."""
    return [clock_gate_charge_basis(d, g, tau, wl, wr) for (wl, wr) in _clock.field_weights(L, True)]


# ------------------------------------------------------------------ sectors
def sector_rows(charge_l, d):
    """Row indices alpha*d + i of theta~ per central charge q = c_l(alpha) + i (mod d)."""
    cl = np.asarray(charge_l)
    qrow = (cl[:, None] + np.arange(d)[None, :]) % d  # (chi_l, d), row-major = alpha*d + i
    flat = qrow.reshape(-1)
    return [np.nonzero(flat == q)[0] for q in range(d)]


def sector_cols(charge_r, d):
    """Column indices j*chi_r + delta of theta~ per central charge q = c_r(delta) - j."""
    cr = np.asarray(charge_r)
    qcol = (cr[None, :] - np.arange(d)[:, None]) % d  # (d, chi_r), row-major = j*chi_r + delta
    flat = qcol.reshape(-1)
    return [np.nonzero(flat == q)[0] for q in range(d)]


def allowed_theta(charge_l, charge_r, d):
    """Boolean (chi_l, d, d, chi_r) mask of the entries of theta' the charge rule allows."""
    cl, cr = np.asarray(charge_l), np.asarray(charge_r)
    s = (cl[:, None, None, None] + np.arange(d)[None, :, None, None]
         + np.arange(d)[None, None, :, None]) % d
    return s == cr[None, None, None, :]


def allowed_site(charge_l, charge_r, d):
    """Boolean (chi_l, d, chi_r) mask: c_l(alpha) + i = c_r(beta) (mod d)."""
    cl, cr = np.asarray(charge_l), np.asarray(charge_r)
    return ((cl[:, None, None] + np.arange(d)[None, :, None]) % d) == cr[None, None, :]


def block_eta(n_rows, n_cols, chi_q, dchi_min, dchi_frac):
    """eta_q of one block (the dense CBE policy per block); 0 for an empty block."""
    if n_rows == 0 or n_cols == 0:
        return 0
    dchi = max(dchi_min, int(np.ceil(dchi_frac * chi_q - 1e-9)))
    return int(min(chi_q + dchi, n_rows, n_cols))


# ------------------------------------------------------------------ one bond
def sym_qr_update(theta, xi_diag, U, charge_l, charge_m, charge_r, *, chi_max, dchi_min=100,
                  dchi_frac=0.1, svd_min=1e-14, tie_tol=1e-10, eps_target=0.0):
    """One CBE update of a charge-conserving two-site block (Sec. III, steps (i)-(v), per block).

    theta: theta' (chi_l, d, d, chi_r) in the charge basis, zero where the charge rule
    forbids; xi_diag: the diagonal of Xi on the left bond (chi_l,) or None (identity);
    U: the gate (d^2 x d^2, charge-conserving). Returns the dense tensors Bm_new
    (chi_l, d, chi~), Bn_new (chi~, d, chi_r), the diagonal xi_new (chi~,), the charges of
    the new middle bond, chi~ per charge, eps, the merged Schmidt values S (descending) and
    the per-block dense updates.
    """
    chiL, d, _, chiR = theta.shape
    charge_l = np.asarray(charge_l) % d
    charge_m = np.asarray(charge_m) % d
    charge_r = np.asarray(charge_r) % d
    xi = np.ones(chiL) if xi_diag is None else np.asarray(xi_diag)

    # (i) theta~' = U theta', theta~ = Xi theta~' (dense arithmetic; the blocks are read next)
    Tp = _bond.apply_gate(U, theta).reshape(chiL * d, d * chiR)
    rows, cols = sector_rows(charge_l, d), sector_cols(charge_r, d)
    row_xi = np.repeat(xi, d)  # Xi acts on alpha of row alpha*d + i

    blocks = []
    for q in range(d):
        chi_q = int(np.sum(charge_m == q))
        eta_q = block_eta(len(rows[q]), len(cols[q]), chi_q, dchi_min, dchi_frac)
        if eta_q == 0:
            blocks.append(None)
            continue
        Tp_q = Tp[np.ix_(rows[q], cols[q])]
        # steps (i)-(iv) of the block: the dense CBE update with every Schmidt value kept
        res = _bond.qr_update(np.diag(row_xi[rows[q]]).astype(np.complex128), None, None,
                              np.ones((1, 1), np.complex128), scheme="cbe", chi_max=eta_q,
                              eta=eta_q, svd_min=0.0, tie_tol=0.0,
                              theta=Tp_q.reshape(len(rows[q]), 1, 1, len(cols[q])))
        res["q"] = q
        res["rows"], res["cols"] = rows[q], cols[q]
        res["T"] = res["theta_t"].reshape(len(rows[q]), len(cols[q]))
        blocks.append(res)

    # (iv)-(v) one cut over all blocks
    merged = [(-float(b["S"][k]), b["q"], k) for b in blocks if b is not None
              for k in range(len(b["S"]))]
    merged.sort()
    S_all = np.array([-v for v, _, _ in merged])
    c = _bond.cbe_cut(S_all, chi_max, svd_min, tie_tol, eps_target)
    chi_sec = np.zeros(d, int)
    for _, q, _ in merged[:c]:
        chi_sec[q] += 1

    kept2 = sum(float(np.sum(b["S"][: chi_sec[b["q"]]] ** 2)) for b in blocks if b is not None)
    nrm2 = sum(float(np.vdot(b["T"], b["T"]).real) for b in blocks if b is not None)
    chi_new = int(chi_sec.sum())
    Bm_new = np.zeros((chiL * d, chi_new), np.complex128)
    Bn_new = np.zeros((chi_new, d * chiR), np.complex128)
    xi_new = np.zeros(chi_new)
    charge_new = np.zeros(chi_new, int)
    resid2 = 0.0
    off = 0
    for b in blocks:
        if b is None:
            continue
        q, k = b["q"], chi_sec[b["q"]]
        Bn_q = b["Bn_new"].reshape(-1, len(b["cols"]))[:k]  # P V Q^[n]
        Bm_q = b["Bm_new"].reshape(len(b["rows"]), -1)[:, :k]  # theta~' B~^n^dag
        Bm_new[np.ix_(b["rows"], np.arange(off, off + k))] = Bm_q
        Bn_new[np.ix_(np.arange(off, off + k), b["cols"])] = Bn_q
        xi_new[off:off + k] = b["S"][:k]
        charge_new[off:off + k] = q
        # explicit distance of the block (Sec. IV): theta~_q - Q L V^dag P V Q^[n]
        P = np.zeros(len(b["S"]))
        P[:k] = 1.0
        V = b["V"]
        approx = b["Q"] @ b["L"] @ (V.conj().T @ (P[:, None] * V)) @ b["Qn"]
        diff = b["T"] - approx
        resid2 += float(np.vdot(diff, diff).real)
        off += k
    xi_new = xi_new / np.sqrt(kept2) if kept2 > 0 else xi_new
    return {
        "Bm_new": Bm_new.reshape(chiL, d, chi_new),
        "Bn_new": Bn_new.reshape(chi_new, d, chiR),
        "xi_new": xi_new,
        "charge_new": charge_new,
        "chi_sector": chi_sec,
        "eps": resid2 / nrm2 if nrm2 > 0 else 0.0,
        "eps_kept": 1.0 - kept2 / nrm2 if nrm2 > 0 else 0.0,
        "norm2_theta": nrm2,
        "S": S_all,
        "chi_new": chi_new,
        "blocks": blocks,
    }


# ------------------------------------------------------------------ chain
class SymMPS:
    """Finite chain in right-isometric form with charges on every bond (Eq. 1, Fig. 1).

    B[m] (chi_m, d, chi_{m+1}) obeys the charge rule of its two bonds; xi[m] is the diagonal
    of the bond matrix left of site m; charges[m] lists c(alpha) on bond m."""

    def __init__(self, B, xi, charges):
        self.B = [np.array(b, np.complex128) for b in B]
        self.xi = [np.array(x, float) for x in xi]
        self.charges = [np.array(c, int) for c in charges]
        self.L = len(B)
        self.d = self.B[0].shape[1]
        self.eps_sum = 0.0

    def bond_dims(self):
        return [len(c) for c in self.charges]


def product_state(L, d, k=0):
    """|k~ k~ ... k~> in the charge basis: every bond of dimension 1, charge m*k on bond m."""
    B, xi, ch = [], [], []
    for m in range(L):
        b = np.zeros((1, d, 1), np.complex128)
        b[0, k, 0] = 1.0
        B.append(b)
    for m in range(L + 1):
        xi.append(np.ones(1))
        ch.append(np.array([(m * k) % d]))
    return SymMPS(B, xi, ch)


def update_bond(st, m, U, **trunc):
    """The gate U on (m, m+1): theta' = B^m B^n, then ``sym_qr_update``."""
    th = np.tensordot(st.B[m], st.B[m + 1], axes=(2, 0))
    res = sym_qr_update(th, st.xi[m], U, st.charges[m], st.charges[m + 1], st.charges[m + 2],
                        **trunc)
    st.B[m], st.B[m + 1] = res["Bm_new"], res["Bn_new"]
    st.xi[m + 1] = res["xi_new"]
    st.charges[m + 1] = res["charge_new"]
    st.eps_sum += res["eps"]
    return res


def tebd_step(st, half, full, **trunc):
    """One Strang step even(dt/2), odd(dt), even(dt/2) on a finite chain (Fig. 2a)."""
    for gates, parity in ((half, 0), (full, 1), (half, 0)):
        for m in range(parity, st.L - 1, 2):
            update_bond(st, m, gates[m], **trunc)


def to_statevector(st):
    """The d^L state vector in the charge basis, site 0 most significant."""
    v = st.xi[0][:, None, None] * st.B[0]
    for m in range(1, st.L):
        v = np.tensordot(v, st.B[m], axes=(v.ndim - 1, 0))
    return v.reshape(-1)


def statevector_to_clock_basis(v, L, d):
    """Back to the Z eigenbasis of Eq. 3: apply F on every site."""
    F = fourier_basis(d)
    t = v.reshape((d,) * L)
    for s in range(L):
        t = np.moveaxis(np.tensordot(F, t, axes=(1, s)), 0, s)
    return t.reshape(-1)
