"""Oracle (test infrastructure): MPS in right-isometric form and the TEBD driver.

State (Eq. 1, Fig. 1): site tensors B[m] of shape (chi_m, d, chi_{m+1}), right
isometric (sum_{i beta} B B^* = 1, Sec. II), and bond matrices Xi[m] on the bond
left of site m, so that the state is sum |alpha>_left Xi[m]_{alpha beta} |beta>_right.

* finite chain of L sites: bonds 0..L, Xi[0] = Xi[L] = [[1]]; a gate on (m, m+1)
  reads Xi[m] and writes Xi[m+1] (Sec. II last paragraph: finite systems).
* uniform MPS with a two-site unit cell (Fig. 1a): sites A = 0, B = 1; Xi[0] sits
  between B and A, Xi[1] between A and B; bond (A,B) reads Xi[0] and writes Xi[1],
  bond (B,A) reads Xi[1] and writes Xi[0].

Time step: second-order Strang splitting with even and odd layers (Fig. 2a):
even(dt/2), odd(dt), even(dt/2) per step, not merged across steps (a reading;
the paper does not state the order).
"""
import numpy as np

from . import bond as _bond
from . import clock as _clock


class MPS:
    def __init__(self, B, Xi, finite=True):
        self.B = [np.array(b, dtype=np.complex128) for b in B]
        self.Xi = [np.array(x, dtype=np.complex128) for x in Xi]
        self.finite = finite
        self.L = len(B)
        self.d = B[0].shape[1]
        self.eps_sum = 0.0
        self.eps_log = []

    def copy(self):
        m = MPS(self.B, self.Xi, self.finite)
        m.eps_sum = self.eps_sum
        m.eps_log = list(self.eps_log)
        return m

    def bond_dims(self):
        return [b.shape[0] for b in self.B] + ([self.B[-1].shape[2]] if self.finite else [])


def product_state(L, d, k=0, finite=True):
    """|k k ... k> with chi = 1 everywhere; Xi = [[1]] on every bond."""
    B = []
    for _ in range(L):
        b = np.zeros((1, d, 1), np.complex128)
        b[0, k, 0] = 1.0
        B.append(b)
    nxi = L + 1 if finite else L
    Xi = [np.ones((1, 1), np.complex128) for _ in range(nxi)]
    return MPS(B, Xi, finite)


def layer_bonds(L, parity, finite=True):
    """Left sites m of the bonds (m, m+1 mod L) in one layer (Fig. 2a)."""
    if finite:
        return list(range(parity, L - 1, 2))
    return list(range(parity, L, 2))


def update_bond(mps, m, U, **trunc):
    """Apply gate U on (m, m+1) with the QR update (Sec. II / Sec. III)."""
    n = (m + 1) % mps.L
    res = _bond.qr_update(mps.Xi[m], mps.B[m], mps.B[n], U, **trunc)
    mps.B[m] = res["Bm_new"]
    mps.B[n] = res["Bn_new"]
    nb = m + 1 if mps.finite else n
    mps.Xi[nb] = res["Xi_new"]
    mps.eps_sum += res["eps"]
    mps.eps_log.append(res["eps"])
    return res


def update_bond_svd(mps, m, U, chi_max, svd_min=1e-14):
    n = (m + 1) % mps.L
    res = _bond.svd_update(mps.Xi[m], mps.B[m], mps.B[n], U, chi_max=chi_max, svd_min=svd_min)
    mps.B[m] = res["Bm_new"]
    mps.B[n] = res["Bn_new"]
    nb = m + 1 if mps.finite else n
    mps.Xi[nb] = res["Xi_new"]
    mps.eps_sum += res["eps"]
    mps.eps_log.append(res["eps"])
    return res


def apply_layer(mps, parity, gates, use_svd=False, **trunc):
    """Gates on all bonds of one parity; gates[m] acts on (m, m+1)."""
    for m in layer_bonds(mps.L, parity, mps.finite):
        if use_svd:
            update_bond_svd(mps, m, gates[m], trunc["chi_max"], trunc.get("svd_min", 1e-14))
        else:
            update_bond(mps, m, gates[m], **trunc)


def strang_gates(L, d, g, dt, finite=True):
    """(half-step gates, full-step gates) for every bond."""
    half = _clock.layer_gates(L, d, g, dt / 2, finite)
    full = _clock.layer_gates(L, d, g, dt, finite)
    return half, full


def tebd_step(mps, half, full, use_svd=False, **trunc):
    """One second-order Strang step: even(dt/2), odd(dt), even(dt/2)."""
    apply_layer(mps, 0, half, use_svd, **trunc)
    apply_layer(mps, 1, full, use_svd, **trunc)
    apply_layer(mps, 0, half, use_svd, **trunc)


def expectation_1site(mps, m, O):
    """<O_m> = tr[(Xi B^m)^dag O (Xi B^m)] (Fig. 1c)."""
    C = np.tensordot(mps.Xi[m], mps.B[m], axes=(1, 0))  # (chi, d, chi')
    return complex(np.einsum("aib,ij,ajb->", C.conj(), O, C))


def expectation_2site(mps, m, O2):
    """<O_{m,m+1}> with O2 a d^2 x d^2 matrix in kron order, from theta = Xi B^m B^n."""
    n = (m + 1) % mps.L
    th = np.tensordot(np.tensordot(mps.Xi[m], mps.B[m], axes=(1, 0)), mps.B[n], axes=(2, 0))
    chiL, d, _, chiR = th.shape
    O4 = O2.reshape(d, d, d, d)
    return complex(np.einsum("aijb,ijkl,aklb->", th.conj(), O4, th))


def norm2_site(mps, m):
    """||Xi[m] B[m]||_F^2, the state norm squared seen from site m."""
    C = np.tensordot(mps.Xi[m], mps.B[m], axes=(1, 0))
    return float(np.vdot(C, C).real)


def entropies(mps):
    """von Neumann entropy on every bond matrix."""
    return [_bond.entropy(x) for x in mps.Xi]


def right_isometry_error(b):
    """max |sum_{i beta} B B^* - 1| for one site tensor (Sec. II)."""
    chi = b.shape[0]
    M = b.reshape(chi, -1)
    return float(np.max(np.abs(M @ M.conj().T - np.eye(chi))))


def to_statevector(mps):
    """Contract a finite MPS into its d^L state vector (Eq. 1), site 0 most significant."""
    if not mps.finite:
        raise ValueError("finite chains only")
    v = np.tensordot(mps.Xi[0], mps.B[0], axes=(1, 0))  # (1, d, chi)
    for m in range(1, mps.L):
        v = np.tensordot(v, mps.B[m], axes=(v.ndim - 1, 0))
    return v.reshape(-1)
