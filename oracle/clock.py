"""Oracle (test infrastructure): the d-state quantum clock model of Sec. IV.

H = -sum_n (Z_n Z_{n+1}^dag + h.c.) - g sum_n (X_n + h.c.)          (Eq. 2)
Z = diag(1, w, ..., w^{d-1}), w = exp(2 pi i / d); X = cyclic shift with ones on
the superdiagonal and X[d-1, 0] = 1                                   (Eq. 3)

Bond split (a reading; the paper only gives the sum): the bond term on (n, n+1) is
h_b = -(Z x Z^dag + Z^dag x Z) - g (w_l (X + X^dag) x 1 + w_r 1 x (X + X^dag)),
with w = 1/2 except w = 1 on the outer site of a finite chain's two end bonds, so
that sum_b h_b equals Eq. 2 exactly. Two-site matrices use kron order: combined
index i*d + j with the left site most significant.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def clock_operators(d):
    """Z and X of Eq. 3 as dense complex128 d x d matrices."""
    if d < 2:
        raise ValueError("d >= 2")
    omega = np.exp(2j * np.pi / d)
    Z = np.diag(omega ** np.arange(d)).astype(np.complex128)
    X = np.zeros((d, d), np.complex128)
    for k in range(d):
        X[k, (k + 1) % d] = 1.0
    return Z, X


def field_weights(L, finite=True):
    """(w_l, w_r) for every bond: how the on-site field is shared between bonds."""
    if not finite:
        return [(0.5, 0.5)] * L
    out = []
    for b in range(L - 1):
        wl = 1.0 if b == 0 else 0.5
        wr = 1.0 if b == L - 2 else 0.5
        out.append((wl, wr))
    return out


def bond_hamiltonian(d, g, wl=0.5, wr=0.5):
    """d^2 x d^2 bond term h_b (row = output (i,j), column = input (i',j'))."""
    Z, X = clock_operators(d)
    one = np.eye(d)
    Xs = X + X.conj().T
    zz = np.kron(Z, Z.conj().T)
    h = -(zz + zz.conj().T) - g * (wl * np.kron(Xs, one) + wr * np.kron(one, Xs))
    return h


def trotter_gate(h, tau):
    """U = exp(-i tau h); tau may be complex (imaginary time)."""
    return sla.expm(-1j * tau * h)


def chain_hamiltonian(L, d, g, finite=True):
    """Sparse d^L x d^L Hamiltonian of Eq. 2, built term by term from Z and X.

    finite=True: open chain with L-1 bonds; finite=False: periodic ring of L sites.
    Built independently of ``bond_hamiltonian`` (from the single-site operators),
    so that the bond split can be checked against it.
    """
    Z, X = clock_operators(d)
    Zs, Xs = sp.csr_matrix(Z), sp.csr_matrix(X)
    eye = sp.identity(d, format="csr", dtype=np.complex128)

    def site_op(ops):
        """Tensor product over all sites; ops maps site -> operator."""
        m = sp.identity(1, format="csr", dtype=np.complex128)
        for s in range(L):
            m = sp.kron(m, ops.get(s, eye), format="csr")
        return m

    H = sp.csr_matrix((d ** L, d ** L), dtype=np.complex128)
    nb = L - 1 if finite else L
    for n in range(nb):
        term = site_op({n: Zs, (n + 1) % L: Zs.conj().T.tocsr()})
        H = H - term - term.conj().T
    for n in range(L):
        term = site_op({n: Xs})
        H = H - g * (term + term.conj().T)
    return H.tocsr()


def layer_gates(L, d, g, tau, finite=True):
    """Gates for every bond of a chain: list of d^2 x d^2 unitaries exp(-i tau h_b)."""
    return [trotter_gate(bond_hamiltonian(d, g, wl, wr), tau)
            for (wl, wr) in field_weights(L, finite)]
