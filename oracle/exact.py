"""Oracle (test infrastructure): state-vector references for small chains.

* ``trotter_statevector``: the same two-site gates as the TEBD driver, applied
  without truncation to the full d^L vector (exact Trotterised evolution).
* ``krylov_evolve``: exp(-i H t) psi with the sparse Hamiltonian of Eq. 2
  (scipy's expm_multiply as a library step).
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import clock as _clock
from . import mps as _mps


def product_vector(L, d, k=0):
    v = np.zeros(d ** L, np.complex128)
    idx = 0
    for _ in range(L):
        idx = idx * d + k
    v[idx] = 1.0
    return v


def apply_two_site(psi, L, d, m, U):
    """Apply U (d^2 x d^2, kron order) on sites (m, m+1) of a finite chain vector."""
    t = psi.reshape(d ** m, d * d, d ** (L - m - 2))
    t = np.einsum("ab,xby->xay", U, t)
    return t.reshape(-1)


def trotter_statevector(psi, L, d, g, dt, steps):
    """Strang steps even(dt/2), odd(dt), even(dt/2) on a finite open chain."""
    half, full = _mps.strang_gates(L, d, g, dt, finite=True)
    for _ in range(steps):
        for gates, parity in ((half, 0), (full, 1), (half, 0)):
            for m in _mps.layer_bonds(L, parity, True):
                psi = apply_two_site(psi, L, d, m, gates[m])
    return psi


def krylov_evolve(psi, L, d, g, t, finite=True):
    H = _clock.chain_hamiltonian(L, d, g, finite)
    return spla.expm_multiply(-1j * t * H, psi)


def local_expectation(psi, L, d, m, O):
    t = psi.reshape(d ** m, d, d ** (L - m - 1))
    return complex(np.einsum("xiy,ij,xjy->", t.conj(), O, t))


def energy(psi, L, d, g, finite=True):
    H = _clock.chain_hamiltonian(L, d, g, finite)
    return complex(np.vdot(psi, H @ psi))
