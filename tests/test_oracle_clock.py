"""Pins for the oracle's clock model (Sec. IV, Eqs. 2-3) and Trotter gates."""
import numpy as np
import pytest

from oracle import clock


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_clock_algebra(d):
    # Z^d = X^d = 1, X Z = w Z X, both unitary: the defining relations of Eq. 3.
    Z, X = clock.clock_operators(d)
    w = np.exp(2j * np.pi / d)
    I = np.eye(d)
    assert np.allclose(np.linalg.matrix_power(Z, d), I, atol=1e-13)
    assert np.allclose(np.linalg.matrix_power(X, d), I, atol=1e-13)
    assert np.allclose(X @ Z, w * Z @ X, atol=1e-13)
    assert np.allclose(X @ X.conj().T, I)
    # Eq. 3 as printed: first row (0 1 0 ...), last row (1 0 ... 0)
    assert X[0, 1] == 1 and X[d - 1, 0] == 1 and np.trace(X) == 0


def test_d2_is_transverse_field_ising():
    # d = 2: Z = sigma_z, X = sigma_x, H = -2 sum sz sz - 2 g sum sx (textbook TFIM)
    L, g = 4, 0.7
    sz = np.diag([1.0, -1.0]).astype(complex)
    sx = np.array([[0, 1], [1, 0]], complex)

    def op(o, s):
        m = np.eye(1)
        for k in range(L):
            m = np.kron(m, o if k == s else np.eye(2))
        return m

    H = sum(-2 * op(sz, n) @ op(sz, n + 1) for n in range(L - 1))
    H = H + sum(-2 * g * op(sx, n) for n in range(L))
    assert np.allclose(clock.chain_hamiltonian(L, 2, g).toarray(), H, atol=1e-13)


@pytest.mark.parametrize("d,L", [(3, 4), (3, 5), (4, 3), (5, 3)])
@pytest.mark.parametrize("finite", [True, False])
def test_bond_split_sums_to_hamiltonian(d, L, finite):
    g = 1.3
    H = clock.chain_hamiltonian(L, d, g, finite).toarray()
    S = np.zeros_like(H)
    ws = clock.field_weights(L, finite)
    for b, (wl, wr) in enumerate(ws):
        h = clock.bond_hamiltonian(d, g, wl, wr)
        n = b
        if finite or n < L - 1:
            emb = np.kron(np.kron(np.eye(d ** n), h), np.eye(d ** (L - n - 2)))
        else:  # wrap-around bond (L-1, 0): permute h onto sites L-1 and 0
            h4 = h.reshape(d, d, d, d)
            emb = np.einsum("ijkl,xy->jxilyk", h4, np.eye(d ** (L - 2))).reshape(d ** L, d ** L)
        S += emb
    assert np.allclose(S, H, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3, 5])
def test_gates_unitary_and_group_law(d):
    h = clock.bond_hamiltonian(d, 1.1, 0.5, 1.0)
    assert np.allclose(h, h.conj().T)
    U1 = clock.trotter_gate(h, 0.03)
    U2 = clock.trotter_gate(h, 0.05)
    U12 = clock.trotter_gate(h, 0.08)
    assert np.allclose(U1 @ U1.conj().T, np.eye(d * d), atol=1e-13)
    assert np.allclose(U1 @ U2, U12, atol=1e-13)
    assert np.allclose(clock.trotter_gate(h, 0.0), np.eye(d * d))
    # first order: U = 1 - i tau h + O(tau^2)
    tau = 1e-6
    assert np.allclose(clock.trotter_gate(h, tau), np.eye(d * d) - 1j * tau * h, atol=1e-10)


@pytest.mark.parametrize("d", [3, 5])
def test_product_state_energy(d):
    # |0...0>: <Z Z^dag + h.c.> = 2 per bond, <X + X^dag> = 0  ->  E = -2 (L-1)
    L = 4
    H = clock.chain_hamiltonian(L, d, 2.0, True)
    v = np.zeros(d ** L, complex)
    v[0] = 1
    assert abs(np.vdot(v, H @ v) - (-2 * (L - 1))) < 1e-13
