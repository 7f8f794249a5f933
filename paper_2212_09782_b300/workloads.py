"""Seeded synthetic inputs shared by the CUDA path, the tests and the bench.

This module draws random numbers and shapes them; it does none of the bond
update's arithmetic. Every generator takes an explicit seed and uses NumPy's
PCG64, so the oracle and the CUDA path see bit-identical inputs.

Workload shapes follow the paper's benchmark (Sec. IV, Fig. 5): theta of shape
(chi, d, d, chi) with i.i.d. complex Gaussian entries, a Haar-like gate (the Q
factor of a complex Gaussian d^2 x d^2 matrix) and a random right isometry for
B^n (the conjugate transpose of the Q factor of a (d chi) x chi Gaussian).
"""
import numpy as np

BASE_SEED = 2212_09782


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def complex_gaussian(r, shape):
    """i.i.d. complex Gaussian, re and im ~ N(0, 1/2)."""
    return (r.standard_normal(shape) + 1j * r.standard_normal(shape)) / np.sqrt(2.0)


def random_unitary(r, n):
    """Q factor of an n x n complex Gaussian matrix (a random unitary)."""
    q, _ = np.linalg.qr(complex_gaussian(r, (n, n)))
    return q


def random_right_isometry(r, chi_l, d, chi_r):
    """B of shape (chi_l, d, chi_r) with B B^dag = 1 over (d, chi_r); needs chi_l <= d chi_r."""
    q, _ = np.linalg.qr(complex_gaussian(r, (d * chi_r, chi_l)))
    # a transpose is a strided view: copy to the row-major layout the device code reads
    return np.ascontiguousarray(q.conj().T.reshape(chi_l, d, chi_r))


def bond_microbench(chi, d, seed=BASE_SEED + 2, dtype=np.complex64):
    """theta (chi,d,d,chi) with ||theta||_F = 1, gate U (d^2 x d^2), B^n (chi,d,chi).

    Returns a dict of host arrays in ``dtype`` (theta, Bn) and complex128 (U).
    """
    r = rng(seed)
    th = complex_gaussian(r, (chi, d, d, chi))
    th /= np.linalg.norm(th)
    U = random_unitary(r, d * d)
    Bn = random_right_isometry(r, chi, d, chi)
    return {"theta": np.ascontiguousarray(th, dtype=dtype), "U": np.ascontiguousarray(U),
            "Bn": np.ascontiguousarray(Bn, dtype=dtype)}


def random_bond(chiL, d, chiM, chiR, seed, xi="dense"):
    """A random two-site block: Xi (chiL x chiL, ||Xi|| = 1), right isometries Bm, Bn, unitary U.

    xi = "dense" (a general complex matrix), "diag" (positive descending
    diagonal) or "eye" (identity scaled to unit norm).
    """
    r = rng(seed)
    if xi == "dense":
        Xi = complex_gaussian(r, (chiL, chiL))
    elif xi == "diag":
        Xi = np.diag(np.sort(r.random(chiL))[::-1] + 0.1).astype(np.complex128)
    else:
        Xi = np.eye(chiL, dtype=np.complex128)
    Xi /= np.linalg.norm(Xi)
    Bm = random_right_isometry(r, chiL, d, chiM)
    Bn = random_right_isometry(r, chiM, d, chiR)
    U = random_unitary(r, d * d)
    return {"Xi": Xi, "Bm": Bm, "Bn": Bn, "U": U}


def near_identity_gate(r, d, scale):
    """exp(-i scale H) for a random Hermitian H, via the eigenbasis of H (U = 1 + O(scale))."""
    A = complex_gaussian(r, (d * d, d * d))
    H = (A + A.conj().T) / 2
    w, V = np.linalg.eigh(H)
    return (V * np.exp(-1j * scale * w)) @ V.conj().T


def random_right_canonical_mps(L, d, chi_max, seed):
    """Random finite MPS with bond dimensions chi_b = min(d^b, d^(L-b), chi_max):
    right-isometric site tensors and diagonal, positive, descending, unit-norm Xi."""
    r = rng(seed)
    dims = [min(d ** min(b, L - b), chi_max) if min(b, L - b) < 64 else chi_max for b in range(L + 1)]
    B = [random_right_isometry(r, dims[m], d, dims[m + 1]) for m in range(L)]
    Xi = []
    for b in range(L + 1):
        x = np.sort(r.random(dims[b]))[::-1] + 1e-3
        Xi.append(x / np.linalg.norm(x))
    return dims, B, Xi


# ------------------------------------------------------------------ Z_d charge sectors
def random_charges(r, n, d, sort=True):
    """n bond charges drawn uniformly from 0..d-1 (sorted: each sector a contiguous run)."""
    c = r.integers(0, d, n)
    return np.sort(c) if sort else c


def charge_rule_theta(charge_l, charge_r, d):
    """Boolean (chi_l, d, d, chi_r) pattern c_l(alpha) + i + j = c_r(delta) (mod d) of a
    charge-conserving two-site block."""
    cl, cr = np.asarray(charge_l), np.asarray(charge_r)
    s = (cl[:, None, None, None] + np.arange(d)[None, :, None, None]
         + np.arange(d)[None, None, :, None]) % d
    return s == cr[None, None, None, :]


def symmetric_theta(r, charge_l, charge_r, d):
    """Complex Gaussian theta' on the charge-conserving pattern, zero elsewhere, unit norm."""
    m = charge_rule_theta(charge_l, charge_r, d)
    th = complex_gaussian(r, m.shape) * m
    return th / np.linalg.norm(th)


def charge_conserving_unitary(r, d, scale=None):
    """A d^2 x d^2 unitary that keeps i + j (mod d): one random unitary per pair-charge block
    (Haar-like), or exp(-i scale H) of a random block-diagonal Hermitian H when scale is set."""
    t = np.add.outer(np.arange(d), np.arange(d)).reshape(-1) % d
    U = np.zeros((d * d, d * d), np.complex128)
    for q in range(d):
        idx = np.nonzero(t == q)[0]
        n = len(idx)
        if scale is None:
            blk = random_unitary(r, n)
        else:
            A = complex_gaussian(r, (n, n))
            w, V = np.linalg.eigh((A + A.conj().T) / 2)
            blk = (V * np.exp(-1j * scale * w)) @ V.conj().T
        U[np.ix_(idx, idx)] = blk
    return U
