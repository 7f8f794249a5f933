"""GPU parity of the blocked Householder QR (Sec. II steps (i)-(ii)) against LAPACK.

Same sign convention as geqrf (real diagonal of R, beta = -sign(Re alpha) norm), so R
is compared element by element; Q through Q R = A and Q^dag Q = 1."""
import numpy as np
import pytest

from paper_2212_09782_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64_fp32": 2e-5, "c64_3xtf32": 2e-5}


def _run(prec, A):
    import torch
    from paper_2212_09782_b300 import lib as L
    dt = torch.complex128 if prec == "c128" else torch.complex64
    Q, R = L.householder_qr(prec, torch.from_numpy(A).to(device="cuda", dtype=dt))
    L.stream_check()
    return Q.cpu().numpy().astype(np.complex128), R.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("prec", list(TOL))
@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (32, 32), (99, 33), (99, 32), (100, 65),
                                 (300, 130), (640, 256), (1200, 257), (400, 385), (1000, 640)])
def test_qr_matches_lapack(prec, m, n):
    # more than two 128-column blocks take the look-ahead paths (whole-factor T, the next
    # block's columns beside V); 400 x 385 ends on a one-column block with 16 rows below
    A = W.complex_gaussian(W.rng(m * 7 + n), (m, n))
    if prec != "c128":
        A = A.astype(np.complex64).astype(np.complex128)
    Q, R = _run(prec, A)
    assert np.isfinite(Q).all() and np.isfinite(R).all()
    tol = TOL[prec]
    assert np.linalg.norm(Q @ R - A) / np.linalg.norm(A) < tol
    assert np.abs(Q.conj().T @ Q - np.eye(n)).max() < tol * 5
    assert np.abs(np.tril(R, -1)).max() == 0
    assert np.abs(np.diag(R).imag).max() <= tol * np.abs(np.diag(R)).max()
    Rl = np.linalg.qr(A, mode="r")
    assert np.linalg.norm(R - Rl) / np.linalg.norm(Rl) < tol * 10


@pytest.mark.parametrize("prec", list(TOL))
@pytest.mark.parametrize("m,n", [(5152, 33), (6000, 40), (13000, 40), (5120, 160), (3000, 128), (330, 64)])
def test_qr_tall_panels(prec, m, n):
    # panels of up to 320 slab rows per CTA of a 16-CTA cluster hold the slab in registers
    # (complex64); taller ones keep every row in shared memory: both forms, one row past
    # a full register share and a ragged last panel; at 13000 rows the panel narrows to fit
    # shared memory, and the outer T takes its column-by-column form
    A = W.complex_gaussian(W.rng(m + n), (m, n))
    if prec != "c128":
        A = A.astype(np.complex64).astype(np.complex128)
    Q, R = _run(prec, A)
    tol = TOL[prec]
    assert np.linalg.norm(Q @ R - A) / np.linalg.norm(A) < tol
    assert np.abs(Q.conj().T @ Q - np.eye(n)).max() < tol * 5
    Rl = np.linalg.qr(A, mode="r")
    assert np.linalg.norm(R - Rl) / np.linalg.norm(Rl) < tol * 10


@pytest.mark.parametrize("prec", list(TOL))
def test_qr_rank_deficient_gives_isometry(prec):
    # Householder returns an exact isometry even for rank-deficient input (Sec. II
    # readings: never CholeskyQR), the case eta > rank theta~
    r = W.rng(3)
    A = W.complex_gaussian(r, (150, 7)) @ W.complex_gaussian(r, (7, 60))
    if prec != "c128":
        A = A.astype(np.complex64).astype(np.complex128)
    Q, R = _run(prec, A)
    tol = TOL[prec]
    assert np.abs(Q.conj().T @ Q - np.eye(60)).max() < tol * 5
    assert np.linalg.norm(Q @ R - A) / np.linalg.norm(A) < tol


@pytest.mark.parametrize("prec", list(TOL))
@pytest.mark.parametrize("m,n,rank", [(2000, 64, 10), (5120, 96, 40)])
def test_qr_tall_rank_deficient(prec, m, n, rank):
    # tall panels of a rank-deficient matrix: the complex64 panels run as a tall-skinny tree
    # (several leaves and a combine); the reflectors of the noise directions are arbitrary,
    # but Q must stay an exact isometry with Q R = A
    r = W.rng(m + rank)
    A = W.complex_gaussian(r, (m, rank)) @ W.complex_gaussian(r, (rank, n))
    if prec != "c128":
        A = A.astype(np.complex64).astype(np.complex128)
    Q, R = _run(prec, A)
    tol = TOL[prec]
    assert np.isfinite(Q).all() and np.isfinite(R).all()
    assert np.abs(Q.conj().T @ Q - np.eye(n)).max() < tol * 5
    assert np.linalg.norm(Q @ R - A) / np.linalg.norm(A) < tol
    assert np.abs(np.tril(R, -1)).max() == 0


@pytest.mark.parametrize("prec", list(TOL))
def test_qr_zero_and_tiny_columns(prec):
    # columns that are exactly zero or at the underflow edge (the rank-deficient blocks
    # of a product-state start) must give finite, unitary reflectors
    tiny = 1e-23 if prec != "c128" else 1e-160
    A = np.zeros((6, 4), np.complex128)
    A[0, 0] = 1.0
    A[2, 1] = tiny
    A[1, 2] = 0.5 + 0.5j
    A[3, 3] = tiny * 1j
    Q, R = _run(prec, A)
    assert np.isfinite(Q).all() and np.isfinite(R).all()
    assert np.abs(Q.conj().T @ Q - np.eye(4)).max() < TOL[prec] * 5
    assert np.abs(Q @ R - A).max() < TOL[prec]
