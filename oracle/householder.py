"""Oracle (test infrastructure): textbook complex Householder QR, column by column.

Used only on tiny matrices, to pin the LAPACK QR that the bond-update oracle
calls as a library step (Sec. II (i)-(ii) need a QR and an LQ). Pure Python
loops over columns; each reflector is H = I - tau v v^dag with v[0] = 1, the
convention of LAPACK's geqrf (so that R's diagonal can be compared directly).
"""
import numpy as np


def householder_qr(A):
    """Return (Q, R) with A = Q R, Q (m x n) with orthonormal columns, R (n x n) upper.

    Requires m >= n. Reflector for column k: alpha = A[k,k], x = A[k+1:, k],
    beta = -sign(Re alpha) * sqrt(|alpha|^2 + ||x||^2), tau = (beta - alpha) / beta,
    v = [1, x / (alpha - beta)]; H^dag = I - conj(tau) v v^dag maps the column to beta e_1.
    """
    A = np.array(A, dtype=np.complex128)
    m, n = A.shape
    if m < n:
        raise ValueError("m >= n required")
    R = A.copy()
    vs, taus = [], []
    for k in range(n):
        alpha = R[k, k]
        x = R[k + 1:, k]
        xnorm = np.sqrt(np.sum(np.abs(x) ** 2))
        if xnorm == 0.0 and alpha.imag == 0.0:
            tau = 0.0
            v = np.zeros(m - k, np.complex128)
            v[0] = 1.0
        else:
            beta = -np.copysign(np.sqrt(abs(alpha) ** 2 + xnorm ** 2), alpha.real)
            tau = (beta - alpha) / beta
            v = np.concatenate([[1.0 + 0j], x / (alpha - beta)])
        # apply H^dag = I - conj(tau) v v^dag to the trailing columns
        sub = R[k:, k:]
        w = v.conj() @ sub
        sub -= np.conj(tau) * np.outer(v, w)
        R[k + 1:, k] = 0.0
        vs.append(v)
        taus.append(tau)
    # form Q = H_0 H_1 ... H_{n-1} [I; 0] by backward accumulation
    Q = np.zeros((m, n), np.complex128)
    Q[:n, :n] = np.eye(n)
    for k in reversed(range(n)):
        v, tau = vs[k], taus[k]
        sub = Q[k:, :]
        w = v.conj() @ sub
        sub -= tau * np.outer(v, w)
    return Q, np.triu(R[:n, :])
