"""Oracle (test infrastructure): one two-site bond update, step by step.

Follows Sec. II (Fig. 2b, steps (i)-(iii)) for the plain QR truncation and
Sec. III (Fig. 3, steps (i)-(v)) for QR with controlled bond expansion (CBE);
``svd_update`` is the SVD-truncated TEBD update that the paper compares against
(Sec. IV, scheme (i)). complex128 throughout; LAPACK QR / eigh / SVD serve as
single steps.

Shapes (row-major, left index most significant):
  Xi : (chi_L, chi_L)          bond matrix on the bond left of site m
  Bm : (chi_L, d, chi_M)       right isometry of site m
  Bn : (chi_M, d, chi_R)       right isometry of site n = m + 1
  U  : (d*d, d*d)              row = output (i, j), column = input (i', j')
  theta as a matrix: rows alpha*d + i, columns j*chi_R + delta.

Readings of points the paper leaves open (each is listed in the design notes):
  * Y0: B^n when eta == chi_M (plain), otherwise the first eta rows of theta~ in
    the row order alpha*d + i (the "slice of the left leg pair", Secs. II-III).
  * eta: plain min(chi_max, d chi_L, d chi_R); CBE min(chi_M + dchi, d chi_L, d chi_R),
    dchi = max(dchi_min, ceil(dchi_frac * chi_M)).
  * CBE cut: keep S_k / ||S|| >= svd_min, at most chi_max, and never split a
    multiplet: while S[c-1] - S[c] <= tie_tol * S[0], lower c.
  * Xi~ is normalised to unit Frobenius norm after every update (Sec. II, ||Xi|| = 1).
  * Truncation error: eps = ||theta~ - approx||_F^2 / ||theta~||_F^2 with the
    approximation built explicitly (Sec. IV: the explicit distance).
"""
import math

import numpy as np


def theta_prime(Bm, Bn):
    """theta'^{i'j'}_{alpha delta} = sum_gamma B^m_{alpha i' gamma} B^n_{gamma j' delta}  (Sec. II (i), without Xi)."""
    return np.tensordot(Bm, Bn, axes=(2, 0))  # (chi_L, d, d, chi_R)


def apply_gate(U, th):
    """theta~'^{ij} = sum_{i'j'} U_{(ij),(i'j')} theta'^{i'j'}  (Sec. II (i))."""
    chiL, d, _, chiR = th.shape
    U4 = U.reshape(d, d, d, d)
    return np.einsum("ijkl,aklb->aijb", U4, th)


def apply_xi(Xi, th):
    """theta~ = Xi theta~' on the left bond index  (Sec. II (i))."""
    return np.tensordot(Xi, th, axes=(1, 0))


def choose_eta(scheme, chiL, chiM, chiR, d, chi_max, dchi_min=100, dchi_frac=0.1):
    """Expansion dimension eta (Sec. II last paragraph; Sec. III)."""
    cap = min(d * chiL, d * chiR)
    if scheme == "plain":
        return min(chi_max, cap)
    dchi = max(dchi_min, int(math.ceil(dchi_frac * chiM)))
    return min(chiM + dchi, cap)


def cbe_cut(S, chi_max, svd_min=1e-14, tie_tol=1e-10, eps_target=0.0):
    """Number of Schmidt values kept after CBE (Sec. III (v), Fig. 4 caption).

    eps_target > 0 further keeps only the fewest values whose discarded weight
    sum_{k >= c} s_k^2 (s = S / ||S||) is at most eps_target; the tie rule comes last."""
    nrm = np.sqrt(np.sum(S ** 2))
    if nrm == 0.0:
        return 1
    s = S / nrm
    c = int(np.sum(s >= svd_min))
    c = max(1, min(c, chi_max))
    if eps_target > 0:
        ce = len(s)
        tail = 0.0
        while ce > 1 and tail + s[ce - 1] ** 2 <= eps_target:
            tail += s[ce - 1] ** 2
            ce -= 1
        c = min(c, ce)
    while c < len(s) and c > 1 and s[c - 1] - s[c] <= tie_tol * s[0]:
        c -= 1
    return c


def qr_update(Xi, Bm, Bn, U, *, scheme="plain", chi_max, eta=None, dchi_min=100,
              dchi_frac=0.1, svd_min=1e-14, tie_tol=1e-10, eps_target=0.0, theta=None, Y0=None,
              sweeps=1):
    """One QR-TEBD bond update.

    theta, if given, is theta' = B^m B^n of shape (chi_L, d, d, chi_R) (then Bm is
    unused). Returns a dict with the new tensors Bm_new (chi_L, d, chi~),
    Xi_new (chi~, chi~), Bn_new (chi~, d, chi_R), the truncation error eps and
    the intermediates Q, L, Qn (and S, V for CBE).

    sweeps > 1 iterates steps (i)-(ii) as the alternating least-squares solver of Sec. II
    (comments after the algorithm): each further sweep keeps the isometry Y = Q^[n] of the
    previous one, forms the optimal X = theta~ Y^dag, gauges it with a QR, updates
    Y = Q^dag theta~ and takes its LQ again. The paper uses one sweep for gates close to
    the identity; a generic theta~ (e.g. a circuit gate, Sec. V) needs more.
    """
    if theta is None:
        theta = theta_prime(Bm, Bn)
    chiL, d, _, chiR = theta.shape
    chiM = Bn.shape[0] if Bn is not None else None
    if Xi is None:
        Xi = np.eye(chiL, dtype=np.complex128)

    # (i) gate and Xi: theta~' = U theta', theta~ = Xi theta~'
    tht_p = apply_gate(U, theta)
    tht = apply_xi(Xi, tht_p)
    Tp = tht_p.reshape(chiL * d, d * chiR)
    T = tht.reshape(chiL * d, d * chiR)

    if eta is None:
        eta = choose_eta(scheme, chiL, chiM, chiR, d, chi_max, dchi_min, dchi_frac)
    if eta > min(d * chiL, d * chiR):
        raise ValueError("eta exceeds d*chi")

    # initial guess Y0 (Sec. II: Y0 = B^n; Secs. II-III: slice of theta~)
    if Y0 is None:
        if scheme == "plain" and chiM == eta:
            Y0 = Bn.reshape(chiM, d * chiR)
        else:
            Y0 = T[:eta, :]

    # (i) X = theta~ Y0^dag, QR(X) -> Q^[m]
    X = T @ Y0.conj().T
    Q, _R = np.linalg.qr(X, mode="reduced")

    # (ii) Y = Q^dag theta~, LQ(Y) = QR(Y^dag)^dag -> L, Q^[n]
    Y = Q.conj().T @ T
    Qh, Rh = np.linalg.qr(Y.conj().T, mode="reduced")
    L = Rh.conj().T
    Qn = Qh.conj().T

    # further sweeps of the alternating least-squares solver (Sec. II comments): Y0 = Q^[n]
    for _ in range(int(sweeps) - 1):
        X = T @ Qn.conj().T
        Q, _R = np.linalg.qr(X, mode="reduced")
        Y = Q.conj().T @ T
        Qh, Rh = np.linalg.qr(Y.conj().T, mode="reduced")
        L = Rh.conj().T
        Qn = Qh.conj().T

    out = {"Q": Q, "L": L, "Qn": Qn, "eta": eta, "X": X, "Y": Y}
    nrm2_theta = float(np.vdot(T, T).real)

    if scheme == "plain":
        # (iii) Xi~ = L, B~^n = Q^[n]
        Xi_new = L
        Bn_new = Qn
        approx = Q @ L @ Qn
    elif scheme == "cbe":
        # (iv) L^dag L = V^dag S^2 V, descending
        w, W = np.linalg.eigh(L.conj().T @ L)
        w = w[::-1]
        W = W[:, ::-1]
        S = np.sqrt(np.maximum(w, 0.0))
        V = W.conj().T
        c = cbe_cut(S, chi_max, svd_min, tie_tol, eps_target)
        # (v) B~^n = P V Q^[n], Xi~ = P S P
        Bn_new = V[:c] @ Qn
        Xi_new = np.diag(S[:c]).astype(np.complex128)
        P = np.zeros(len(S))
        P[:c] = 1.0
        approx = Q @ L @ (V.conj().T @ (P[:, None] * V)) @ Qn
        out.update(S=S, V=V, chi_new=c)
    else:
        raise ValueError(scheme)

    # (iii) Hastings form: B~^m = theta~' B~^{n dag}
    Bm_new = Tp @ Bn_new.conj().T

    diff = T - approx
    eps = float(np.vdot(diff, diff).real) / nrm2_theta if nrm2_theta > 0 else 0.0
    xnorm = np.linalg.norm(Xi_new)
    Xi_new = Xi_new / xnorm

    chi_new = Xi_new.shape[0]
    out.update(
        Bm_new=Bm_new.reshape(chiL, d, chi_new),
        Xi_new=Xi_new,
        Bn_new=Bn_new.reshape(chi_new, d, chiR),
        eps=eps,
        norm_L=float(xnorm),
        norm_theta=math.sqrt(nrm2_theta),
        theta_t=tht,
    )
    return out


def svd_update(Xi, Bm, Bn, U, *, chi_max, svd_min=1e-14, theta=None):
    """SVD-truncated TEBD update (Sec. IV scheme (i)) with the same Hastings form."""
    if theta is None:
        theta = theta_prime(Bm, Bn)
    chiL, d, _, chiR = theta.shape
    if Xi is None:
        Xi = np.eye(chiL, dtype=np.complex128)
    tht_p = apply_gate(U, theta)
    tht = apply_xi(Xi, tht_p)
    Tp = tht_p.reshape(chiL * d, d * chiR)
    T = tht.reshape(chiL * d, d * chiR)
    Us, S, Vh = np.linalg.svd(T, full_matrices=False)
    nrm = np.sqrt(np.sum(S ** 2))
    c = int(np.sum(S / nrm >= svd_min))
    c = max(1, min(c, chi_max))
    Bn_new = Vh[:c]
    Xi_new = np.diag(S[:c] / np.sqrt(np.sum(S[:c] ** 2))).astype(np.complex128)
    Bm_new = Tp @ Bn_new.conj().T
    eps = float(np.sum(S[c:] ** 2) / np.sum(S ** 2))
    return {
        "Bm_new": Bm_new.reshape(chiL, d, c),
        "Xi_new": Xi_new,
        "Bn_new": Bn_new.reshape(c, d, chiR),
        "eps": eps,
        "S": S,
    }


def schmidt_values(Xi):
    """Schmidt values on a bond: singular values of Xi (Sec. II)."""
    return np.linalg.svd(Xi, compute_uv=False)


def entropy(Xi):
    """von Neumann entropy -sum p ln p, p = s^2 / sum s^2, natural log (Fig. 4)."""
    s = schmidt_values(Xi)
    p = s ** 2 / np.sum(s ** 2)
    p = p[p > 1e-300]
    return float(-np.sum(p * np.log(p)))
