"""Pins for the oracle's bond update (Sec. II, Sec. III) against mathematics.

Each test fixes a property the paper or linear algebra guarantees, chosen so that
a dropped term, a wrong conjugation, a transposed operand or a swapped index in
``oracle.bond`` fails at least one of them.
"""
import numpy as np
import pytest

from oracle import bond, householder
from paper_2212_09782_b300 import workloads as W


def brute_gate(U, th):
    # theta~[a,i,j,b] = sum_{k,l} U[i*d+j, k*d+l] theta[a,k,l,b], written as loops
    chiL, d, _, chiR = th.shape
    out = np.zeros_like(th)
    for i in range(d):
        for j in range(d):
            for k in range(d):
                for l in range(d):
                    out[:, i, j, :] += U[i * d + j, k * d + l] * th[:, k, l, :]
    return out


def brute_theta(Xi, Bm, Bn):
    chiL, d, chiM = Bm.shape
    chiR = Bn.shape[2]
    th = np.zeros((chiL, d, d, chiR), complex)
    for a in range(chiL):
        for i in range(d):
            for j in range(d):
                for b in range(chiR):
                    s = 0
                    for be in range(chiL):
                        for ga in range(chiM):
                            s += Xi[a, be] * Bm[be, i, ga] * Bn[ga, j, b]
                    th[a, i, j, b] = s
    return th


def test_gate_and_theta_against_loops():
    r = W.rng(1)
    bd = W.random_bond(3, 2, 4, 3, seed=5)
    th = bond.apply_xi(bd["Xi"], bond.theta_prime(bd["Bm"], bd["Bn"]))
    assert np.allclose(th, brute_theta(bd["Xi"], bd["Bm"], bd["Bn"]), atol=1e-14)
    t0 = W.complex_gaussian(r, (3, 3, 3, 2))
    U = W.random_unitary(r, 9)
    assert np.allclose(bond.apply_gate(U, t0), brute_gate(U, t0), atol=1e-14)


@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (8, 8), (12, 5), (20, 7)])
def test_textbook_householder_matches_lapack(m, n):
    r = W.rng(100 + m * n)
    A = W.complex_gaussian(r, (m, n))
    Q1, R1 = householder.householder_qr(A)
    Q2, R2 = np.linalg.qr(A, mode="reduced")
    assert np.allclose(Q1 @ R1, A, atol=1e-13)
    assert np.allclose(Q1.conj().T @ Q1, np.eye(n), atol=1e-13)
    assert np.allclose(np.triu(R1), R1)
    # same sign convention as geqrf: R and Q agree element by element
    assert np.allclose(R1, R2, atol=1e-12)
    assert np.allclose(Q1, Q2, atol=1e-12)
    assert np.all(np.abs(np.imag(np.diag(R1))) < 1e-13)


def test_householder_rank_deficient_is_isometry():
    r = W.rng(7)
    A = W.complex_gaussian(r, (10, 2)) @ W.complex_gaussian(r, (2, 6))  # rank 2, 6 columns
    Q, R = householder.householder_qr(A)
    assert np.allclose(Q.conj().T @ Q, np.eye(6), atol=1e-13)
    assert np.allclose(Q @ R, A, atol=1e-13)


@pytest.mark.parametrize("xi", ["dense", "diag", "eye"])
@pytest.mark.parametrize("dims", [(2, 3, 4, 3), (4, 3, 5, 4), (6, 2, 7, 5)])
def test_identity_gate_reproduces_theta(xi, dims):
    # Sec. II: Y0 = B^n; with U = 1, theta = Xi B^m B^n lies in B^n's row space,
    # so X = Xi B^m, Q R = X, Y = R B^n and Q L Q^[n] = theta exactly.
    chiL, d, chiM, chiR = dims
    bd = W.random_bond(chiL, d, chiM, chiR, seed=sum(dims), xi=xi)
    U = np.eye(d * d, dtype=complex)
    out = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], U, chi_max=chiM, eta=chiM)
    T = out["theta_t"].reshape(chiL * d, d * chiR)
    assert out["eps"] < 1e-26
    assert np.allclose(out["Q"] @ out["L"] @ out["Qn"], T, atol=1e-14)
    # Hastings form: Xi B~^m B~^n reproduces theta~ (state unchanged, Sec. II (iii))
    Bm = out["Bm_new"].reshape(chiL * d, -1)
    Bn = out["Bn_new"].reshape(Bm.shape[1], -1)
    Xi_old = bd["Xi"]
    left = (Xi_old @ Bm.reshape(chiL, -1)).reshape(chiL * d, -1)
    assert np.allclose(left @ Bn, T, atol=1e-13)
    # new Xi = L / ||L|| with ||L|| = ||theta|| = ||Xi|| = 1
    assert abs(out["norm_L"] - 1.0) < 1e-13


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("scheme", ["plain", "cbe"])
def test_exact_when_eta_covers_rank(seed, scheme):
    # Sec. II last paragraph / Sec. III (i): slice guess with eta >= rank theta~ is exact
    r = W.rng(seed)
    chiL, d, chiR, rank = 4, 3, 5, 6
    T0 = (W.complex_gaussian(r, (chiL * d, rank)) @ W.complex_gaussian(r, (rank, d * chiR)))
    T0 = (T0 / np.linalg.norm(T0)).reshape(chiL, d, d, chiR)
    U = W.random_unitary(r, d * d)
    th = bond.apply_gate(U.conj().T, T0)  # so that theta~ = U theta has rank 6
    Bn = W.random_right_isometry(r, 3, d, chiR)
    out = bond.qr_update(None, None, Bn, U, scheme=scheme, chi_max=100, eta=8, theta=th,
                         dchi_min=0)
    T = out["theta_t"].reshape(chiL * d, d * chiR)
    assert np.allclose(T, T0.reshape(chiL * d, d * chiR), atol=1e-14)
    assert out["eps"] < 1e-26
    assert np.allclose(out["Q"] @ out["L"] @ out["Qn"], T, atol=1e-13)
    if scheme == "cbe":
        assert out["chi_new"] == rank  # values below 1e-14 are dropped


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("scheme", ["plain", "cbe"])
def test_isometries(seed, scheme):
    bd = W.random_bond(5, 3, 6, 4, seed=seed)
    out = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], scheme=scheme, chi_max=6,
                         dchi_min=3)
    Q, Qn = out["Q"], out["Qn"]
    assert np.allclose(Q.conj().T @ Q, np.eye(Q.shape[1]), atol=1e-13)       # A^dag A = 1
    assert np.allclose(Qn @ Qn.conj().T, np.eye(Qn.shape[0]), atol=1e-13)
    Bn = out["Bn_new"].reshape(out["Bn_new"].shape[0], -1)
    assert np.allclose(Bn @ Bn.conj().T, np.eye(Bn.shape[0]), atol=1e-13)    # right isometric
    assert abs(np.linalg.norm(out["Xi_new"]) - 1) < 1e-14
    # L lower triangular (LQ)
    assert np.allclose(np.tril(out["L"]), out["L"], atol=1e-14)


@pytest.mark.parametrize("seed", range(25))
def test_qr_error_never_below_svd_optimum(seed):
    # Eckart-Young: no rank-eta approximation beats the truncated SVD
    r = W.rng(1000 + seed)
    chiL, d, chiM, chiR = 3, 2, 3, 3
    bd = W.random_bond(chiL, d, chiM, chiR, seed=2000 + seed)
    U = W.random_unitary(r, d * d)
    out = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], U, chi_max=chiM, eta=chiM)
    T = out["theta_t"].reshape(chiL * d, d * chiR)
    s = np.linalg.svd(T, compute_uv=False)
    opt = np.sum(s[chiM:] ** 2) / np.sum(s ** 2)
    assert out["eps"] >= opt * (1 - 1e-12) - 1e-15


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("scheme", ["plain", "cbe"])
def test_error_projector_identity(seed, scheme):
    # M -> P1 M P2 with P1 = Q Q^dag, P2 = Qn^dag Qn is an orthogonal projector, so
    # ||theta - approx||^2 = ||theta||^2 - ||kept||^2 (derived from Sec. II (i)-(ii))
    bd = W.random_bond(4, 3, 5, 4, seed=50 + seed)
    out = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], scheme=scheme, chi_max=4,
                         dchi_min=3)
    if scheme == "plain":
        kept = out["norm_L"] ** 2
    else:
        kept = float(np.sum(out["S"][: out["chi_new"]] ** 2))
    assert abs(out["eps"] - (1 - kept / out["norm_theta"] ** 2)) < 1e-13


@pytest.mark.parametrize("seed", range(4))
def test_norm_kept_under_unitary_gate(seed):
    # no truncation (eta = d chi): ||L|| = ||theta~|| = ||Xi|| = 1
    bd = W.random_bond(3, 3, 4, 3, seed=80 + seed)
    out = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], chi_max=9, eta=9)
    assert abs(out["norm_theta"] - 1) < 1e-13
    assert abs(out["norm_L"] - 1) < 1e-13
    assert out["eps"] < 1e-26


@pytest.mark.parametrize("seed", range(4))
def test_cbe_schmidt_values_are_singular_values_of_L(seed):
    bd = W.random_bond(5, 3, 5, 5, seed=90 + seed)
    out = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], scheme="cbe", chi_max=50,
                         dchi_min=4)
    sv = np.linalg.svd(out["L"], compute_uv=False)
    S = out["S"]
    assert np.allclose(S[: len(sv)], sv, atol=1e-12 * sv[0])
    # V's rows are the conjugated right singular vectors: L^dag L V^dag = V^dag S^2
    V = out["V"]
    assert np.allclose(out["L"].conj().T @ out["L"] @ V.conj().T, V.conj().T * S ** 2,
                       atol=1e-12)
    # canonical form: Xi~ diagonal, positive, descending (Sec. III)
    x = np.diag(out["Xi_new"]).real
    assert np.all(np.diff(x) <= 0) and np.all(x > 0)
    assert np.allclose(out["Xi_new"], np.diag(np.diag(out["Xi_new"])))


def test_cbe_cut_eps_target():
    # s^2 = (16, 4, 1, 1/4, 1/16) / 21.3125: dropping the last value discards 0.00293 of the
    # weight, the last two 0.0147, the last three 0.0616
    S = np.array([4.0, 2.0, 1.0, 0.5, 0.25])
    assert bond.cbe_cut(S, chi_max=10) == 5
    assert bond.cbe_cut(S, chi_max=10, eps_target=0.01) == 4
    assert bond.cbe_cut(S, chi_max=10, eps_target=0.02) == 3
    assert bond.cbe_cut(S, chi_max=10, eps_target=0.1) == 2
    assert bond.cbe_cut(S, chi_max=2, eps_target=0.01) == 2      # chi_max still binds
    assert bond.cbe_cut(S, chi_max=10, eps_target=0.9) == 1      # at least one value kept
    # the rule: discarded weight <= eps_target, and one more value would exceed it
    rng = np.random.default_rng(3)
    for _ in range(20):
        T = np.sort(rng.exponential(size=30))[::-1]
        eps = float(rng.uniform(1e-4, 0.2))
        c = bond.cbe_cut(T, chi_max=100, svd_min=0.0, eps_target=eps)
        w = T ** 2 / np.sum(T ** 2)
        assert w[c:].sum() <= eps + 1e-15
        if c > 1:
            assert w[c - 1:].sum() > eps


def test_cbe_cut_rules():
    S = np.array([1.0, 0.5, 0.5 - 1e-12, 0.1, 1e-15, 0.0])
    assert bond.cbe_cut(S, chi_max=10) == 4          # 1e-15 / ||S|| < 1e-14 dropped
    assert bond.cbe_cut(S, chi_max=2) == 1           # would split the degenerate pair
    assert bond.cbe_cut(S, chi_max=3) == 3
    assert bond.cbe_cut(np.array([1.0]), chi_max=5) == 1


@pytest.mark.parametrize("seed", range(5))
def test_agrees_with_svd_tebd_at_small_dt(seed):
    # Sec. II: U = 1 + O(dt) makes Y0 = B^n optimal to zeroth order; one sweep is close
    # to the SVD result. Pin: Schmidt values agree to O(dt^2)-level in the canonical case.
    r = W.rng(300 + seed)
    bd = W.random_bond(4, 3, 6, 4, seed=400 + seed, xi="diag")
    U = W.near_identity_gate(r, 3, 1e-3)
    q = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], U, scheme="cbe", chi_max=6, dchi_min=0,
                       dchi_frac=0.0)
    s = bond.svd_update(bd["Xi"], bd["Bm"], bd["Bn"], U, chi_max=6)
    assert np.allclose(np.diag(q["Xi_new"]).real, np.diag(s["Xi_new"]).real, atol=1e-5)
    assert q["eps"] >= s["eps"] * (1 - 1e-9) - 1e-16


def test_eta_policy():
    assert bond.choose_eta("plain", 1, 1, 1, 5, 1024) == 5
    assert bond.choose_eta("plain", 1024, 1024, 1024, 5, 1024) == 1024
    assert bond.choose_eta("cbe", 1024, 1024, 1024, 5, 1024) == 1024 + 103
    assert bond.choose_eta("cbe", 10, 10, 10, 3, 1024) == 30
    assert bond.choose_eta("cbe", 400, 400, 400, 5, 1024, 100, 0.1) == 500


def _designed_theta(r, m, n, spec):
    """theta~ = Ua diag(spec) Vb^dag with random unitaries (a chosen singular spectrum)."""
    Ua = np.linalg.qr(W.complex_gaussian(r, (m, m)))[0][:, : len(spec)]
    Vb = np.linalg.qr(W.complex_gaussian(r, (n, n)))[0][:, : len(spec)]
    return (Ua * spec) @ Vb.conj().T


def test_sweeps_one_is_the_single_update():
    bd = W.random_bond(8, 3, 8, 8, seed=71, xi="dense")
    a = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], chi_max=8)
    b = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], chi_max=8, sweeps=1)
    assert np.array_equal(a["Xi_new"], b["Xi_new"]) and a["eps"] == b["eps"]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sweeps_never_increase_eps_and_reach_svd_optimum(seed):
    # Sec. II: each half sweep minimises ||theta~ - X Y|| exactly over one factor (X = theta~ Y^dag
    # for an isometric Y, then Y = Q^dag theta~), so eps cannot grow from sweep to sweep; the
    # iteration is a subspace iteration on theta~^dag theta~, so with a gap below eta it reaches
    # the Eckart-Young optimum (the SVD truncation error). A random gate (far from the identity)
    # on a random bond
    r = W.rng(300 + seed)
    chiL, d, chiM, chiR = 10, 3, 6, 10
    bd = W.random_bond(chiL, d, chiM, chiR, seed=400 + seed, xi="dense")
    U = W.random_unitary(r, d * d)
    eps = [bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], U, chi_max=chiM, sweeps=k)["eps"]
           for k in range(1, 41)]
    assert all(b <= a * (1 + 1e-12) + 1e-15 for a, b in zip(eps, eps[1:])), eps
    opt = bond.svd_update(bd["Xi"], bd["Bm"], bd["Bn"], U, chi_max=chiM)["eps"]
    assert eps[0] > opt * (1 + 1e-6)          # one sweep is not optimal for a generic gate
    assert abs(eps[-1] - opt) <= 1e-8 * opt   # forty sweeps are


def test_sweeps_converge_at_the_subspace_iteration_rate():
    # theta~ with singular values 1 (x eta) then r (x the rest): the right space after k sweeps
    # is Y0 (theta~^dag theta~)^k orthonormalised, so the angle to the dominant space shrinks
    # by r^2 per sweep and the excess error eps_k - eps_opt by r^4
    rr = 0.5
    r = W.rng(77)
    m, n, eta = 24, 30, 6
    spec = np.r_[np.ones(eta), rr * np.ones(8)]
    T = _designed_theta(r, m, n, spec).reshape(m // 3, 3, 3, n // 3)
    Y0 = np.linalg.qr(W.complex_gaussian(r, (n, eta)))[0].conj().T
    opt = float(np.sum(spec[eta:] ** 2) / np.sum(spec ** 2))
    ex = []
    for k in range(1, 9):
        out = bond.qr_update(None, None, None, np.eye(9), chi_max=eta, eta=eta, theta=T, Y0=Y0, sweeps=k)
        ex.append(out["eps"] - opt)
    ratios = [b / a for a, b in zip(ex[3:], ex[4:])]
    assert all(0.5 * rr ** 4 < q < 2.0 * rr ** 4 for q in ratios), (ex, ratios)


def test_sweeps_reach_the_dominant_singular_values():
    # converged, the kept Schmidt values are the eta largest singular values of theta~
    r = W.rng(78)
    m, n, eta = 24, 30, 5
    spec = np.r_[np.linspace(1.0, 0.6, eta), 0.3 * np.linspace(1.0, 0.1, 10)]
    T = _designed_theta(r, m, n, spec).reshape(m // 3, 3, 3, n // 3)
    Y0 = np.linalg.qr(W.complex_gaussian(r, (n, eta)))[0].conj().T
    out = bond.qr_update(None, None, None, np.eye(9), chi_max=eta, eta=eta, theta=T, Y0=Y0, sweeps=60)
    s = np.linalg.svd(out["Xi_new"], compute_uv=False) * out["norm_L"]
    assert np.allclose(s, spec[:eta], rtol=1e-10, atol=0)


def test_tie_rule_makes_the_kept_subspace_unique():
    # Schmidt values with an exactly degenerate pair straddling chi_max = 3. A cut inside the
    # pair keeps one vector of the degenerate plane, and which one depends on the path (here
    # on the initial guess Y0): the truncated state is then not a function of theta~. The
    # tie rule drops the whole pair, and the kept subspace no longer depends on Y0.
    r = W.rng(91)
    n = 12
    s = np.array([1.0, 0.7, 0.4, 0.4, 0.2, 0.1, 0.05, 0.02, 0.01, 5e-3, 2e-3, 1e-3])
    Us, Vs = W.random_unitary(r, n), W.random_unitary(r, n)
    T = (Us * s) @ Vs.conj().T
    th = T.reshape(6, 2, 2, 6)
    U = np.eye(4, dtype=np.complex128)
    Y0s = [T[:n], W.complex_gaussian(r, (n, n))]

    def proj(tie_tol, Y0):
        o = bond.qr_update(None, None, None, U, scheme="cbe", chi_max=3, eta=n, theta=th, Y0=Y0,
                           svd_min=0.0, tie_tol=tie_tol)
        B = o["Bn_new"].reshape(o["chi_new"], -1)
        return o["chi_new"], B.conj().T @ B

    (ca, Pa), (cb, Pb) = (proj(1e-10, Y0) for Y0 in Y0s)
    assert ca == cb == 2
    assert np.max(np.abs(Pa - Pb)) < 1e-12
    # the two kept vectors are the dominant right singular vectors of theta~
    Vt = Vs.conj().T[:2]
    assert np.max(np.abs(Pa - Vt.conj().T @ Vt)) < 1e-12
    # without the rule (tie_tol = 0 never fires on values equal only to rounding) the cut
    # falls inside the pair and the kept subspace depends on Y0
    (ca, Pa), (cb, Pb) = (proj(0.0, Y0) for Y0 in Y0s)
    assert ca == cb == 3
    assert np.max(np.abs(Pa - Pb)) > 1e-3
