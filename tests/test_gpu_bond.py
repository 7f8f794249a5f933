"""GPU parity: the CUDA bond update against the oracle on the same seeded inputs.

Compared quantities are gauge invariant (Sec. II: the isometric form leaves a
unitary freedom on the new bond): the Schmidt values of Xi~, the projector
B~^n^dag B~^n, the block B~^m B~^n, (Xi~ B~^n)^dag (Xi~ B~^n), and eps.
"""
import numpy as np
import pytest

from oracle import bond
from paper_2212_09782_b300 import workloads as W
from tests.gpu_helpers import TOL, compare, rounded, run_gpu, subspace_tol

pytestmark = pytest.mark.gpu

PRECS = ["c128", "c64_fp32", "c64_3xtf32", "c64_tf32"]


def _case(dims, seed, xi, prec):
    chiL, d, chiM, chiR = dims
    bd = W.random_bond(chiL, d, chiM, chiR, seed=seed, xi=xi)
    return {k: rounded(v, prec) if k != "U" else v for k, v in bd.items()}


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims,xi", [
    ((4, 3, 4, 4), "dense"),
    ((16, 5, 16, 16), "dense"),
    ((33, 3, 33, 33), "diag"),      # ragged: dchi = 99
    ((48, 5, 48, 48), "eye"),       # two QR panels, cluster of 2
    ((100, 3, 100, 100), "dense"),
    ((130, 4, 130, 130), "diag"),   # dchi = 520: several tensor-core tiles, ragged tail
])
def test_plain_truncating(prec, dims, xi):
    bd = _case(dims, seed=sum(dims) * 7 + len(xi), xi=xi, prec=prec)
    chiM = dims[2]
    tr_o = dict(scheme="plain", chi_max=chiM)
    orc = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], **tr_o)
    from paper_2212_09782_b300 import lib as L
    t = L.trunc_default(L.PLAIN, chiM)
    xk = {"dense": 1, "diag": 2, "eye": 1}[xi]
    gpu = run_gpu(prec, bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], t, xi_kind=xk)
    assert gpu["eta"] == orc["eta"] == chiM
    compare(gpu, orc, TOL[prec])


@pytest.mark.parametrize("prec", ["c128", "c64_3xtf32"])
def test_identity_xi_and_theta_given(prec):
    # the C2 form: theta' supplied, Xi = 1
    r = W.rng(11)
    chi, d = 64, 5
    th = W.complex_gaussian(r, (chi, d, d, chi))
    th = rounded(th / np.linalg.norm(th), prec)
    U = W.random_unitary(r, d * d)
    Bn = rounded(W.random_right_isometry(r, chi, d, chi), prec)
    orc = bond.qr_update(None, None, Bn, U, chi_max=chi, theta=th)
    from paper_2212_09782_b300 import lib as L
    gpu = run_gpu(prec, None, None, Bn, U, L.trunc_default(L.PLAIN, chi), theta=th)
    compare(gpu, orc, TOL[prec])


@pytest.mark.parametrize("prec", ["c128", "c64_3xtf32"])
@pytest.mark.parametrize("dims", [(8, 3, 5, 8), (1, 2, 1, 1), (2, 4, 3, 5)])
def test_plain_slice_guess(prec, dims):
    # eta != chi_m: Y0 is the first eta rows of theta~ (Sec. II last paragraph)
    chiL, d, chiM, chiR = dims
    bd = _case(dims, seed=77 + sum(dims), xi="dense", prec=prec)
    chi_max = 16
    orc = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], chi_max=chi_max)
    from paper_2212_09782_b300 import lib as L
    gpu = run_gpu(prec, bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], L.trunc_default(L.PLAIN, chi_max))
    assert gpu["eta"] == orc["eta"]
    keys = ("s", "BB", "G")
    rank = np.linalg.matrix_rank(orc["theta_t"].reshape(chiL * d, -1))
    if rank >= orc["eta"]:
        keys = keys + ("P",)
    compare(gpu, orc, TOL[prec], keys=keys)


@pytest.mark.parametrize("prec", ["c128", "c64_3xtf32", "c64_fp32"])
@pytest.mark.parametrize("dims", [(6, 3, 6, 6), (20, 4, 24, 20), (40, 3, 37, 45)])
def test_cbe(prec, dims):
    chiL, d, chiM, chiR = dims
    bd = _case(dims, seed=500 + sum(dims), xi="diag", prec=prec)
    chi_max = max(chiM - 2, 1)
    kw = dict(dchi_min=4, dchi_frac=0.1)
    orc = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], scheme="cbe", chi_max=chi_max, **kw)
    from paper_2212_09782_b300 import lib as L
    t = L.trunc_default(L.CBE, chi_max, dchi_min=4, dchi_frac=0.1)
    gpu = run_gpu(prec, bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], t, xi_kind=2)
    assert gpu["eta"] == orc["eta"]
    assert gpu["chi_new"] == orc["chi_new"]
    S = orc["S"]
    k = S >= 1e-6 * S[0]
    assert np.allclose(gpu["S"][: len(S)][k], S[k], rtol=TOL[prec], atol=0)
    # Xi~ diagonal, positive, descending (canonical form)
    x = gpu["Xi_new"]
    assert np.abs(x - np.diag(np.diag(x))).max() < 1e-6
    compare(gpu, orc, TOL[prec], sub_tol=subspace_tol(TOL[prec], prec, S, orc["chi_new"]))


@pytest.mark.parametrize("prec", ["c128", "c64_3xtf32", "c64_fp32"])
@pytest.mark.parametrize("dims", [(120, 4, 128, 120), (250, 3, 251, 240)])
def test_cbe_many_jacobi_rounds(prec, dims):
    # eta = 228 and 351 (odd: one idle partner per round): hundreds of rounds per sweep of
    # the complex64 one-sided Jacobi and of the complex128 two-sided one
    chiL, d, chiM, chiR = dims
    bd = _case(dims, seed=900 + sum(dims), xi="diag", prec=prec)
    chi_max = chiM - 2
    orc = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], scheme="cbe", chi_max=chi_max)
    from paper_2212_09782_b300 import lib as L
    gpu = run_gpu(prec, bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], L.trunc_default(L.CBE, chi_max), xi_kind=2)
    assert gpu["eta"] == orc["eta"] == min(chiM + 100, d * chiL, d * chiR)
    assert gpu["chi_new"] == orc["chi_new"] == chi_max
    S = orc["S"]
    k = S >= 1e-4 * S[0]
    assert np.allclose(gpu["S"][: len(S)][k], S[k], rtol=TOL[prec], atol=0)
    # the cut falls inside a dense spectrum (gap ~1.8e-3 S_1): the kept space is resolved to
    # PERTURB / gap (measured 1.6e-5 for the projector in complex64 3xTF32, 9e-6 on CUDA cores)
    compare(gpu, orc, TOL[prec], sub_tol=subspace_tol(TOL[prec], prec, S, orc["chi_new"]))


@pytest.mark.parametrize("prec", ["c128", "c64_3xtf32"])
def test_cbe_eps_target(prec):
    # the cut at a target truncation error: the fewest Schmidt values whose discarded
    # weight is at most eps_target; the target is placed mid-way between two tail sums
    dims = (20, 4, 24, 20)
    bd = _case(dims, seed=777, xi="diag", prec=prec)
    kw = dict(dchi_min=4, dchi_frac=0.1)
    base = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], scheme="cbe", chi_max=60, **kw)
    S = base["S"]
    w = S ** 2 / np.sum(S ** 2)
    tails = np.cumsum(w[::-1])[::-1]          # tails[c] = weight discarded when keeping c
    c_want = max(2, len(S) // 3)
    eps_target = float(np.sqrt(tails[c_want] * tails[c_want - 1]))
    orc = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], scheme="cbe", chi_max=60,
                         eps_target=eps_target, **kw)
    assert orc["chi_new"] == c_want
    from paper_2212_09782_b300 import lib as L
    t = L.trunc_default(L.CBE, 60, dchi_min=4, dchi_frac=0.1, eps_target=eps_target)
    gpu = run_gpu(prec, bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], t, xi_kind=2)
    assert gpu["chi_new"] == orc["chi_new"] == c_want
    k = S >= 1e-6 * S[0]
    assert np.allclose(gpu["S"][: len(S)][k], S[k], rtol=TOL[prec], atol=0)
    compare(gpu, orc, TOL[prec], sub_tol=subspace_tol(TOL[prec], prec, S, orc["chi_new"]))


@pytest.mark.parametrize("prec", ["c128", "c64_3xtf32"])
def test_exact_when_eta_covers_rank(prec):
    # Sec. II / III: eta >= rank theta~ reproduces theta~: eps ~ 0, Xi B~^m B~^n = theta~
    r = W.rng(5)
    chiL, d, chiR, rank = 10, 3, 12, 6
    T0 = W.complex_gaussian(r, (chiL * d, rank)) @ W.complex_gaussian(r, (rank, d * chiR))
    T0 = (T0 / np.linalg.norm(T0)).reshape(chiL, d, d, chiR)
    U = W.random_unitary(r, d * d)
    th = rounded(bond.apply_gate(U.conj().T, T0), prec)
    Bn = rounded(W.random_right_isometry(r, 4, d, chiR), prec)
    from paper_2212_09782_b300 import lib as L
    # complex64 Schmidt values of a rank-deficient block sit at the FP32 rounding
    # floor (~1e-7 relative), so the complex64 cut uses svd_min = 1e-5
    svd_min = 1e-14 if prec == "c128" else 1e-5
    gpu = run_gpu(prec, None, None, Bn, U,
                  L.trunc_default(L.CBE, 100, dchi_min=0, eta=8, svd_min=svd_min), theta=th)
    assert gpu["chi_new"] == rank
    # eps = 1 - kept / ||theta~||^2 from two FP64 sums: zero up to their rounding
    assert gpu["eps"] < (1e-14 if prec == "c128" else 1e-6)


def _c2_full_size(prec, tol):
    import torch
    from paper_2212_09782_b300 import lib as L
    wl = W.bond_microbench(1024, 5)
    th = wl["theta"].astype(np.complex128)
    Bn = wl["Bn"].astype(np.complex128)
    U = wl["U"]
    orc = bond.qr_update(None, None, Bn, U, chi_max=1024, theta=th)
    gpu = run_gpu(prec, None, None, Bn, U, L.trunc_default(L.PLAIN, 1024), theta=th)
    s_g = np.linalg.svd(gpu["Xi_new"], compute_uv=False)
    s_o = np.linalg.svd(orc["Xi_new"], compute_uv=False)
    errs = {"schmidt": np.linalg.norm(s_g - s_o) / np.linalg.norm(s_o),
            "eps": abs(gpu["eps"] - orc["eps"]) / orc["eps"]}
    # principal angles between the GPU and oracle right spaces: all cosines ~ 1
    Bg = gpu["Bn_new"].reshape(1024, -1)
    Bo = orc["Bn_new"].reshape(1024, -1)
    cosines = np.linalg.svd(Bg @ Bo.conj().T, compute_uv=False)
    errs["angles"] = 1 - cosines.min()
    # B~^m B~^n applied to random probes
    r = W.rng(9)
    v = W.complex_gaussian(r, (Bg.shape[1], 8))
    bm_g = gpu["Bm_new"].reshape(-1, 1024)
    bm_o = orc["Bm_new"].reshape(-1, 1024)
    a, b = bm_g @ (Bg @ v), bm_o @ (Bo @ v)
    errs["BB"] = np.linalg.norm(a - b) / np.linalg.norm(b)
    print(prec, errs)
    bad = {k: e for k, e in errs.items() if not e < tol}
    assert not bad, (bad, errs)
    torch.cuda.synchronize()


def test_c2_full_size_against_oracle():
    """The bench workload (chi = 1024, d = 5, complex64 3xTF32) against the full oracle."""
    _c2_full_size("c64_3xtf32", 1e-5)


@pytest.mark.slow
def test_c2_full_size_c128_against_oracle():
    """The same workload on the complex128 path (FP64 throughout) at the 1e-10 bar."""
    _c2_full_size("c128", 1e-10)


@pytest.mark.parametrize("prec", ["c64_tf32", "c64_3xtf32"])
def test_reorth_restores_isometry(prec):
    # Precision pattern (1): one re-orthogonalisation pass of the right isometry. The
    # QR's TF32 rounding leaves B~^n B~^n^dag - 1 at the TF32 level; the pass
    # Q <- Q (1 - D/2), D = Q^dag Q - 1, takes it to O(|D|^2) plus complex64 rounding,
    # and the result still matches the oracle.
    from paper_2212_09782_b300 import lib as L
    dims = (130, 4, 130, 130)
    bd = _case(dims, seed=91, xi="diag", prec=prec)
    orc = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], scheme="plain", chi_max=130)
    iso = {}
    for ro in (0, 1):
        t = L.trunc_default(L.PLAIN, 130, reorth=ro)
        gpu = run_gpu(prec, bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], t, xi_kind=2)
        Bn = gpu["Bn_new"].reshape(130, -1)
        iso[ro] = np.abs(Bn @ Bn.conj().T - np.eye(130)).max()
        compare(gpu, orc, TOL[prec])
    print(prec, "max |B B^dag - 1| without / with the pass:", iso[0], iso[1])
    assert iso[1] <= 2e-6            # measured 9.6e-7 (1xTF32), 1.1e-6 (3xTF32)
    if prec == "c64_tf32":           # measured 9.0e-4 without the pass
        assert iso[0] > 1e-5 and iso[1] < iso[0] / 10


def _spectrum_matrix(r, n, spec):
    """A square matrix U diag(s) W^dag with a chosen singular spectrum s (descending)."""
    s = {"flat": lambda: np.ones(n), "graded": lambda: 10.0 ** (-6.0 * np.arange(n) / max(n - 1, 1)),
         "decay": lambda: np.exp(-np.arange(n) / max(n / 8, 1)),
         "rankdef": lambda: np.r_[np.linspace(1, 0.1, n - n // 2), np.zeros(n // 2)],
         # values whose row products underflow FP32 (the product-state start of a CBE run)
         "underflow": lambda: np.r_[1.0, 0.5, 10.0 ** -np.linspace(18, 30, n - 2)]}[spec]()
    U = np.linalg.qr(W.complex_gaussian(r, (n, n)))[0]
    V = np.linalg.qr(W.complex_gaussian(r, (n, n)))[0]
    return (U * s) @ V.conj().T, s


@pytest.mark.parametrize("prec", ["c128", "c64_3xtf32"])
@pytest.mark.parametrize("n,spec", [(1, "flat"), (2, "flat"), (5, "underflow"), (17, "graded"),
                                    (33, "underflow"), (64, "rankdef"), (128, "graded"),
                                    (257, "decay"), (300, "flat"), (1126, "decay")])
def test_cbe_decompose(prec, n, spec):
    # step (iv) alone: w = eigenvalues of Rz Rz^dag (= s^2), descending; the rows of Vh are
    # orthonormal and diagonalise Rz Rz^dag (degenerate spectra: any basis of each eigenspace)
    import torch
    from paper_2212_09782_b300 import lib as L
    from tests.gpu_helpers import to_dev
    r = W.rng(1000 + n)
    Rz, s = _spectrum_matrix(r, n, spec)
    Rz = rounded(Rz, prec)
    w, Vh, sweeps = L.cbe_decompose(prec, to_dev(Rz, prec))
    L.stream_check()
    w, Vh, sweeps = w.cpu().numpy(), Vh.cpu().numpy(), int(sweeps.item())
    assert np.all(np.isfinite(w)) and np.all(np.isfinite(Vh))
    # complex64: FP32 rows and rotations (~sqrt(sweeps * n) roundings per row; measured
    # up to 7.2e-6 at n = 257)
    tol = 1e-12 if prec == "c128" else 2e-5
    M = Rz @ Rz.conj().T
    ref = np.sort(np.linalg.eigvalsh(M))[::-1]
    assert np.all(np.diff(w) <= 0)
    assert np.abs(w - ref).max() <= tol * max(ref[0], 1e-300), np.abs(w - ref).max()
    assert np.abs(Vh @ Vh.conj().T - np.eye(n)).max() <= tol * 10
    recon = Vh.conj().T @ (w[:, None] * Vh)
    assert np.linalg.norm(recon - M) <= tol * 10 * np.linalg.norm(M)
    # both precisions use the one-sided solver (complex128: FP64 rows and rotations)
    assert 1 <= sweeps <= 40 or n == 1, sweeps
    # it resolves the singular values themselves to the rows' accuracy: against LAPACK's SVD
    # of Rz (the square roots of eigvalsh(Rz Rz^dag) lose everything below ~1e-8 s_1)
    sv = np.sqrt(np.maximum(w, 0))
    sref = np.linalg.svd(Rz, compute_uv=False)
    assert np.abs(sv - sref).max() <= (1e-13 if prec == "c128" else 1e-5) * sref[0]


def test_inputs_passed_as_the_bench_does():
    # bench.py hands the workload arrays to the binding as they come (torch.from_numpy +
    # .cuda()), not through this suite's row-major copies: the same update must match the
    # oracle that way too
    import torch
    from paper_2212_09782_b300 import lib as L
    wl = W.bond_microbench(128, 5)
    orc = bond.qr_update(None, None, wl["Bn"].astype(np.complex128), wl["U"], chi_max=128,
                         theta=wl["theta"].astype(np.complex128))
    up = L.BondUpdater("c64_3xtf32", 128, 5, 128, 128, L.trunc_default(L.PLAIN, 128), xi_kind=0,
                       theta_given=True)
    up.run(torch.from_numpy(wl["U"]).cuda(), torch.from_numpy(wl["Bn"]).cuda(),
           theta=torch.from_numpy(wl["theta"]).cuda())
    L.stream_check()
    _bm, xi, _bn, st = up.outputs()
    s_g = np.linalg.svd(xi.cpu().numpy().astype(np.complex128), compute_uv=False)
    s_o = np.linalg.svd(orc["Xi_new"], compute_uv=False)
    assert np.linalg.norm(s_g - s_o) / np.linalg.norm(s_o) < 1e-5
    assert abs(float(st[0]) - orc["eps"]) / orc["eps"] < 1e-5
    # a strided view is refused rather than read in the wrong order
    with pytest.raises(ValueError):
        up.run(torch.from_numpy(wl["U"]).cuda(), torch.from_numpy(wl["Bn"]).cuda().permute(2, 1, 0),
               theta=torch.from_numpy(wl["theta"]).cuda())


@pytest.mark.parametrize("prec", ["c128", "c64_3xtf32"])
@pytest.mark.parametrize("scheme", ["plain", "cbe"])
def test_als_sweeps_match_oracle(prec, scheme):
    # a random unitary gate (far from the identity, Sec. V) on a random bond: the single sweep
    # of the paper and four sweeps of the alternating least-squares solver (Sec. II comments)
    # against the oracle's, and the extra sweeps lower eps
    from paper_2212_09782_b300 import lib as L
    dims = (40, 3, 24, 40)
    bd = _case(dims, seed=1234, xi="diag", prec=prec)
    chi_max = 24 if scheme == "plain" else 30
    kw = {} if scheme == "plain" else dict(dchi_min=6, dchi_frac=0.1)
    eps = {}
    for k in (1, 4):
        orc = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], scheme=scheme, chi_max=chi_max,
                             sweeps=k, **kw)
        t = L.trunc_default(L.PLAIN if scheme == "plain" else L.CBE, chi_max, sweeps=k, **kw)
        gpu = run_gpu(prec, bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], t, xi_kind=2)
        assert gpu["chi_new"] == orc.get("chi_new", orc["eta"])
        sub = subspace_tol(TOL[prec], prec, orc["S"], orc["chi_new"]) if scheme == "cbe" else None
        compare(gpu, orc, TOL[prec], sub_tol=sub)
        eps[k] = gpu["eps"]
    assert eps[4] < eps[1]



@pytest.mark.parametrize("scheme", ["plain", "cbe"])
def test_emulated_fp64_bond_against_oracle(scheme):
    # complex128 with the large products on the tensor cores (Ozaki slices): a bond whose
    # contractions and QR updates are big enough for that path, at the complex128 bar
    from paper_2212_09782_b300 import lib as L
    dims = (400, 5, 400, 400)
    bd = _case(dims, seed=4004, xi="diag", prec="c128_oz")
    chi_max = 400 if scheme == "plain" else 380
    kw = {} if scheme == "plain" else dict(dchi_min=40, dchi_frac=0.1)
    orc = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], scheme=scheme, chi_max=chi_max, **kw)
    t = L.trunc_default(L.PLAIN if scheme == "plain" else L.CBE, chi_max, **kw)
    gpu = run_gpu("c128_oz", bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], t, xi_kind=2)
    sub = subspace_tol(TOL["c128_oz"], "c128_oz", orc["S"], orc["chi_new"]) if scheme == "cbe" else None
    errs = compare(gpu, orc, TOL["c128_oz"], sub_tol=sub)
    print(scheme, errs)


@pytest.mark.slow
def test_c2_full_size_c128_oz_against_oracle():
    """The bench workload with FP64 emulated on the tensor cores, at the 1e-10 bar."""
    _c2_full_size("c128_oz", 1e-10)


@pytest.mark.parametrize("prec", ["c64_3xtf32", "c64_tf32"])
@pytest.mark.parametrize("dims", [(256, 3, 200, 256), (144, 3, 48, 16)])
def test_lower_triangular_xi(prec, dims):
    # xi_kind 3: a lower-triangular Xi (the L / ||L|| a plain update leaves on its bond). The
    # product Xi theta~' then stops each tensor-core tile's K loop after the tile's last row
    # (144 x 144 output, chi_l = d^2 chi_r: no swap) or, after the library's N > M swap,
    # after the tile's last column (256 x 2304). The K-tiles skipped hold only zeros of Xi, so the update matches
    # the dense product's to rounding, and the oracle
    bd = _case(dims, seed=sum(dims) + 3, xi="dense", prec=prec)
    Xi = np.tril(bd["Xi"])
    Xi = Xi / np.linalg.norm(Xi)
    chiM = dims[2]
    from paper_2212_09782_b300 import lib as L
    t = L.trunc_default(L.PLAIN, chiM)
    dense = run_gpu(prec, Xi, bd["Bm"], bd["Bn"], bd["U"], t, xi_kind=1)
    lower = run_gpu(prec, Xi, bd["Bm"], bd["Bn"], bd["U"], t, xi_kind=3)
    for k in ("Bm_new", "Xi_new", "Bn_new"):
        a, b = lower[k], dense[k]
        assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max(), k
    assert abs(lower["eps"] - dense["eps"]) <= 1e-6 * max(dense["eps"], 1e-12)
    orc = bond.qr_update(Xi, bd["Bm"], bd["Bn"], bd["U"], scheme="plain", chi_max=chiM)
    compare(lower, orc, TOL[prec])
