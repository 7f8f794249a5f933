"""Shared helpers of the GPU parity tests: run the CUDA bond update and compare
gauge-invariant quantities with the oracle on identical inputs."""
import numpy as np

# 1xTF32 (10-bit products) is outside the 1e-5 bar: measured against the oracle at
# chi ~ 100-250, d = 3-4: Schmidt values ~4e-5, eps ~1e-4, projector-type invariants ~2e-3
TOL = {"c128": 1e-10, "c128_oz": 1e-10, "c64_3xtf32": 1e-5, "c64_fp32": 1e-5, "c64_tf32": 5e-3}

# Unit perturbation of the bond matrix that the arithmetic leaves (relative to its norm):
# complex64 stores X, Q, Y and L in FP32 (unit roundoff 6e-8) between FP32-accumulated
# products; complex128 stores them in FP64.
PERTURB = {"c128": 1e-15, "c128_oz": 1e-14, "c64_3xtf32": 1e-7, "c64_fp32": 1e-7, "c64_tf32": 1e-7}


def subspace_tol(tol, prec, S, c):
    """Tolerance of the kept-subspace invariants (projector, B~^m B~^n, G) after a cut at c
    values of the spectrum S (descending): the kept space moves by up to |E| / gap under a
    perturbation E of L (Davis-Kahan), gap = (S[c-1] - S[c]) / S[0], so the comparison is held
    to max(tol, PERTURB / gap); the Schmidt values and eps stay at tol."""
    if c >= len(S) or S[0] <= 0:
        return tol
    gap = (S[c - 1] - S[c]) / S[0]
    return max(tol, PERTURB[prec] / max(gap, 1e-300))


def to_dev(a, prec):
    import torch
    dt = torch.complex128 if prec.startswith("c128") else torch.complex64
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dt, device="cuda")


def host(a):
    return a.detach().cpu().numpy().astype(np.complex128)


def rounded(a, prec):
    """Inputs as the device sees them (complex64 paths store complex64)."""
    return a.astype(np.complex64).astype(np.complex128) if not prec.startswith("c128") else np.asarray(a, np.complex128)


def run_gpu(prec, Xi, Bm, Bn, U, trunc, theta=None, xi_kind=None):
    import torch
    from paper_2212_09782_b300 import lib as L
    chiL = (theta.shape[0] if theta is not None else Bm.shape[0])
    d = U.shape[0]
    d = int(round(d ** 0.5))
    chiM, chiR = Bn.shape[0], Bn.shape[2]
    if xi_kind is None:
        xi_kind = 0 if Xi is None else 1
    up = L.BondUpdater(prec, chiL, d, chiM, chiR, trunc, xi_kind=xi_kind,
                       theta_given=theta is not None)
    xi_dev = None
    if Xi is not None:
        xi_dev = to_dev(np.diag(Xi) if xi_kind == 2 else Xi, prec)
    gate = torch.from_numpy(np.ascontiguousarray(U, np.complex128)).cuda()
    info = up.run(gate, to_dev(Bn, prec), theta=None if theta is None else to_dev(theta, prec),
                  bm=None if Bm is None else to_dev(Bm, prec), xi=xi_dev)
    L.stream_check()
    bm, xi, bn, st = up.outputs()
    return {"Bm_new": host(bm), "Xi_new": host(xi), "Bn_new": host(bn),
            "eps": float(st[0].item()), "th2": float(st[1].item()), "kept": float(st[2].item()),
            "chi_new": info.chi_new, "eta": info.eta, "S": up.schmidt.cpu().numpy()}


def invariants(out):
    Xi = out["Xi_new"]
    c = Xi.shape[0]
    Bn = out["Bn_new"].reshape(c, -1)
    Bm = out["Bm_new"].reshape(-1, c)
    return {
        "s": np.linalg.svd(Xi, compute_uv=False),
        "P": Bn.conj().T @ Bn,                  # projector on the new right space
        "BB": Bm @ Bn,                          # theta~' P_n
        "G": (Xi @ Bn).conj().T @ (Xi @ Bn),    # Y^dag Y / ||L||^2
    }


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def compare(gpu, orc, tol, keys=("s", "P", "BB", "G"), eps=True, sub_tol=None):
    """sub_tol: the tolerance of the kept-subspace invariants (P, BB, G), default tol."""
    ig, io = invariants(gpu), invariants(orc)
    errs = {k: rel(ig[k], io[k]) for k in keys}
    if eps:
        errs["eps"] = abs(gpu["eps"] - orc["eps"]) / max(abs(orc["eps"]), 1e-300)
        if orc["eps"] < 1e-7:
            errs["eps"] = abs(gpu["eps"] - orc["eps"])
    lim = {k: (sub_tol if (sub_tol is not None and k in ("P", "BB", "G")) else tol) for k in errs}
    bad = {k: v for k, v in errs.items() if not (v <= lim[k])}
    assert not bad, (bad, errs)
    # exact isometry of B~^n (Sec. II: Q^[n] has orthonormal rows)
    c = gpu["Xi_new"].shape[0]
    Bn = gpu["Bn_new"].reshape(c, -1)
    iso = np.abs(Bn @ Bn.conj().T - np.eye(c)).max()
    assert iso <= max(tol, 1e-6 if tol > 1e-9 else 1e-12), iso
    assert abs(np.linalg.norm(gpu["Xi_new"]) - 1) <= max(tol, 1e-6)
    return errs
