"""GPU parity of the complex GEMM (CUDA cores and tcgen05 tensor cores) against numpy.

A library matmul in complex128 is the plain definition of the contraction."""
import numpy as np
import pytest

from paper_2212_09782_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-13, "c64_fp32": 3e-7, "c64_3xtf32": 3e-7, "c64_tf32": 4e-3}


def tol(prec, k):
    # FP32 accumulation of k complex products: max error ~ eps32 * sqrt(k) * a few; the
    # 3xTF32 path promotes its tensor-core partial sums to FP32 and must match that
    if prec in ("c64_fp32", "c64_3xtf32"):
        return TOL[prec] * np.sqrt(k) + 2e-6
    return TOL[prec]


@pytest.mark.parametrize("prec", list(TOL))
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (37, 5, 3), (128, 64, 128), (300, 170, 333),
                                   (640, 384, 1000), (257, 1030, 515)])
@pytest.mark.parametrize("ops", ["nn", "nc", "ct", "tn"])
def test_zgemm(prec, m, n, k, ops):
    import torch
    from paper_2212_09782_b300 import lib as L
    r = W.rng(m * 1000 + n * 10 + k)
    ta, tb = ops[0] in "tc", ops[1] in "tc"
    ca, cb = ops[0] == "c", ops[1] == "c"
    A = W.complex_gaussian(r, (k, m) if ta else (m, k))
    B = W.complex_gaussian(r, (n, k) if tb else (k, n))
    C0 = W.complex_gaussian(r, (m, n))
    dt = torch.complex128 if prec == "c128" else torch.complex64
    if prec != "c128":
        A, B, C0 = (x.astype(np.complex64).astype(np.complex128) for x in (A, B, C0))
    opA = A.T if ta else A
    opA = opA.conj() if ca else opA
    opB = B.T if tb else B
    opB = opB.conj() if cb else opB
    alpha, beta = 0.7 - 0.2j, -0.5 + 0.25j
    ref = alpha * (opA @ opB) + beta * C0
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dt)
    Cd = dev(C0)
    L.zgemm(prec, dev(A), dev(B), conj_a=ca, conj_b=cb, trans_a=ta, trans_b=tb, alpha=alpha,
            beta=beta, C_out=Cd)
    L.stream_check()
    got = Cd.cpu().numpy().astype(np.complex128)
    scale = np.abs(alpha) * np.sqrt(k) + np.abs(beta)
    err = np.abs(got - ref).max() / scale
    assert err < tol(prec, k), err


@pytest.mark.parametrize("prec", ["c64_3xtf32", "c64_tf32"])
@pytest.mark.parametrize("ops", ["nn", "ct"])
def test_zgemm_tail_wave_split(prec, ops):
    # 38 x 8 = 304 output tiles: two full waves on 148 SMs and one tile row left over, which
    # runs with its K split across the idle SMs (then summed); beta != 0 exercises the sum
    import torch
    from paper_2212_09782_b300 import lib as L
    m, n, k = 4864, 1024, 512
    r = W.rng(4242)
    ta, ca = ops[0] in "tc", ops[0] == "c"
    A = W.complex_gaussian(r, (k, m) if ta else (m, k)).astype(np.complex64).astype(np.complex128)
    B = W.complex_gaussian(r, (k, n)).astype(np.complex64).astype(np.complex128)
    C0 = W.complex_gaussian(r, (m, n)).astype(np.complex64).astype(np.complex128)
    opA = A.T if ta else A
    opA = opA.conj() if ca else opA
    ref = 0.5 * (opA @ B) + (0.25 - 0.5j) * C0
    Cd = torch.from_numpy(C0).to(device="cuda", dtype=torch.complex64)
    out = L.zgemm(prec, torch.from_numpy(A).to(device="cuda", dtype=torch.complex64),
                  torch.from_numpy(B).to(device="cuda", dtype=torch.complex64), conj_a=ca,
                  trans_a=ta, alpha=0.5, beta=0.25 - 0.5j, C_out=Cd)
    L.stream_check()
    got = out.cpu().numpy().astype(np.complex128)
    scale = np.abs(opA).max() * np.abs(B).max() * k
    assert np.abs(got - ref).max() / scale < (tol(prec, k) if prec != "c64_tf32" else 4e-3)
