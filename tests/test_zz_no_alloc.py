"""qrtebd_zgemm_noalloc: the GEMM variant for callers that cannot allocate device memory.

It keeps its scratch in a fixed device array inside the library instead of a caller
workspace. Checked through the C ABI against qrtebd_zgemm on two calls in a row (the
second reuses the array the first left behind), and for its size limit. Collected
last so that a run stopping at the first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2212_09782_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _fn(L):
    f = L.raw().qrtebd_zgemm_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_longlong, C.c_longlong,
                  C.c_int, C.c_void_p, C.c_longlong, C.c_longlong, C.c_int, C.c_void_p,
                  C.c_longlong, C.c_longlong, C.POINTER(C.c_double), C.POINTER(C.c_double),
                  C.c_void_p]
    return f


def _noalloc(L, prec, A, B, Cm, ta, ca, tb, cb, alpha, beta):
    m = A.shape[1] if ta else A.shape[0]
    k = A.shape[0] if ta else A.shape[1]
    n = B.shape[0] if tb else B.shape[1]
    sam, sak = (1, A.shape[1]) if ta else (A.shape[1], 1)
    sbk, sbn = (1, B.shape[1]) if tb else (B.shape[1], 1)
    al = (C.c_double * 2)(alpha.real, alpha.imag)
    be = (C.c_double * 2)(beta.real, beta.imag)
    f = _fn(L)
    return f(L.PRECISIONS[prec], m, n, k, C.c_void_p(A.data_ptr()), sam, sak, int(ca),
             C.c_void_p(B.data_ptr()), sbk, sbn, int(cb), C.c_void_p(Cm.data_ptr()),
             Cm.shape[1], 1, al, be, L.stream_handle())


@pytest.mark.parametrize("prec", ["c64_3xtf32", "c64_tf32"])
def test_noalloc_matches_zgemm_twice(prec):
    import torch
    from paper_2212_09782_b300 import lib as L
    # 512^3 fills the embedded B'^T region exactly and leaves room for only two split-K
    # partial blocks; 300 x 512 x 512 takes the N > M swap at the cap
    cases = [((200, 300, 400), "nn", 0.7 - 0.2j, 0.0),
             ((512, 96, 512), "ct", 1.0, -0.5 + 0.25j),
             ((512, 512, 512), "nc", 0.3 + 0.1j, 1.0),
             ((300, 512, 512), "tn", 1.0, 0.0)]
    for (m, n, k), ops, alpha, beta in cases:
        r = W.rng(m + n + k)
        ta, tb = ops[0] in "tc", ops[1] in "tc"
        ca, cb = ops[0] == "c", ops[1] == "c"
        dev = lambda x: torch.from_numpy(x.astype(np.complex64)).cuda()
        A = dev(W.complex_gaussian(r, (k, m) if ta else (m, k)))
        B = dev(W.complex_gaussian(r, (n, k) if tb else (k, n)))
        C0 = dev(W.complex_gaussian(r, (m, n)))
        ref = L.zgemm(prec, A, B, conj_a=ca, conj_b=cb, trans_a=ta, trans_b=tb, alpha=alpha,
                      beta=beta, C_out=C0.clone())
        got = C0.clone()
        assert _noalloc(L, prec, A, B, got, ta, ca, tb, cb, complex(alpha), complex(beta)) == 0
        L.stream_check()
        scale = abs(alpha) * np.sqrt(k) + abs(beta)
        tol = 3e-7 * np.sqrt(k) + 2e-6 if prec == "c64_3xtf32" else 4e-3
        err = (got - ref).abs().max().item() / scale
        assert err < tol, err


def test_noalloc_empty_sizes_as_zgemm():
    import torch
    from paper_2212_09782_b300 import lib as L
    f = _fn(L)
    A = torch.ones(8, 4, dtype=torch.complex64, device="cuda")
    B = torch.ones(4, 6, dtype=torch.complex64, device="cuda")
    C0 = torch.full((8, 6), 2 - 1j, dtype=torch.complex64, device="cuda")
    al = (C.c_double * 2)(1.0, 0.0)
    be = (C.c_double * 2)(0.0, 0.5)
    ptr = lambda t: C.c_void_p(t.data_ptr())

    def call(m, n, k, Cm):
        return f(L.C64_3XTF32, m, n, k, ptr(A), 4, 1, 0, ptr(B), 6, 1, 0, ptr(Cm), 6, 1, al, be,
                 L.stream_handle())
    # k = 0: C = beta C
    got = C0.clone()
    assert call(8, 6, 0, got) == 0
    L.stream_check()
    assert torch.allclose(got, C0 * 0.5j)
    # m = 0 or n = 0: nothing written
    for m, n in ((0, 6), (8, 0)):
        got = C0.clone()
        assert call(m, n, 4, got) == 0
        L.stream_check()
        assert torch.equal(got, C0)
    assert call(-1, 6, 4, C0.clone()) == L.ERR_INVALID_ARG


def test_noalloc_rejects_oversize_and_cuda_core_precisions():
    import torch
    from paper_2212_09782_b300 import lib as L
    A = torch.zeros(513, 8, dtype=torch.complex64, device="cuda")
    B = torch.zeros(8, 8, dtype=torch.complex64, device="cuda")
    Cm = torch.zeros(513, 8, dtype=torch.complex64, device="cuda")
    rc = _noalloc(L, "c64_3xtf32", A, B, Cm, False, False, False, False, 1 + 0j, 0j)
    assert rc == L.ERR_INVALID_ARG
    assert "QRTEBD_NOALLOC_MAX_DIM" in L.raw().qrtebd_last_error_message().decode()
    A2 = torch.zeros(8, 8, dtype=torch.complex64, device="cuda")
    C2 = torch.zeros(8, 8, dtype=torch.complex64, device="cuda")
    assert _noalloc(L, "c64_fp32", A2, B, C2, False, False, False, False, 1 + 0j, 0j) == L.ERR_INVALID_ARG
