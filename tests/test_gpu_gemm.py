"""GPU parity of the complex GEMM (CUDA cores and tcgen05 tensor cores) against numpy.

A library matmul in complex128 is the plain definition of the contraction."""
import numpy as np
import pytest

from paper_2212_09782_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-13, "c128_oz": 1e-13, "c64_fp32": 3e-7, "c64_3xtf32": 3e-7, "c64_tf32": 4e-3}


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
    dt = torch.complex128 if prec.startswith("c128") else torch.complex64
    if not prec.startswith("c128"):
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


@pytest.mark.parametrize("prec", ["c64_3xtf32", "c64_tf32"])
@pytest.mark.parametrize("m,n,k", [(640, 384, 1000), (5000, 160, 333), (300, 170, 2500)])
@pytest.mark.parametrize("config", [(128, 1, 0), (128, 1, 1), (128, 3, 0), (256, 5, 0),
                                    (128, 32, 0), (256, 1, 0)])
def test_zgemm_tuned_configs(prec, m, n, k, config):
    # every launch configuration the autotuner can choose (tile width 128/256, K-splits,
    # tail-wave split) gives the same product; entries are keyed on the swapped shape
    # (M >= N), which these m >= n cases are already
    import torch
    from paper_2212_09782_b300 import lib as L
    r = W.rng(m + 7 * n + 13 * k)
    A = W.complex_gaussian(r, (m, k)).astype(np.complex64).astype(np.complex128)
    B = W.complex_gaussian(r, (k, n)).astype(np.complex64).astype(np.complex128)
    C0 = W.complex_gaussian(r, (m, n)).astype(np.complex64).astype(np.complex128)
    alpha, beta = 1.0 + 0.5j, 0.5 - 1.0j
    ref = alpha * (A @ B) + beta * C0
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=torch.complex64)
    L.autotune_clear()
    try:
        L.autotune_set((m, n, k, 1 if prec == "c64_3xtf32" else 0), config)
        Cd = dev(C0)
        L.zgemm(prec, dev(A), dev(B), alpha=alpha, beta=beta, C_out=Cd)
        L.stream_check()
    finally:
        L.autotune_clear()
    got = Cd.cpu().numpy().astype(np.complex128)
    err = np.abs(got - ref).max() / (np.abs(alpha) * np.sqrt(k) + np.abs(beta))
    assert err < tol(prec, k), err


def test_autotune_bond_table_and_parity():
    # the tuner records the products of one bond update, times the candidates of each and
    # keeps the fastest (never slower than the heuristic as measured); an update with the
    # tuned table still matches the oracle
    from oracle import bond
    from paper_2212_09782_b300 import lib as L
    from tests.gpu_helpers import TOL as BTOL, compare, rounded, run_gpu
    chi, d = 192, 4
    t = L.trunc_default(L.PLAIN, chi)
    L.autotune_clear()
    try:
        n = L.autotune_bond("c64_3xtf32", chi, d, chi, chi, t, xi_kind=0, theta_given=True)
        ents = L.autotune_entries()
        assert n == len(ents) > 0
        for e in ents:
            M, N, K, three = e["shape"]
            bn, splits, tail = e["config"]
            assert M >= N and three == 1 and bn in (128, 256) and 0 <= splits <= 32
            assert 0 < e["ms_tuned"] <= e["ms_default"]
        assert L.autotune_bond("c64_3xtf32", chi, d, chi, chi, t, xi_kind=0, theta_given=True) == 0
        r = W.rng(77)
        th = W.complex_gaussian(r, (chi, d, d, chi))
        th = rounded(th / np.linalg.norm(th), "c64_3xtf32")
        U = W.random_unitary(r, d * d)
        Bn = rounded(W.random_right_isometry(r, chi, d, chi), "c64_3xtf32")
        orc = bond.qr_update(None, None, Bn, U, chi_max=chi, theta=th)
        gpu = run_gpu("c64_3xtf32", None, None, Bn, U, t, theta=th)
        compare(gpu, orc, BTOL["c64_3xtf32"])
    finally:
        L.autotune_clear()


@pytest.mark.parametrize("m,n,k", [(2048, 1024, 777), (1500, 600, 2048), (1030, 2100, 333), (5120, 256, 130),
                                   (128, 256, 5000), (1024, 100, 4097), (300, 130, 2000)])
@pytest.mark.parametrize("ops", ["nn", "ct", "tc", "nc"])
def test_zgemm_emulated_fp64(m, n, k, ops):
    # complex128 on the tensor cores (Ozaki slices): products large enough for the tensor-core
    # path (>= 64 output tiles), and products of few tiles and a long K whose slice pairs are
    # split over CTAs and summed; ragged in every dimension, transposed and conjugated operands;
    # relative to the FP64 product the error must stay at complex128 level
    import torch
    from paper_2212_09782_b300 import lib as L
    r = W.rng(m + 7 * n + 13 * k)
    ta, tb = ops[0] in "tc", ops[1] in "tc"
    ca, cb = ops[0] == "c", ops[1] == "c"
    A = W.complex_gaussian(r, (k, m) if ta else (m, k))
    B = W.complex_gaussian(r, (n, k) if tb else (k, n))
    # rows of very different magnitudes: each row takes its own power-of-two scale
    A = A * (10.0 ** r.uniform(-6, 6, size=(A.shape[0], 1)))
    C0 = W.complex_gaussian(r, (m, n))
    opA = (A.T if ta else A)
    opA = opA.conj() if ca else opA
    opB = (B.T if tb else B)
    opB = opB.conj() if cb else opB
    alpha, beta = 0.7 - 0.2j, -0.5 + 0.25j
    ref = alpha * (opA @ opB) + beta * C0
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=torch.complex128)
    Cd = dev(C0)
    L.zgemm("c128_oz", dev(A), dev(B), conj_a=ca, conj_b=cb, trans_a=ta, trans_b=tb, alpha=alpha,
            beta=beta, C_out=Cd)
    L.stream_check()
    got = Cd.cpu().numpy()
    # error of each row relative to the size of that row's terms
    row_scale = np.abs(opA) @ np.abs(opB) * abs(alpha) + abs(beta) * np.abs(C0)
    err = (np.abs(got - ref) / row_scale).max()
    assert err < 1e-13, err


def test_zgemm_emulated_fp64_exact_on_integers():
    # integer operands of up to 8 bits are single slices: every product and every 128-term
    # chunk sum is an integer below 2^24, so the emulated product must be exact
    import torch
    from paper_2212_09782_b300 import lib as L
    r = W.rng(99)
    m, n, k = 1024, 1024, 1000
    A = r.integers(-127, 128, size=(m, k)) + 1j * r.integers(-127, 128, size=(m, k))
    B = r.integers(-127, 128, size=(k, n)) + 1j * r.integers(-127, 128, size=(k, n))
    ref = A @ B
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=torch.complex128)
    out = L.zgemm("c128_oz", dev(A), dev(B))
    L.stream_check()
    assert np.array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("prec", ["c64_3xtf32", "c64_tf32"])
@pytest.mark.parametrize("m,n,k", [(128, 64, 128), (640, 384, 1000), (300, 170, 334), (258, 1030, 516),
                                   (4864, 1024, 512)])
@pytest.mark.parametrize("ops", ["nn", "nc", "ct", "tn", "cc"])
def test_zgemm_operand_prep_in_kernel(prec, m, n, k, ops):
    # 128-column tiles forced through the tuning table, so the in-kernel preparation runs
    # (raw operands split and embedded by the epilogue warps into swizzled stages) for every
    # layout it takes: A contiguous along K or M, B along K or N, conjugated, K ragged
    # against the 16-value stage; it must equal the separate pass bit for bit and numpy
    import torch
    from paper_2212_09782_b300 import lib as L
    three = 1 if prec == "c64_3xtf32" else 0
    M, N = (n, m) if n > m else (m, n)
    r = W.rng(m * 1000 + n * 10 + k)
    ta, tb = ops[0] in "tc", ops[1] in "tc"
    ca, cb = ops[0] == "c", ops[1] == "c"
    A = W.complex_gaussian(r, (k, m) if ta else (m, k)).astype(np.complex64)
    B = W.complex_gaussian(r, (n, k) if tb else (k, n)).astype(np.complex64)
    C0 = W.complex_gaussian(r, (m, n)).astype(np.complex64)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    alpha, beta = 0.7 - 0.2j, -0.5 + 0.25j
    outs = []
    prev = L.tc_operand_prep(0)
    try:
        L.autotune_set((M, N, k, three), (128, 0, 1))
        for mode in (0, 1):
            L.tc_operand_prep(mode)
            Cd = dev(C0)
            L.zgemm(prec, dev(A), dev(B), conj_a=ca, conj_b=cb, trans_a=ta, trans_b=tb, alpha=alpha,
                    beta=beta, C_out=Cd)
            L.stream_check()
            outs.append(Cd.cpu().numpy().astype(np.complex128))
    finally:
        L.tc_operand_prep(prev)
        L.autotune_clear()
    assert np.array_equal(outs[0], outs[1])
    opA = A.astype(np.complex128)
    opA = opA.T if ta else opA
    opA = opA.conj() if ca else opA
    opB = B.astype(np.complex128)
    opB = opB.T if tb else opB
    opB = opB.conj() if cb else opB
    ref = alpha * (opA @ opB) + beta * C0.astype(np.complex128)
    err = np.abs(outs[0] - ref).max() / (np.abs(alpha) * np.sqrt(k) + np.abs(beta))
    assert err < tol(prec, k), err


def test_operand_prep_mode_switch():
    from paper_2212_09782_b300 import lib as L
    prev = L.tc_operand_prep(0)
    try:
        assert L.tc_operand_prep(1) == 0
        with pytest.raises(L.QrtebdError):
            L.tc_operand_prep(2)
    finally:
        L.tc_operand_prep(prev)
