"""ctypes binding of libqrtebd (include/qrtebd.h): argument marshalling only.

Device memory comes from torch CUDA tensors (complex64 / complex128); every step
of the bond update runs in the library's CUDA kernels. Loading fails loudly if
the shared library is missing: there is no CPU fallback.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqrtebd.so")

OK = 0
ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NUMERIC, ERR_NOT_ADMITTED = -1, -2, -3, -4, -5, -6
C128, C64_3XTF32, C64_TF32, C64_FP32, C128_OZ = 0, 1, 2, 3, 4
PLAIN, CBE = 0, 1
PRECISIONS = {"c128": C128, "c64_3xtf32": C64_3XTF32, "c64_tf32": C64_TF32, "c64_fp32": C64_FP32,
              "c128_oz": C128_OZ}


def is_c128(precision):
    """complex128 storage (FP64 arithmetic, or FP64 emulated on the tensor cores)."""
    p = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
    return p in (C128, C128_OZ)


class Trunc(C.Structure):
    _fields_ = [("scheme", C.c_int), ("chi_max", C.c_int), ("eta", C.c_int), ("dchi_min", C.c_int),
                ("dchi_frac", C.c_double), ("svd_min", C.c_double), ("tie_tol", C.c_double),
                ("eps_explicit", C.c_int), ("eps_target", C.c_double), ("reorth", C.c_int),
                ("sweeps", C.c_int)]


class BondIO(C.Structure):
    _fields_ = [("precision", C.c_int), ("chi_l", C.c_int), ("d", C.c_int), ("chi_m", C.c_int),
                ("chi_r", C.c_int), ("xi_kind", C.c_int), ("xi", C.c_void_p), ("bm", C.c_void_p),
                ("bn", C.c_void_p), ("theta", C.c_void_p), ("gate", C.c_void_p),
                ("bm_out", C.c_void_p), ("xi_out", C.c_void_p), ("bn_out", C.c_void_p),
                ("stats_out", C.c_void_p), ("schmidt_out", C.c_void_p),
                ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t)]


class SymBondIO(C.Structure):
    _fields_ = [("precision", C.c_int), ("chi_l", C.c_int), ("d", C.c_int), ("chi_m", C.c_int),
                ("chi_r", C.c_int), ("charge_l", C.POINTER(C.c_int)),
                ("charge_m", C.POINTER(C.c_int)), ("charge_r", C.POINTER(C.c_int)),
                ("xi_kind", C.c_int), ("xi", C.c_void_p), ("theta", C.c_void_p),
                ("bm", C.c_void_p), ("bn", C.c_void_p),
                ("gate", C.c_void_p), ("bm_out", C.c_void_p), ("xi_out", C.c_void_p),
                ("bn_out", C.c_void_p), ("charge_out", C.POINTER(C.c_int)),
                ("chi_sector_out", C.POINTER(C.c_int)), ("stats_out", C.c_void_p),
                ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t)]


class BondInfo(C.Structure):
    _fields_ = [("eta", C.c_int), ("chi_new", C.c_int)]


class QrtebdError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.qrtebd_last_error_message().decode() if _lib else ""
        super().__init__(f"{where}: {strerror(status)} ({status}) {msg}")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libqrtebd.so not built ({LIB_PATH}); run python -m paper_2212_09782_b300.build")
    lib = C.CDLL(LIB_PATH)
    P, I, D, S = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    LL = C.c_longlong
    sig = {
        "qrtebd_trunc_default": (I, [C.POINTER(Trunc), I, I]),
        "qrtebd_bond_workspace_size": (I, [I, I, I, I, I, I, I, C.POINTER(Trunc), C.POINTER(S)]),
        "qrtebd_bond_update": (I, [C.POINTER(BondIO), C.POINTER(Trunc), P, C.POINTER(BondInfo)]),
        "qrtebd_sym_bond_workspace_size": (I, [I, I, I, I, I, C.POINTER(I), C.POINTER(I),
                                               C.POINTER(I), I, I, C.POINTER(Trunc),
                                               C.POINTER(S), C.POINTER(I)]),
        "qrtebd_clock_bond_gate_charge": (I, [I, D, D, D, D, D, C.POINTER(D)]),
        "qrtebd_sym_bond_update": (I, [C.POINTER(SymBondIO), C.POINTER(Trunc), P,
                                       C.POINTER(BondInfo)]),
        "qrtebd_stream_check": (I, [P]),
        "qrtebd_set_spin_limit": (I, [LL]),
        "qrtebd_selftest_barrier_timeout": (I, [P]),
        "qrtebd_zgemm": (I, [I, I, I, I, P, LL, LL, I, P, LL, LL, I, P, LL, LL,
                             C.POINTER(D), C.POINTER(D), P, S, P]),
        "qrtebd_zgemm_workspace_size": (S, [I, I, I]),
        "qrtebd_clock_bond_gate": (I, [I, D, D, D, D, D, C.POINTER(D)]),
        "qrtebd_strerror": (C.c_char_p, [I]),
        "qrtebd_last_error_message": (C.c_char_p, []),
        "qrtebd_version": (C.c_char_p, []),
        "qrtebd_launch_count": (C.c_longlong, []),
        "qrtebd_layer_workers": (I, []),
        "qrtebd_autotune_bond": (I, [I, I, I, I, I, I, I, C.POINTER(Trunc), P, C.POINTER(I)]),
        "qrtebd_autotune_count": (I, []),
        "qrtebd_autotune_entry": (I, [I, C.POINTER(I), C.POINTER(I), C.POINTER(D)]),
        "qrtebd_autotune_set": (I, [C.POINTER(I), C.POINTER(I)]),
        "qrtebd_autotune_clear": (None, []),
        "qrtebd_tc_operand_prep": (I, [I, C.POINTER(I)]),
        "qrtebd_cbe_decompose_workspace_size": (S, [I, I]),
        "qrtebd_cbe_decompose": (I, [I, I, P, LL, P, P, P, S, P, P]),
        "qrtebd_householder_qr": (I, [I, I, I, P, LL, P, LL, P, S, P]),
        "qrtebd_qr_workspace_size": (S, [I, I, I]),
        "qrtebd_profile_enable": (I, [I]),
        "qrtebd_profile_read": (I, [I, C.POINTER(D), C.POINTER(C.c_longlong), C.POINTER(D),
                                    C.POINTER(D)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def raw():
    """The ctypes CDLL handle."""
    return _lib


def strerror(status):
    return _lib.qrtebd_strerror(status).decode()


def check(status, where):
    if status != OK:
        raise QrtebdError(status, where)


def version():
    return _lib.qrtebd_version().decode()


def trunc_default(scheme=PLAIN, chi_max=1024, **over):
    t = Trunc()
    check(_lib.qrtebd_trunc_default(C.byref(t), scheme, chi_max), "trunc_default")
    for k, v in over.items():
        setattr(t, k, v)
    return t


def clock_bond_gate(d, g, wl, wr, tau):
    """exp(-i tau h_b) of the clock model as a complex128 numpy (d^2, d^2) array (host)."""
    out = np.zeros(2 * d ** 4, np.float64)
    tau = complex(tau)
    check(_lib.qrtebd_clock_bond_gate(d, g, wl, wr, tau.real, tau.imag,
                                      out.ctypes.data_as(C.POINTER(C.c_double))), "clock_bond_gate")
    return out.view(np.complex128).reshape(d * d, d * d)


def clock_bond_gate_charge(d, g, wl, wr, tau):
    """The clock-model bond gate in the charge (Fourier) basis of the Z_d symmetry."""
    out = np.zeros(2 * d ** 4, np.float64)
    tau = complex(tau)
    check(_lib.qrtebd_clock_bond_gate_charge(d, g, wl, wr, tau.real, tau.imag,
                                             out.ctypes.data_as(C.POINTER(C.c_double))),
          "clock_bond_gate_charge")
    return out.view(np.complex128).reshape(d * d, d * d)


def bond_workspace_size(precision, chi_l, d, chi_m, chi_r, trunc, xi_kind=1, theta_given=False):
    n = C.c_size_t(0)
    check(_lib.qrtebd_bond_workspace_size(precision, chi_l, d, chi_m, chi_r, xi_kind,
                                          1 if theta_given else 0, C.byref(trunc), C.byref(n)),
          "bond_workspace_size")
    return n.value


def _ptr(t):
    """Device pointer of a tensor the C ABI reads as dense row-major data. A tensor with any
    other strides (a transpose, a permuted view) would be read in the wrong order, so it is
    refused rather than copied behind the caller's back."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError(f"the library takes contiguous (row-major) tensors; got shape "
                         f"{tuple(t.shape)} with strides {t.stride()} (call .contiguous())")
    return C.c_void_p(t.data_ptr())


def _ptr_rows(t):
    """Device pointer of a 2-D tensor passed with its row stride as the leading dimension:
    rows may be spaced out, the elements of a row must be adjacent."""
    if t.dim() != 2 or t.stride(1) != 1 or t.stride(0) < t.shape[1]:
        raise ValueError(f"expected a 2-D tensor with unit column stride; got shape "
                         f"{tuple(t.shape)} with strides {t.stride()}")
    return C.c_void_p(t.data_ptr())


def stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class BondUpdater:
    """Holds the workspace and output buffers for repeated updates of one shape.

    Inputs are torch CUDA tensors of the precision's dtype (complex128 for c128 / c128_oz,
    complex64 otherwise); ``gate`` is a complex128 CUDA tensor (d^2, d^2).
    """

    def __init__(self, precision, chi_l, d, chi_m, chi_r, trunc, xi_kind=1, theta_given=False,
                 device="cuda"):
        import torch
        self.torch = torch
        self.precision = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
        self.dtype = torch.complex128 if is_c128(self.precision) else torch.complex64
        self.dims = (chi_l, d, chi_m, chi_r)
        self.trunc = trunc
        self.xi_kind = xi_kind
        self.theta_given = theta_given
        nbytes = bond_workspace_size(self.precision, chi_l, d, chi_m, chi_r, trunc, xi_kind, theta_given)
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        eta = self.eta_bound()
        self.bm_out = torch.empty(chi_l * d * eta, dtype=self.dtype, device=device)
        self.xi_out = torch.empty(eta * eta, dtype=self.dtype, device=device)
        self.bn_out = torch.empty(eta * d * chi_r, dtype=self.dtype, device=device)
        self.stats = torch.zeros(4, dtype=torch.float64, device=device)
        self.schmidt = torch.zeros(max(eta, 1), dtype=torch.float64, device=device)

    def eta_bound(self):
        chi_l, d, chi_m, chi_r = self.dims
        t = self.trunc
        cap = min(d * chi_l, d * chi_r)
        if t.eta > 0:
            return min(t.eta, cap)
        if t.scheme == PLAIN:
            return min(t.chi_max, cap)
        import math
        dchi = max(t.dchi_min, int(math.ceil(t.dchi_frac * chi_m - 1e-9)))
        return min(chi_m + dchi, cap)

    def run(self, gate, bn, theta=None, bm=None, xi=None, stream=None):
        """Enqueue one update; returns BondInfo (eta, chi_new). Outputs stay in this object."""
        chi_l, d, chi_m, chi_r = self.dims
        io = BondIO()
        io.precision = self.precision
        io.chi_l, io.d, io.chi_m, io.chi_r = chi_l, d, chi_m, chi_r
        io.xi_kind = self.xi_kind if xi is not None else 0
        io.xi = _ptr(xi)
        io.bm = _ptr(bm)
        io.bn = _ptr(bn)
        io.theta = _ptr(theta)
        io.gate = _ptr(gate)
        io.bm_out = _ptr(self.bm_out)
        io.xi_out = _ptr(self.xi_out)
        io.bn_out = _ptr(self.bn_out)
        io.stats_out = _ptr(self.stats)
        io.schmidt_out = _ptr(self.schmidt)
        io.workspace = _ptr(self.workspace)
        io.workspace_bytes = self.workspace.numel()
        info = BondInfo()
        check(_lib.qrtebd_bond_update(C.byref(io), C.byref(self.trunc), stream_handle(stream),
                                      C.byref(info)), "bond_update")
        self.info = info
        return info

    def outputs(self):
        """(Bm_new (chi_l, d, c), Xi_new (c, c), Bn_new (c, d, chi_r), stats) as torch views."""
        chi_l, d, chi_m, chi_r = self.dims
        c = self.info.chi_new
        return (self.bm_out[: chi_l * d * c].view(chi_l, d, c),
                self.xi_out[: c * c].view(c, c),
                self.bn_out[: c * d * chi_r].view(c, d, chi_r),
                self.stats)


def _int_array(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int32))
    return a, a.ctypes.data_as(C.POINTER(C.c_int))


def sym_bond_workspace_size(precision, chi_l, d, chi_m, chi_r, charge_l, charge_m, charge_r,
                            trunc, xi_kind=2, theta_given=True):
    """(workspace bytes, eta_sum) of a charge-conserving CBE update."""
    precision = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
    (al, pl), (am, pm), (ar, pr) = _int_array(charge_l), _int_array(charge_m), _int_array(charge_r)
    n, e = C.c_size_t(0), C.c_int(0)
    check(_lib.qrtebd_sym_bond_workspace_size(precision, chi_l, d, chi_m, chi_r, pl, pm, pr,
                                              xi_kind, 1 if theta_given else 0, C.byref(trunc),
                                              C.byref(n), C.byref(e)),
          "sym_bond_workspace_size")
    return n.value, e.value


class SymBondUpdater:
    """Workspace and outputs of one charge-conserving CBE update (Sec. III with Z_d charges).

    The charges of the three bonds are host integer sequences; theta' (chi_l, d, d, chi_r),
    the diagonal xi (chi_l,) and the complex128 gate (d^2, d^2) are torch CUDA tensors.
    """

    def __init__(self, precision, d, charge_l, charge_m, charge_r, trunc, xi_kind=2,
                 theta_given=True, device="cuda"):
        import torch
        self.precision = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
        self.dtype = torch.complex128 if is_c128(self.precision) else torch.complex64
        self.charges = [np.asarray(c, np.int32) for c in (charge_l, charge_m, charge_r)]
        chi_l, chi_m, chi_r = (len(c) for c in self.charges)
        self.dims = (chi_l, d, chi_m, chi_r)
        self.trunc = trunc
        self.xi_kind = xi_kind
        nbytes, self.eta_sum = sym_bond_workspace_size(self.precision, chi_l, d, chi_m, chi_r,
                                                       *self.charges, trunc, xi_kind,
                                                       theta_given)
        self.cap = min(trunc.chi_max, self.eta_sum)
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        self.bm_out = torch.empty(chi_l * d * self.cap, dtype=self.dtype, device=device)
        self.xi_out = torch.empty(self.cap, dtype=self.dtype, device=device)
        self.bn_out = torch.empty(self.cap * d * chi_r, dtype=self.dtype, device=device)
        self.stats = torch.zeros(4, dtype=torch.float64, device=device)
        self.charge_out = np.zeros(self.cap, np.int32)
        self.chi_sector = np.zeros(d, np.int32)

    def run(self, gate, theta=None, xi=None, bm=None, bn=None, stream=None):
        """One update (synchronises the stream once); returns BondInfo (eta_sum, chi_new).
        theta' is given, or B^m and B^n are (then theta' = B^m B^n in the library)."""
        chi_l, d, chi_m, chi_r = self.dims
        io = SymBondIO()
        io.precision = self.precision
        io.chi_l, io.d, io.chi_m, io.chi_r = chi_l, d, chi_m, chi_r
        (cl, io.charge_l), (cm, io.charge_m), (cr, io.charge_r) = (_int_array(c) for c in self.charges)
        io.xi_kind = self.xi_kind if xi is not None else 0
        io.xi = _ptr(xi)
        io.theta = _ptr(theta)
        io.bm = _ptr(bm)
        io.bn = _ptr(bn)
        io.gate = _ptr(gate)
        io.bm_out = _ptr(self.bm_out)
        io.xi_out = _ptr(self.xi_out)
        io.bn_out = _ptr(self.bn_out)
        io.charge_out = self.charge_out.ctypes.data_as(C.POINTER(C.c_int))
        io.chi_sector_out = self.chi_sector.ctypes.data_as(C.POINTER(C.c_int))
        io.stats_out = _ptr(self.stats)
        io.workspace = _ptr(self.workspace)
        io.workspace_bytes = self.workspace.numel()
        info = BondInfo()
        check(_lib.qrtebd_sym_bond_update(C.byref(io), C.byref(self.trunc), stream_handle(stream),
                                          C.byref(info)), "sym_bond_update")
        self.info = info
        return info

    def outputs(self):
        """(Bm_new (chi_l, d, c), xi_new (c,), Bn_new (c, d, chi_r), charges (c,), stats)."""
        chi_l, d, chi_m, chi_r = self.dims
        c = self.info.chi_new
        return (self.bm_out[: chi_l * d * c].view(chi_l, d, c), self.xi_out[:c],
                self.bn_out[: c * d * chi_r].view(c, d, chi_r), self.charge_out[:c].copy(),
                self.stats)


PROF_TC_GEMM, PROF_QR_PANEL, PROF_SIMT_GEMM, PROF_PREP, PROF_GATE, PROF_BOND_GEMM = 0, 1, 2, 3, 4, 5


def launch_count():
    return int(_lib.qrtebd_launch_count())


def profile_enable(on=True):
    check(_lib.qrtebd_profile_enable(1 if on else 0), "profile_enable")


def profile_read(family):
    """(total_ms, launches, flops, bytes) of one kernel family since profile_enable."""
    t, f, b = C.c_double(0), C.c_double(0), C.c_double(0)
    n = C.c_longlong(0)
    check(_lib.qrtebd_profile_read(family, C.byref(t), C.byref(n), C.byref(f), C.byref(b)),
          "profile_read")
    return t.value, n.value, f.value, b.value


def stream_check(stream=None):
    check(_lib.qrtebd_stream_check(stream_handle(stream)), "stream_check")


def set_spin_limit(polls=0):
    """Poll limit of the library's grid-wide barriers on the current device (0: default)."""
    check(_lib.qrtebd_set_spin_limit(int(polls)), "set_spin_limit")


def selftest_barrier_timeout(stream=None):
    """Enqueue one CTA whose grid barrier nothing releases; stream_check then raises TIMEOUT."""
    check(_lib.qrtebd_selftest_barrier_timeout(stream_handle(stream)), "selftest_barrier_timeout")


def householder_qr(precision, A, stream=None):
    """QR of a 2-D torch CUDA tensor (m x n, m >= n): returns (Q, R); A is left untouched."""
    import torch
    prec = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
    m, n = A.shape
    W = A.clone().contiguous()
    Q = torch.empty(m, n, dtype=A.dtype, device=A.device)
    nb = _lib.qrtebd_qr_workspace_size(prec, m, n)
    ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=A.device)
    check(_lib.qrtebd_householder_qr(prec, m, n, _ptr(W), n, _ptr(Q), n, _ptr(ws), ws.numel(),
                                     stream_handle(stream)), "householder_qr")
    return Q, torch.triu(W[:n])


def zgemm(precision, A, B, conj_a=False, conj_b=False, trans_a=False, trans_b=False,
          alpha=1.0, beta=0.0, C_out=None, stream=None):
    """C = alpha op(A) op(B) + beta C for 2-D torch CUDA tensors (row-major, contiguous)."""
    import torch
    prec = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
    m = A.shape[1] if trans_a else A.shape[0]
    k = A.shape[0] if trans_a else A.shape[1]
    n = B.shape[0] if trans_b else B.shape[1]
    sam, sak = (1, A.shape[1]) if trans_a else (A.shape[1], 1)
    sbk, sbn = (1, B.shape[1]) if trans_b else (B.shape[1], 1)
    if C_out is None:
        C_out = torch.zeros(m, n, dtype=A.dtype, device=A.device)
    ws = None
    nb = 0
    if prec in (C64_3XTF32, C64_TF32, C128_OZ):
        nb = _lib.qrtebd_zgemm_workspace_size(m, n, k)
        ws = torch.empty(nb, dtype=torch.uint8, device=A.device)
    al = (C.c_double * 2)(complex(alpha).real, complex(alpha).imag)
    be = (C.c_double * 2)(complex(beta).real, complex(beta).imag)
    check(_lib.qrtebd_zgemm(prec, m, n, k, _ptr(A), sam, sak, int(conj_a), _ptr(B), sbk, sbn,
                            int(conj_b), _ptr(C_out), C_out.shape[1], 1, al, be, _ptr(ws), nb,
                            stream_handle(stream)), "zgemm")
    return C_out


class MpsDesc(C.Structure):
    _fields_ = [("L", C.c_int), ("d", C.c_int), ("infinite", C.c_int), ("chi_max", C.c_int),
                ("precision", C.c_int), ("product_state", C.c_void_p)]


def _mps_sigs():
    P, I, D = C.c_void_p, C.c_int, C.c_double
    PP = C.POINTER(C.c_void_p)
    sig = {
        "qrtebd_mps_create": (I, [C.POINTER(MpsDesc), P, PP]),
        "qrtebd_mps_destroy": (I, [P]),
        "qrtebd_apply_gate_layer": (I, [P, I, C.POINTER(D), C.POINTER(Trunc), C.POINTER(D)]),
        "qrtebd_expectation": (I, [P, I, I, C.POINTER(D), C.POINTER(D)]),
        "qrtebd_truncation_error": (I, [P, I, C.POINTER(D)]),
        "qrtebd_schmidt": (I, [P, I, C.POINTER(D), I, C.POINTER(I)]),
        "qrtebd_entropy": (I, [P, I, C.POINTER(D)]),
        "qrtebd_bond_dims": (I, [P, C.POINTER(I), I, C.POINTER(I)]),
        "qrtebd_sync": (I, [P]),
        "qrtebd_mps_save": (I, [P, C.c_char_p]),
        "qrtebd_mps_load": (I, [C.c_char_p, P, PP]),
        "qrtebd_apply_gate_layer_batched": (I, [C.POINTER(C.c_void_p), I, I, C.POINTER(C.POINTER(D)),
                                                C.POINTER(Trunc), C.POINTER(C.POINTER(D))]),
        "qrtebd_mps_set_site": (I, [P, I, C.POINTER(D), I, I]),
        "qrtebd_mps_set_bond": (I, [P, I, C.POINTER(D), I, I]),
    }
    for name, (res, args) in sig.items():
        f = getattr(_lib, name)
        f.restype = res
        f.argtypes = args


_mps_sigs()


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class MPS:
    """Device-resident MPS (qrtebd_mps_*). Gates and operators are complex128 numpy arrays."""

    def __init__(self, L, d, chi_max, precision="c128", infinite=False, product_state=None,
                 stream=None, _handle=None):
        self.L, self.d, self.infinite = L, d, bool(infinite)
        self.stream = stream
        if _handle is not None:
            self.h = _handle
            return
        prec = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
        self._ps = None
        if product_state is not None:
            self._ps = np.ascontiguousarray(np.asarray(product_state, np.complex128).reshape(L, d))
        desc = MpsDesc(L, d, 1 if infinite else 0, chi_max, prec,
                       None if self._ps is None else self._ps.ctypes.data)
        h = C.c_void_p()
        check(_lib.qrtebd_mps_create(C.byref(desc), stream_handle(stream), C.byref(h)), "mps_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _lib.qrtebd_mps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nbonds(self):
        return self.L if self.infinite else self.L - 1

    def apply_layer(self, parity, gates, trunc, want_eps=False):
        g = np.ascontiguousarray(np.asarray(gates, np.complex128).reshape(self.nbonds, -1))
        eps = np.zeros(self.nbonds) if want_eps else None
        check(_lib.qrtebd_apply_gate_layer(self.h, parity, _dptr(g.view(np.float64)), C.byref(trunc),
                                           None if eps is None else _dptr(eps)), "apply_gate_layer")
        return eps

    def expectation(self, site, op):
        op = np.ascontiguousarray(np.asarray(op, np.complex128))
        ns = 1 if op.shape[0] == self.d else 2
        out = np.zeros(2)
        check(_lib.qrtebd_expectation(self.h, site, ns, _dptr(op.view(np.float64)), _dptr(out)),
              "expectation")
        return complex(out[0], out[1])

    def truncation_error(self, bond=-1):
        out = C.c_double(0)
        check(_lib.qrtebd_truncation_error(self.h, bond, C.byref(out)), "truncation_error")
        return out.value

    def bond_dims(self):
        buf = (C.c_int * (self.L + 1))()
        n = C.c_int(0)
        check(_lib.qrtebd_bond_dims(self.h, buf, self.L + 1, C.byref(n)), "bond_dims")
        return list(buf[: n.value])

    def schmidt(self, bond):
        cap = max(self.bond_dims())
        S = np.zeros(cap)
        n = C.c_int(0)
        check(_lib.qrtebd_schmidt(self.h, bond, _dptr(S), cap, C.byref(n)), "schmidt")
        return S[: n.value]

    def entropy(self, bond):
        out = C.c_double(0)
        check(_lib.qrtebd_entropy(self.h, bond, C.byref(out)), "entropy")
        return out.value

    def sync(self):
        check(_lib.qrtebd_sync(self.h), "sync")

    def set_site(self, site, B):
        """Load site tensor B (chi_l, d, chi_r) from host data."""
        B = np.ascontiguousarray(np.asarray(B, np.complex128))
        check(_lib.qrtebd_mps_set_site(self.h, site, _dptr(B.view(np.float64)), B.shape[0],
                                       B.shape[2]), "mps_set_site")

    def set_bond(self, bond, xi, diagonal=False):
        """Load bond matrix Xi (chi x chi, or its chi diagonal entries) from host data."""
        xi = np.ascontiguousarray(np.asarray(xi, np.complex128))
        chi = xi.shape[0]
        check(_lib.qrtebd_mps_set_bond(self.h, bond, _dptr(xi.view(np.float64)), chi,
                                       1 if diagonal else 0), "mps_set_bond")

    def save(self, path):
        check(_lib.qrtebd_mps_save(self.h, str(path).encode()), "mps_save")

    @classmethod
    def load(cls, path, stream=None):
        h = C.c_void_p()
        check(_lib.qrtebd_mps_load(str(path).encode(), stream_handle(stream), C.byref(h)), "mps_load")
        # shape information is read back through bond_dims
        import struct
        with open(path, "rb") as f:
            _, L, d, inf, _chi, _prec = struct.unpack("6i", f.read(24))
        obj = cls.__new__(cls)
        obj.h = h
        obj.stream = stream
        obj.L, obj.d, obj.infinite = L, d, bool(inf)
        return obj


def cbe_decompose(precision, Rz, stream=None):
    """Step (iv) of CBE for a square torch CUDA tensor Rz: returns (w, Vh, sweeps) with w the
    eigenvalues of Rz Rz^dag (descending, float64) and Vh its conjugated eigenvectors as
    rows (complex128), Rz Rz^dag = Vh^dag diag(w) Vh."""
    import torch
    prec = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
    n = Rz.shape[0]
    w = torch.empty(n, dtype=torch.float64, device=Rz.device)
    Vh = torch.empty(n, n, dtype=torch.complex128, device=Rz.device)
    nb = _lib.qrtebd_cbe_decompose_workspace_size(prec, n)
    ws = torch.empty(nb, dtype=torch.uint8, device=Rz.device)
    sw = torch.zeros(1, dtype=torch.int32, device=Rz.device)
    check(_lib.qrtebd_cbe_decompose(prec, n, _ptr_rows(Rz), Rz.stride(0), _ptr(w), _ptr(Vh), _ptr(ws), nb,
                                    _ptr(sw), stream_handle(stream)), "cbe_decompose")
    return w, Vh, sw


def autotune_bond(precision, chi_l, d, chi_m, chi_r, trunc, xi_kind=1, theta_given=False,
                  stream=None):
    """Tune the tensor-core launch configurations of one bond-update shape (synchronous);
    returns the number of product shapes newly tuned."""
    prec = PRECISIONS.get(precision, precision) if isinstance(precision, str) else precision
    n = C.c_int(0)
    check(_lib.qrtebd_autotune_bond(prec, chi_l, d, chi_m, chi_r, xi_kind, 1 if theta_given else 0,
                                    C.byref(trunc), stream_handle(stream), C.byref(n)),
          "autotune_bond")
    return n.value


def autotune_entries():
    """The autotuner's table: [{shape: (M, N, K, three), config: (bn, splits, tail),
    ms_tuned, ms_default}]."""
    out = []
    for i in range(_lib.qrtebd_autotune_count()):
        sh, cf, ms = (C.c_int * 4)(), (C.c_int * 3)(), (C.c_double * 2)()
        check(_lib.qrtebd_autotune_entry(i, sh, cf, ms), "autotune_entry")
        out.append({"shape": tuple(sh), "config": tuple(cf), "ms_tuned": ms[0], "ms_default": ms[1]})
    return out


def autotune_set(shape, config):
    """Insert or replace a table entry (e.g. one saved from autotune_entries)."""
    check(_lib.qrtebd_autotune_set((C.c_int * 4)(*shape), (C.c_int * 3)(*config)), "autotune_set")


def autotune_clear():
    _lib.qrtebd_autotune_clear()


def tc_operand_prep(mode):
    """Operand preparation of the complex64 tensor-core products: 1 (default) as a separate
    pass, 0 inside the GEMM kernel (128-column tiles); returns the previous mode."""
    prev = C.c_int(0)
    check(_lib.qrtebd_tc_operand_prep(int(mode), C.byref(prev)), "tc_operand_prep")
    return prev.value


def autotune_save(path):
    """Write the autotuner's table as JSON (shape, config, timings per entry)."""
    import json
    with open(path, "w") as f:
        json.dump(autotune_entries(), f)


def autotune_load(path):
    """Insert every entry of a table written by autotune_save; returns the entry count."""
    import json
    with open(path) as f:
        ents = json.load(f)
    for e in ents:
        autotune_set(tuple(e["shape"]), tuple(e["config"]))
    return len(ents)


def layer_workers():
    """Worker streams (and bond-update workspaces) of the batched-layer executor."""
    return int(_lib.qrtebd_layer_workers())


def clock_layer_gates(L, d, g, tau, infinite=False):
    """Gates of every bond (library clock-model builder), shape (nbonds, d^2, d^2)."""
    nb = L if infinite else L - 1
    out = np.zeros((nb, d * d, d * d), np.complex128)
    for b in range(nb):
        if infinite:
            wl = wr = 0.5
        else:
            wl = 1.0 if b == 0 else 0.5
            wr = 1.0 if b == L - 2 else 0.5
        out[b] = clock_bond_gate(d, g, wl, wr, tau)
    return out


def apply_layer_batched(states, parity, gates, trunc, want_eps=False):
    """One layer on several states at once (qrtebd_apply_gate_layer_batched)."""
    n = len(states)
    arrs = [np.ascontiguousarray(np.asarray(g, np.complex128).reshape(s.nbonds, -1)).view(np.float64)
            for s, g in zip(states, gates)]
    hs = (C.c_void_p * n)(*[s.h.value if isinstance(s.h, C.c_void_p) else s.h for s in states])
    gp = (C.POINTER(C.c_double) * n)(*[_dptr(a) for a in arrs])
    eps = [np.zeros(s.nbonds) for s in states] if want_eps else None
    ep = (C.POINTER(C.c_double) * n)(*[_dptr(e) for e in eps]) if want_eps else None
    check(_lib.qrtebd_apply_gate_layer_batched(hs, n, parity, gp, C.byref(trunc), ep),
          "apply_gate_layer_batched")
    return eps


def tebd_step_batched(states, halves, fulls, trunc):
    """Strang step on several states, each layer batched across them."""
    apply_layer_batched(states, 0, halves, trunc)
    apply_layer_batched(states, 1, fulls, trunc)
    apply_layer_batched(states, 0, halves, trunc)


def tebd_step(mps, half, full, trunc):
    """Strang step even(dt/2), odd(dt), even(dt/2) (Fig. 2a)."""
    mps.apply_layer(0, half, trunc)
    mps.apply_layer(1, full, trunc)
    mps.apply_layer(0, half, trunc)
