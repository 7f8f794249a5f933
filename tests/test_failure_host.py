"""Failure detection on the host (no GPU): refusals the library makes before it touches
the device. A workspace one byte short of qrtebd_bond_workspace_size is refused with OOM
before any launch; a checkpoint that is truncated, padded, mislabelled or carries a bond
dimension the state cannot hold is refused with INVALID_ARG before any device memory is
taken."""
import ctypes as C
import struct

import pytest


@pytest.fixture(scope="module")
def L():
    from paper_2212_09782_b300 import lib
    return lib


def _io(L, prec, chi_l, d, chi_m, chi_r, ws_bytes):
    io = L.BondIO()
    io.precision = prec
    io.chi_l, io.d, io.chi_m, io.chi_r = chi_l, d, chi_m, chi_r
    io.xi_kind = 0
    # addresses that are never dereferenced: the refusal comes before any device work
    fake = 1 << 40
    io.bn, io.theta, io.gate = fake, fake + 4096, fake + 8192
    io.bm_out, io.xi_out, io.bn_out = fake + 12288, fake + 16384, fake + 20480
    io.workspace = fake + 24576
    io.workspace_bytes = ws_bytes
    return io


@pytest.mark.parametrize("prec", ["c128", "c64_3xtf32", "c64_fp32"])
@pytest.mark.parametrize("scheme", ["plain", "cbe"])
def test_workspace_one_byte_short_is_oom(L, prec, scheme):
    p = L.PRECISIONS[prec]
    chi_l, d, chi_m, chi_r = 40, 3, 40, 40
    tr = L.trunc_default(L.PLAIN if scheme == "plain" else L.CBE, 40)
    need = L.bond_workspace_size(p, chi_l, d, chi_m, chi_r, tr, xi_kind=0, theta_given=True)
    io = _io(L, p, chi_l, d, chi_m, chi_r, need - 1)
    info = L.BondInfo()
    st = L.raw().qrtebd_bond_update(C.byref(io), C.byref(tr), None, C.byref(info))
    assert st == L.ERR_OOM
    assert b"workspace too small" in L.raw().qrtebd_last_error_message()


def test_bad_arguments_are_refused(L):
    tr = L.trunc_default(L.PLAIN, 8)
    info = L.BondInfo()
    assert L.raw().qrtebd_bond_update(None, C.byref(tr), None, C.byref(info)) == L.ERR_INVALID_ARG
    io = _io(L, L.C128, 8, 2, 8, 8, 1 << 30)
    io.gate = None
    assert L.raw().qrtebd_bond_update(C.byref(io), C.byref(tr), None, C.byref(info)) == L.ERR_INVALID_ARG
    io = _io(L, 9, 8, 2, 8, 8, 1 << 30)  # no such precision
    assert L.raw().qrtebd_bond_update(C.byref(io), C.byref(tr), None, C.byref(info)) == L.ERR_INVALID_ARG


MAGIC = 0x51525442


def _checkpoint_bytes(L_sites=4, d=2, chi=(1, 2, 4, 2, 1), prec=0, chi_max=4, magic=MAGIC, extra=0,
                      short=0):
    """A checkpoint in the library's layout: header, bond dimensions, diagonal flags, site
    tensors, bond matrices with their diagonals, accumulated eps (finite chain)."""
    esz = 16 if prec == 0 else 8
    nb = L_sites + 1
    out = struct.pack("6i", magic, L_sites, d, 0, chi_max, prec)
    out += struct.pack(f"{nb}i", *chi) + bytes([1] * nb)
    body = sum(chi[m] * d * chi[m + 1] for m in range(L_sites)) * esz
    body += sum(c * c + c for c in chi) * esz + nb * 8
    out += bytes(body + extra)
    return out[: len(out) - short] if short else out


@pytest.mark.parametrize("case", ["truncated", "padded", "magic", "chi", "header"])
def test_bad_checkpoint_is_refused_before_allocation(L, tmp_path, case):
    kw = {"truncated": dict(short=1), "padded": dict(extra=1), "magic": dict(magic=0x1234),
          "chi": dict(chi=(1, 2, 5, 2, 1)), "header": dict(d=1)}[case]
    path = tmp_path / "state.qrtebd"
    path.write_bytes(_checkpoint_bytes(**kw))
    h = C.c_void_p()
    st = L.raw().qrtebd_mps_load(str(path).encode(), None, C.byref(h))
    assert st == L.ERR_INVALID_ARG and not h.value
    msg = L.raw().qrtebd_last_error_message().decode()
    want = {"truncated": "truncated", "padded": "truncated", "magic": "not a qrtebd checkpoint",
            "chi": "out of range", "header": "corrupt header"}[case]
    assert want in msg, msg


def test_missing_checkpoint_is_refused(L, tmp_path):
    h = C.c_void_p()
    st = L.raw().qrtebd_mps_load(str(tmp_path / "absent").encode(), None, C.byref(h))
    assert st == L.ERR_INVALID_ARG and not h.value


def test_sweeps_out_of_range_is_refused(L):
    nb = C.c_size_t(0)
    for k in (-1, 1001):
        t = L.trunc_default(L.PLAIN, 8, sweeps=k)
        st = L.raw().qrtebd_bond_workspace_size(L.C64_3XTF32, 8, 2, 8, 8, 1, 0, C.byref(t), C.byref(nb))
        assert st == L.ERR_INVALID_ARG
    t = L.trunc_default(L.PLAIN, 8)
    assert t.sweeps == 1


def test_xi_kinds_on_the_host(L):
    # xi_kind 3 (a lower-triangular Xi with its zeros stored) takes the dense kind's workspace;
    # kinds outside 0..3 are refused before any device work
    t = L.trunc_default(L.PLAIN, 40)
    for prec in ("c128", "c64_3xtf32"):
        p = L.PRECISIONS[prec]
        dense = L.bond_workspace_size(p, 40, 3, 40, 40, t, xi_kind=1)
        assert L.bond_workspace_size(p, 40, 3, 40, 40, t, xi_kind=3) == dense
    nb = C.c_size_t(0)
    for k in (-1, 4):
        st = L.raw().qrtebd_bond_workspace_size(L.C64_3XTF32, 40, 3, 40, 40, k, 0, C.byref(t), C.byref(nb))
        assert st == L.ERR_INVALID_ARG
    io = _io(L, L.C64_3XTF32, 40, 3, 40, 40, 1 << 30)
    io.xi_kind = 4
    info = L.BondInfo()
    assert L.raw().qrtebd_bond_update(C.byref(io), C.byref(t), None, C.byref(info)) == L.ERR_INVALID_ARG
