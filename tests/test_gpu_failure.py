"""Failure detection on the GPU, in the forms that leave the context usable: a bounded
wait that runs out (a barrier that nothing releases) and a NaN that reaches the FP64
norms are both reported by qrtebd_stream_check, the error word is cleared by that read,
and the next update on the same context matches the oracle. A checkpoint cut short by
one byte is refused, and the intact one reloads bit for bit."""
import numpy as np
import pytest

from oracle import bond
from paper_2212_09782_b300 import workloads as W
from tests.gpu_helpers import TOL, compare, rounded, run_gpu

pytestmark = pytest.mark.gpu


def _clean_update_matches_oracle(prec):
    from paper_2212_09782_b300 import lib as L
    dims = (24, 3, 24, 24)
    bd = W.random_bond(*dims, seed=4242, xi="dense")
    bd = {k: rounded(v, prec) if k != "U" else v for k, v in bd.items()}
    orc = bond.qr_update(bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], scheme="plain", chi_max=24)
    gpu = run_gpu(prec, bd["Xi"], bd["Bm"], bd["Bn"], bd["U"], L.trunc_default(L.PLAIN, 24))
    compare(gpu, orc, TOL[prec])


def test_barrier_wait_runs_out_and_is_reported():
    import torch
    from paper_2212_09782_b300 import lib as L
    L.stream_check()  # nothing pending
    L.set_spin_limit(1 << 12)
    try:
        L.selftest_barrier_timeout()
        with pytest.raises(L.QrtebdError) as e:
            L.stream_check()
        assert e.value.status == L.ERR_TIMEOUT
        L.stream_check()  # the read cleared the word
    finally:
        L.set_spin_limit(0)
    torch.cuda.synchronize()
    # the default limit is back: the fused QR updates' grid barriers complete as before
    for prec in ("c128", "c64_3xtf32"):
        _clean_update_matches_oracle(prec)
        L.stream_check()


@pytest.mark.parametrize("prec", ["c128", "c64_3xtf32"])
def test_nan_input_is_reported_as_numeric(prec):
    import torch
    from paper_2212_09782_b300 import lib as L
    r = W.rng(17)
    chi, d = 16, 3
    th = W.complex_gaussian(r, (chi, d, d, chi))
    th /= np.linalg.norm(th)
    th[3, 1, 2, 5] = np.nan
    U = W.random_unitary(r, d * d)
    Bn = W.random_right_isometry(r, chi, d, chi)
    with pytest.raises(L.QrtebdError) as e:
        run_gpu(prec, None, None, rounded(Bn, prec), U, L.trunc_default(L.PLAIN, chi),
                theta=rounded(th, prec))
    assert e.value.status == L.ERR_NUMERIC
    L.stream_check()  # cleared
    torch.cuda.synchronize()
    _clean_update_matches_oracle(prec)


def test_truncated_checkpoint_is_refused(tmp_path):
    from paper_2212_09782_b300 import lib as L
    L_sites, d, chi = 8, 3, 16
    s = L.MPS(L_sites, d, chi, precision="c128")
    gh = L.clock_layer_gates(L_sites, d, 1.5, 0.025, False)
    gf = L.clock_layer_gates(L_sites, d, 1.5, 0.05, False)
    tr = L.trunc_default(L.PLAIN, chi)
    for _ in range(3):
        L.tebd_step(s, gh, gf, tr)
    s.sync()
    path = tmp_path / "state.qrtebd"
    s.save(path)
    data = path.read_bytes()
    short = tmp_path / "short.qrtebd"
    short.write_bytes(data[:-1])
    with pytest.raises(L.QrtebdError) as e:
        L.MPS.load(short)
    assert e.value.status == L.ERR_INVALID_ARG and "truncated" in str(e.value)
    t = L.MPS.load(path)
    assert t.bond_dims() == s.bond_dims()
    for b in range(1, L_sites):
        assert np.array_equal(t.schmidt(b), s.schmidt(b))
        assert t.entropy(b) == s.entropy(b) and t.entropy(b) > 0
    assert t.truncation_error(-1) == s.truncation_error(-1)
    t.close()
    s.close()
