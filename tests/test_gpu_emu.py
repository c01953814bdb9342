"""The emulated-FP64 path (precision HT_PREC_EMU): the chain applications of
the absorption (Sec. 3.3) run as exact digit products on the tensor cores.

Parity is held to the same bars as the FP64 path: elementwise against
Algorithm 1 of the oracle after the sign normalisation, and the invariants
(exact zeros, orthogonality <= 20 n eps, relative backward errors <= 1e-12,
the bound stated for the emulated path) on every workload shape, including
the graded pencils whose entries span 16 decades.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import checks
from oracle import househt as hh
from paper_1710_08538_gb300 import pencils

pytestmark = pytest.mark.gpu

EMU_BWD = 1e-12


@pytest.fixture(scope="module")
def ht():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_1710_08538_gb300 as m
    return m


def run(ht, A, B, nb=32, prec=None, want_qz=True, **kw):
    n = A.shape[0]
    prec = ht.HT_PREC_EMU if prec is None else prec
    dA, dB = ht.colmajor(A), ht.colmajor(B)
    dQ = ht.colmajor(np.zeros((n, n))) if want_qz else None
    dZ = ht.colmajor(np.zeros((n, n))) if want_qz else None
    st = ht.reduce(dA, dB, dQ, dZ, want_qz=want_qz, opts=ht.options(nb=nb, precision=prec, **kw), with_stats=True)
    torch.cuda.synchronize()
    out = [dA.cpu().numpy(), dB.cpu().numpy()]
    if want_qz:
        out += [dQ.cpu().numpy(), dZ.cpu().numpy()]
    return out, st


@pytest.mark.parametrize("n,nb", [(40, 8), (64, 16), (100, 32), (161, 20)])
def test_emu_elementwise_vs_algorithm1(ht, n, nb):
    A, B = pencils.random_qr(n, 700 + n)
    (H, T, Q, Z), _ = run(ht, A, B, nb=nb)
    ref = checks.sign_normalize(*hh.househt(A, B, nb=nb)[:4])
    got = checks.sign_normalize(H, T, Q, Z)
    for name, a, b in zip("HTQZ", ref, got):
        err = float(np.max(np.abs(a - b)))
        assert err <= 1e-10 * max(1.0, float(np.max(np.abs(a)))), (name, err)


@pytest.mark.parametrize("kind", list(pencils.WORKLOADS))
@pytest.mark.parametrize("n,nb", [(5, 2), (33, 8), (66, 16), (129, 32), (300, 32), (517, 24)])
def test_emu_invariants_workloads(ht, kind, n, nb):
    A, B = pencils.make(kind, n, 31 * n + nb)
    (H, T, Q, Z), _ = run(ht, A, B, nb=nb)
    checks.assert_invariants(A, B, H, T, Q, Z, bwd_tol=EMU_BWD)


def test_emu_matches_fp64_path(ht):
    n = 400
    A, B = pencils.shifted_triu(n, 4000)
    got_e, _ = run(ht, A, B)
    got_f, _ = run(ht, A, B, prec=ht.HT_PREC_FP64)
    for a, b in zip(checks.sign_normalize(*got_f), checks.sign_normalize(*got_e)):
        assert float(np.max(np.abs(a - b))) <= 1e-10


def test_emu_without_qz_and_early_absorption(ht):
    n = 150
    A, B = pencils.near_infinite(n, 77)
    (H, T), st = run(ht, A, B, nb=32, want_qz=False)
    assert checks.structure_violations(H, T) == (0, 0)
    (H, T, Q, Z), st = run(ht, A, B, nb=32, max_ir=1, ir_tol_scale=1e-300)
    assert st["early_absorptions"] > 0
    checks.assert_invariants(A, B, H, T, Q, Z, bwd_tol=EMU_BWD)


def test_emu_config5_graded_n1024(ht):
    """Graded pencil (entries over 16 decades), the workload on which the
    emulated path's per-line scaling matters; invariants in FP64 on the GPU."""
    from paper_1710_08538_gb300 import check
    n = 1024
    A, B = pencils.graded(n, 5000)
    dA, dB = ht.colmajor(A), ht.colmajor(B)
    A0, B0 = dA.clone(), dB.clone()
    dQ, dZ = torch.empty_like(dA), torch.empty_like(dA)
    ht.reduce(dA, dB, dQ, dZ, opts=ht.options(nb=32, precision=ht.HT_PREC_EMU))
    rep = check.invariants(A0, B0, dA, dB, dQ, dZ)
    assert check.passes(rep, bwd_tol=EMU_BWD), rep


def test_emu_config5_graded_full_size(ht):
    """Config 5 at its own size: the graded pencil of order 8192 on the
    emulated path, with the a-posteriori check on (probe estimates within the
    stated 1e-12, no fallback) and 16-probe invariants in FP64 on the GPU."""
    from paper_1710_08538_gb300 import check
    n = 8192
    A, B = pencils.graded(n, 8192)
    dA, dB = ht.colmajor(A), ht.colmajor(B)
    del A, B
    A0, B0 = dA.clone(), dB.clone()
    dQ, dZ = torch.empty_like(dA), torch.empty_like(dA)
    st = ht.reduce(dA, dB, dQ, dZ, opts=ht.options(nb=32, precision=ht.HT_PREC_EMU, emu_check=1), with_stats=True)
    assert st["emu_fallback"] == 0 and max(st["emu_bwd_est"]) <= EMU_BWD, st["emu_bwd_est"]
    rep = check.invariants(A0, B0, dA, dB, dQ, dZ, probes=16, seed=3)
    assert check.passes(rep, bwd_tol=EMU_BWD), rep


def test_emu_config3_shape_n2048(ht):
    from paper_1710_08538_gb300 import check
    n = 2048
    A, B = pencils.shifted_triu(n, 3000)
    dA, dB = ht.colmajor(A), ht.colmajor(B)
    A0, B0 = dA.clone(), dB.clone()
    dQ, dZ = torch.empty_like(dA), torch.empty_like(dA)
    ht.reduce(dA, dB, dQ, dZ, opts=ht.options(nb=32, precision=ht.HT_PREC_EMU))
    rep = check.invariants(A0, B0, dA, dB, dQ, dZ)
    assert check.passes(rep, bwd_tol=EMU_BWD), rep


def test_emu_unsupported_options(ht):
    A, B = pencils.random_qr(40, 1)
    with pytest.raises(ht.HtError) as e:
        run(ht, A, B, nb=48)
    assert e.value.code == ht.HT_ERR_NOT_IMPLEMENTED
    with pytest.raises(ht.HtError) as e:
        run(ht, A, B, nb=16, emu_slices=5)
    assert e.value.code == ht.HT_ERR_NOT_IMPLEMENTED


@pytest.mark.parametrize("mode", [1, 2])
def test_emu_check_and_fallback(ht, mode):
    """ht_options.emu_check: mode 1 reports probe estimates of the backward
    errors and keeps the emulated result when they hold the stated 1e-12;
    mode 2 treats the check as failed and redoes the reduction in FP64 from
    the saved pencil, which then equals an FP64 call bit for bit."""
    n = 300
    A, B = pencils.random_qr(n, 4300)
    dA, dB = ht.colmajor(A), ht.colmajor(B)
    dQ, dZ = ht.colmajor(np.zeros((n, n))), ht.colmajor(np.zeros((n, n)))
    st = ht.reduce(dA, dB, dQ, dZ, opts=ht.options(precision=ht.HT_PREC_EMU, emu_check=mode), with_stats=True)
    torch.cuda.synchronize()
    got = [x.cpu().numpy() for x in (dA, dB, dQ, dZ)]
    checks.assert_invariants(A, B, *got, bwd_tol=1e-12)
    ea, eb = st["emu_bwd_est"]
    rep = checks.invariant_report(A, B, *got)
    assert 0.0 < ea <= 1e-12 and 0.0 < eb <= 1e-12, (ea, eb)
    # the probe estimate is within a small factor of the true Frobenius-norm error
    assert ea <= 5 * rep["bwd_a"] + 1e-16 and rep["bwd_a"] <= 5 * ea + 1e-16, (ea, rep["bwd_a"])
    if mode == 1:
        assert st["emu_fallback"] == 0
    else:
        assert st["emu_fallback"] == 1
        fA, fB = ht.colmajor(A), ht.colmajor(B)
        fQ, fZ = ht.colmajor(np.zeros((n, n))), ht.colmajor(np.zeros((n, n)))
        ht.reduce(fA, fB, fQ, fZ, opts=ht.options(precision=ht.HT_PREC_FP64))
        torch.cuda.synchronize()
        for a, b in zip((fA, fB, fQ, fZ), got):
            assert np.array_equal(a.cpu().numpy(), b)
