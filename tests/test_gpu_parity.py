"""Parity of the CUDA library (through the C ABI) with the CPU oracle.

Elementwise: the GPU result equals Algorithm 1 of the oracle run with the
same panel width, and Algorithm 2 / the Givens reduction, after fixing the
diagonal sign freedom (they agree up to rounding, see checks.sign_normalize).
Invariants: structure (exact zeros), orthogonality and backward errors
<= 20 n eps on every workload of the paper's shape, the edge cases (n <= 2,
n = 3, k not dividing n - j, forced early absorption, singular B) and the
sizes of the benchmark configurations.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import checks
from oracle import househt as hh
from paper_1710_08538_gb300 import pencils

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ht():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_1710_08538_gb300 as m
    return m


def run_gpu(ht, A, B, nb=32, want_qz=True, **kw):
    n = A.shape[0]
    dA, dB = ht.colmajor(A), ht.colmajor(B)
    dQ = ht.colmajor(np.zeros((n, n))) if want_qz else None
    dZ = ht.colmajor(np.zeros((n, n))) if want_qz else None
    st = ht.reduce(dA, dB, dQ, dZ, want_qz=want_qz, opts=ht.options(nb=nb, **kw), with_stats=True)
    torch.cuda.synchronize()
    out = [dA.cpu().numpy(), dB.cpu().numpy()]
    if want_qz:
        out += [dQ.cpu().numpy(), dZ.cpu().numpy()]
    return out, st


def test_smoke(ht):
    import __graft_entry__ as g
    g.smoke()


@pytest.mark.parametrize("n,nb", [(20, 4), (37, 5), (64, 16), (100, 32), (130, 64)])
def test_elementwise_vs_algorithm1(ht, n, nb):
    A, B = pencils.random_qr(n, 500 + n)
    (H, T, Q, Z), _ = run_gpu(ht, A, B, nb=nb)
    ref = checks.sign_normalize(*hh.househt(A, B, nb=nb)[:4])
    got = checks.sign_normalize(H, T, Q, Z)
    for name, a, b in zip("HTQZ", ref, got):
        err = float(np.max(np.abs(a - b)))
        assert err <= 1e-10 * max(1.0, float(np.max(np.abs(a)))), (name, err)


def test_elementwise_vs_algorithm2_and_givens(ht):
    n = 48
    A, B = pencils.random_qr(n, 4848)
    (H, T, Q, Z), _ = run_gpu(ht, A, B, nb=8)
    got = checks.sign_normalize(H, T, Q, Z)
    for ref in (oracle.basic_househt(A, B)[:4], oracle.givens_ht(A, B)):
        ref = checks.sign_normalize(*ref)
        for a, b in zip(ref, got):
            assert float(np.max(np.abs(a - b))) <= 1e-10


@pytest.mark.parametrize("kind", list(pencils.WORKLOADS))
@pytest.mark.parametrize("n,nb", [(3, 1), (4, 2), (5, 2), (9, 4), (33, 8), (66, 16), (129, 32), (200, 64)])
def test_invariants_workloads(ht, kind, n, nb):
    A, B = pencils.make(kind, n, 77 + n)
    (H, T, Q, Z), st = run_gpu(ht, A, B, nb=nb)
    checks.assert_invariants(A, B, H, T, Q, Z)
    if kind == "saddle_point" and n >= 4:
        assert st["perturbed_pivots"] > 0


@pytest.mark.parametrize("n", [0, 1, 2])
def test_tiny_n(ht, n):
    A, B = pencils.random_qr(n, 3)
    if n > 0:
        B = B + np.tril(np.ones((n, n)), -1)  # junk below the diagonal must be ignored and zeroed
    (H, T, Q, Z), _ = run_gpu(ht, A, B) if n > 0 else ((A, B, np.eye(0), np.eye(0)), None)
    assert np.array_equal(H, A) and np.array_equal(T, np.triu(B))
    assert np.array_equal(Q, np.eye(n)) and np.array_equal(Z, np.eye(n))


def test_lower_part_of_B_is_ignored(ht):
    n = 40
    A, B = pencils.random_qr(n, 40)
    junk = B + np.tril(np.full((n, n), 7.0), -1)
    (H, T, Q, Z), _ = run_gpu(ht, A, junk, nb=8)
    checks.assert_invariants(A, B, H, T, Q, Z)


def test_without_qz(ht):
    n = 70
    A, B = pencils.random_qr(n, 70)
    (H, T), _ = run_gpu(ht, A, B, nb=16, want_qz=False)
    (H2, T2, Q, Z), _ = run_gpu(ht, A, B, nb=16, want_qz=True)
    assert np.array_equal(H, H2) and np.array_equal(T, T2)


def test_forced_early_absorption(ht):
    """IR tolerance 0: every solve with k >= 1 fails after max_ir corrections,
    so each panel ends after one column (undo + early absorption)."""
    n = 60
    A, B = pencils.random_qr(n, 61)
    (H, T, Q, Z), st = run_gpu(ht, A, B, nb=8, ir_tol_scale=-1.0, max_ir=2)
    assert st["early_absorptions"] >= n // 3
    checks.assert_invariants(A, B, H, T, Q, Z)
    ref = checks.sign_normalize(*hh.househt(A, B, nb=8, ir_tol_scale=0.0, max_ir=2)[:4])
    got = checks.sign_normalize(H, T, Q, Z)
    for a, b in zip(ref, got):
        assert float(np.max(np.abs(a - b))) <= 1e-10


def test_idempotent(ht):
    n = 50
    rng = np.random.default_rng(5)
    A = np.triu(rng.standard_normal((n, n)), -1)
    B = np.triu(rng.standard_normal((n, n))) + 3 * np.eye(n)
    (H, T, Q, Z), _ = run_gpu(ht, A, B, nb=8)
    assert np.array_equal(Q, np.eye(n)) and np.array_equal(Z, np.eye(n))
    assert np.array_equal(H, A) and np.array_equal(T, B)


def test_nonfinite_input_rejected(ht):
    n = 16
    A, B = pencils.random_qr(n, 16)
    A[3, 4] = np.nan
    with pytest.raises(ht.HtError) as e:
        run_gpu(ht, A, B, nb=4)
    assert e.value.code == ht.HT_ERR_NONFINITE


def test_config1_n256_eigenvalues(ht):
    """n = 256 random pencil (Test Suite 1 shape): invariants and generalized
    eigenvalues against LAPACK dggev."""
    import scipy.linalg as sla
    from scipy.optimize import linear_sum_assignment
    n = 256
    A, B = pencils.random_qr(n, 1000)
    (H, T, Q, Z), st = run_gpu(ht, A, B, nb=32)
    checks.assert_invariants(A, B, H, T, Q, Z)
    ev = sla.eigvals(A, B)
    eh = sla.eigvals(H, T)
    C = np.abs(ev[:, None] - eh[None, :]) / (1 + np.abs(ev[:, None]))
    i, j = linear_sum_assignment(C)
    assert np.max(C[i, j]) <= 1e-8


def test_config2_n4096_near_infinite(ht):
    """n = 4096, 10% of B's diagonal 1e-12: IR is needed on many columns;
    invariants in FP64 on the GPU."""
    from paper_1710_08538_gb300 import check
    n = 4096
    A, B = pencils.near_infinite(n, 2000)
    dA, dB = ht.colmajor(A), ht.colmajor(B)
    A0, B0 = dA.clone(), dB.clone()
    dQ, dZ = torch.empty_like(dA), torch.empty_like(dA)
    st = ht.reduce(dA, dB, dQ, dZ, opts=ht.options(nb=32), with_stats=True)
    rep = check.invariants(A0, B0, dA, dB, dQ, dZ)
    assert check.passes(rep), rep
    assert st["cols_with_ir"] > 0


def test_batched_matches_single(ht):
    sizes = [5, 40, 17, 64, 3, 100]
    As, Bs, Qs, Zs, refs = [], [], [], [], []
    for i, n in enumerate(sizes):
        A, B = pencils.random_qr(n, 900 + i)
        refs.append((A, B))
        As.append(ht.colmajor(A)); Bs.append(ht.colmajor(B))
        Qs.append(ht.colmajor(np.zeros((n, n)))); Zs.append(ht.colmajor(np.zeros((n, n))))
    ht.reduce_batched(As, Bs, Qs, Zs)
    torch.cuda.synchronize()
    for (A, B), dA, dB, dQ, dZ in zip(refs, As, Bs, Qs, Zs):
        checks.assert_invariants(A, B, dA.cpu().numpy(), dB.cpu().numpy(), dQ.cpu().numpy(), dZ.cpu().numpy())


def test_batched_lanes_match_single_calls(ht):
    """Twelve pencils of uneven order (up to 700) in one ht_reduce_batched
    call.  The batch runs on concurrent lanes (host threads with streams of
    their own, each launch whose CTAs wait on one another capped at a share of
    the SMs: the panel then takes the grid-synchronous solve), and gives the
    results of one ht_reduce call per pencil, elementwise after sign
    normalisation, and the invariants."""
    sizes = [700, 3, 129, 450, 64, 257, 333, 96, 511, 5, 200, 640]
    As, Bs, Qs, Zs, refs = [], [], [], [], []
    for i, n in enumerate(sizes):
        A, B = pencils.random_qr(n, 1900 + i)
        refs.append((A, B))
        As.append(ht.colmajor(A)); Bs.append(ht.colmajor(B))
        Qs.append(ht.colmajor(np.zeros((n, n)))); Zs.append(ht.colmajor(np.zeros((n, n))))
    ht.reduce_batched(As, Bs, Qs, Zs)
    torch.cuda.synchronize()
    for (A, B), dA, dB, dQ, dZ in zip(refs, As, Bs, Qs, Zs):
        got = [x.cpu().numpy() for x in (dA, dB, dQ, dZ)]
        checks.assert_invariants(A, B, *got)
        n = A.shape[0]
        if n <= 2:
            continue
        sA, sB = ht.colmajor(A), ht.colmajor(B)
        sQ, sZ = ht.colmajor(np.zeros((n, n))), ht.colmajor(np.zeros((n, n)))
        ht.reduce(sA, sB, sQ, sZ)
        torch.cuda.synchronize()
        ref = checks.sign_normalize(*[x.cpu().numpy() for x in (sA, sB, sQ, sZ)])
        gotn = checks.sign_normalize(*got)
        for name, a, b in zip("HTQZ", ref, gotn):
            err = float(np.max(np.abs(a - b)))
            assert err <= 1e-10 * max(1.0, float(np.max(np.abs(a)))), (n, name, err)


def test_batched_device_pointer_arrays(ht):
    """ht_reduce_batched with its pointer arrays in device memory (the
    cuBLAS-batched convention) gives the results of host pointer arrays."""
    sizes = [150, 7, 90]
    out = []
    for dev_arrays in (False, True):
        As, Bs, Qs, Zs = [], [], [], []
        for i, n in enumerate(sizes):
            A, B = pencils.random_qr(n, 2500 + i)
            As.append(ht.colmajor(A)); Bs.append(ht.colmajor(B))
            Qs.append(ht.colmajor(np.zeros((n, n)))); Zs.append(ht.colmajor(np.zeros((n, n))))
        n_arr = (ctypes.c_int * 3)(*sizes)
        ld = (ctypes.c_int * 3)(*sizes)
        ptrs = [[x.data_ptr() for x in L] for L in (As, Bs, Qs, Zs)]
        if dev_arrays:
            keep = [torch.tensor(p, dtype=torch.int64, device="cuda") for p in ptrs]
            args = [ctypes.cast(ctypes.c_void_p(t.data_ptr()), ctypes.POINTER(ctypes.c_void_p)) for t in keep]
        else:
            args = [(ctypes.c_void_p * 3)(*p) for p in ptrs]
        torch.cuda.synchronize()
        rc = ht.lib().ht_reduce_batched(3, n_arr, args[0], ld, args[1], ld, args[2], args[3], 1, None)
        assert rc == 0
        torch.cuda.synchronize()
        out.append([[x.cpu().numpy() for x in L] for L in (As, Bs, Qs, Zs)])
    for L0, L1 in zip(out[0], out[1]):
        for a, b in zip(L0, L1):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", ["fp64", "emu"])
def test_elementwise_vs_algorithm1_three_solve_blocks(ht, prec):
    """n = 600: the trailing system has up to 599 rows, so the look-ahead
    solve runs a chain of three 256-row diagonal blocks (block inverses, far
    updates one step behind, progress words) and the restores span several
    stripes; the result still equals the oracle's Algorithm 1 elementwise."""
    n, nb = 600, 32
    A, B = pencils.random_qr(n, 1600)
    p = ht.HT_PREC_FP64 if prec == "fp64" else ht.HT_PREC_EMU
    (H, T, Q, Z), _ = run_gpu(ht, A, B, nb=nb, precision=p)
    ref = checks.sign_normalize(*hh.househt(A, B, nb=nb)[:4])
    got = checks.sign_normalize(H, T, Q, Z)
    for name, a, b in zip("HTQZ", ref, got):
        err = float(np.max(np.abs(a - b)))
        assert err <= 1e-10 * max(1.0, float(np.max(np.abs(a)))), (name, err)


def test_bounded_wait_times_out_and_library_recovers(ht):
    """A bounded device wait that runs out: with the test option wait_polls = 1
    the cross-CTA waits of the look-ahead solve and of the restore chains give
    up almost at once, the kernels raise HT_ERR_TIMEOUT in the error word, keep
    joining their grid barriers and return; the call reports the error, the
    device status word agrees, and the next call on the same workspace
    succeeds."""
    n = 600
    A, B = pencils.random_qr(n, 1601)
    with pytest.raises(ht.HtError) as e:
        run_gpu(ht, A, B, nb=32, wait_polls=1)
    assert e.value.code == ht.HT_ERR_TIMEOUT
    status = ctypes.c_int(-1)
    assert ht.lib().ht_last_device_status(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                          ctypes.byref(status)) == ht.HT_OK
    assert status.value == ht.HT_ERR_TIMEOUT
    (H, T, Q, Z), _ = run_gpu(ht, A, B, nb=32)
    checks.assert_invariants(A, B, H, T, Q, Z)
    assert ht.lib().ht_last_device_status(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                          ctypes.byref(status)) == ht.HT_OK
    assert status.value == ht.HT_OK


def test_device_philox_known_answers(ht):
    """The device generator of the Remark 2.2 perturbation reproduces the
    published Philox4x32-10 known-answer vectors (tests/golden)."""
    import os
    rows = []
    for ln in open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")):
        ln = ln.split("#")[0].split()
        if ln:
            w = [int(x, 16) for x in ln]
            rows.append((w[0:4], w[4:6], w[6:10]))
    got = ht.philox4x32_10([(c, k) for c, k, _ in rows])
    assert got == [o for _, _, o in rows]
