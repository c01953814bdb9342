"""The front ends on the GPU (through the C ABI): ht_reduce_general (the QZ
front end of Sec. 1, a QR of a general B before Algorithm 1) and the
zero-column preprocessing of Sec. 3.4.1 (ht_options.preprocess), against the
oracle's oracle/front.py elementwise (after fixing the sign freedom of the
reduction) and by the invariants against the input pencil."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import checks
from oracle import front
from paper_1710_08538_gb300 import pencils

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -52


@pytest.fixture(scope="module")
def ht():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_1710_08538_gb300 as m
    return m


def run(ht, A, B, general, **kw):
    n = A.shape[0]
    dA, dB = ht.colmajor(A), ht.colmajor(B)
    dQ, dZ = ht.colmajor(np.zeros((n, n))), ht.colmajor(np.zeros((n, n)))
    fn = ht.reduce_general if general else ht.reduce
    fn(dA, dB, dQ, dZ, opts=ht.options(**kw))
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in (dA, dB, dQ, dZ)]


def report(A, B, H, T, Q, Z):
    sh, st = checks.structure_violations(H, T)
    return {"sh": sh, "st": st, "oq": checks.orthogonality(Q), "oz": checks.orthogonality(Z),
            "ba": np.linalg.norm(Q @ H @ Z.T - A) / np.linalg.norm(A),
            "bb": np.linalg.norm(Q @ T @ Z.T - B) / np.linalg.norm(B)}


def assert_close(ref, got, tol=1e-10):
    ref = checks.sign_normalize(*ref)
    got = checks.sign_normalize(*got)
    for name, a, b in zip("HTQZ", ref, got):
        err = float(np.max(np.abs(a - b)))
        assert err <= tol * max(1.0, float(np.max(np.abs(a)))), (name, err)


@pytest.mark.parametrize("n,nb", [(40, 8), (130, 32)])
def test_general_vs_oracle(ht, n, nb):
    rng = np.random.default_rng(3000 + n)
    A, B = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    got = run(ht, A, B, True, nb=nb)
    assert_close(front.general(A, B, nb=nb), got)


@pytest.mark.parametrize("prec", ["fp64", "emu"])
def test_general_invariants(ht, prec):
    n = 700
    rng = np.random.default_rng(3700)
    A, B = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    p = ht.HT_PREC_FP64 if prec == "fp64" else ht.HT_PREC_EMU
    H, T, Q, Z = run(ht, A, B, True, precision=p)
    r = report(A, B, H, T, Q, Z)
    tol = 20 * n * EPS
    assert r["sh"] == 0 and r["st"] == 0, r
    assert max(r["oq"], r["oz"]) <= tol, r
    assert max(r["ba"], r["bb"]) <= (tol if prec == "fp64" else 1e-12), r


def _triu_with_zero_columns(n, cols, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    B = np.triu(rng.standard_normal((n, n))) + 3 * np.eye(n)
    B[:, cols] = 0.0
    return A, B


def test_preprocess_vs_oracle(ht):
    A, B = _triu_with_zero_columns(150, [0, 7, 8, 40, 41, 42, 99, 149], 17)
    H, T, Q, Z = run(ht, A, B, False, nb=16, preprocess=1)
    ref = front.preprocess(A, B, nb=16)
    assert ref[4] == 8
    assert_close(ref[:4], (H, T, Q, Z))


@pytest.mark.parametrize("n", [40, 300])
def test_preprocess_saddle_point(ht, n):
    """Test Suite 4's shape: B = diag(I, 0) has n/4 zero columns; they are
    deflated as infinite eigenvalues in generalized Schur form, and the rest
    is a valid HT reduction of the input pencil."""
    A, B = pencils.saddle_point(n, 11 + n)
    B = np.triu(B)
    l = len(front.zero_columns(B))
    H, T, Q, Z = run(ht, A, B, False, nb=32, preprocess=1)
    r = report(A, B, H, T, Q, Z)
    tol = 20 * n * EPS
    assert r["sh"] == 0 and r["st"] == 0, r
    assert max(r["oq"], r["oz"], r["ba"], r["bb"]) <= tol, r
    assert not np.any(T[:, :l])
    assert not np.any(np.tril(H[:, :l], -1))
    # no elementwise comparison here: a saddle-point pencil has 2l infinite
    # eigenvalues (Jordan blocks of size 2) and the preprocessing deflates l of
    # them, so the trailing B is singular and its reduction not unique


def test_general_rejects_preprocess(ht):
    n = 10
    A, B = np.eye(n), np.eye(n)
    dA, dB = ht.colmajor(A), ht.colmajor(B)
    dQ, dZ = ht.colmajor(np.zeros((n, n))), ht.colmajor(np.zeros((n, n)))
    with pytest.raises(Exception):
        ht.reduce_general(dA, dB, dQ, dZ, opts=ht.options(preprocess=1))
