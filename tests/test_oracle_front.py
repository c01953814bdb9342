"""Pins of the oracle's QZ front end (Sec. 1) and zero-column preprocessing
(Sec. 3.4.1), oracle/front.py: structure, orthogonality and backward errors
against the input pencil, and the generalized eigenvalues against LAPACK
(scipy.linalg.eigvals), including the l infinite eigenvalues the
preprocessing deflates."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import checks
from oracle import front
from paper_1710_08538_gb300 import pencils

EPS = 2.0 ** -52


def report(A, B, H, T, Q, Z):
    """Invariants against the full B (not its upper triangle)."""
    n = A.shape[0]
    sh, st = checks.structure_violations(H, T)
    return {"sh": sh, "st": st, "oq": checks.orthogonality(Q), "oz": checks.orthogonality(Z),
            "ba": np.linalg.norm(Q @ H @ Z.T - A) / np.linalg.norm(A),
            "bb": np.linalg.norm(Q @ T @ Z.T - B) / np.linalg.norm(B), "tol": 20 * n * EPS}


def finite_eigs(A, B):
    w = sla.eigvals(A, B)
    return w[np.isfinite(w) & (np.abs(w) < 1e8)]


def assert_same_eigs(a, b, tol):
    """Each eigenvalue of a matched to the nearest unused one of b."""
    a, b = list(a), list(b)
    assert len(a) == len(b), (len(a), len(b))
    for w in a:
        i = int(np.argmin([abs(w - z) for z in b]))
        assert abs(w - b[i]) <= tol * max(1.0, abs(w)), (w, b[i])
        b.pop(i)


@pytest.mark.parametrize("n", [3, 6, 13, 30])
def test_general_front_end(n):
    rng = np.random.default_rng(40 + n)
    A, B = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    H, T, Q, Z = front.general(A, B, nb=4)
    r = report(A, B, H, T, Q, Z)
    assert r["sh"] == 0 and r["st"] == 0, r
    assert max(r["oq"], r["oz"], r["ba"], r["bb"]) <= r["tol"], r
    assert_same_eigs(sla.eigvals(H, T), sla.eigvals(A, B), 1e-8)


def _triu_with_zero_columns(n, cols, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    B = np.triu(rng.standard_normal((n, n))) + 3 * np.eye(n)
    B[:, cols] = 0.0
    return A, B


@pytest.mark.parametrize("case", ["saddle", "triu"])
def test_preprocess_deflates_zero_columns(case):
    if case == "saddle":
        A, B = pencils.saddle_point(16, 7)
        B = np.triu(B)
    else:
        A, B = _triu_with_zero_columns(12, [2, 5, 6, 11], 8)
    zc = front.zero_columns(B)
    H, T, Q, Z, l = front.preprocess(A, B, nb=4)
    assert l == len(zc) > 1
    r = report(A, B, H, T, Q, Z)
    assert r["sh"] == 0 and r["st"] == 0, r
    assert max(r["oq"], r["oz"], r["ba"], r["bb"]) <= r["tol"], r
    # the first l columns: T zero, H upper triangular (generalized Schur form)
    assert not np.any(T[:, :l])
    assert not np.any(np.tril(H[:, :l], -1))
    # l infinite eigenvalues (exact zeros on T's diagonal), the finite ones unchanged
    assert int(np.sum(np.diag(T) == 0.0)) >= l
    assert_same_eigs(finite_eigs(H, T), finite_eigs(A, B), 1e-7)


def test_preprocess_nothing_to_deflate_is_algorithm1():
    A, B = pencils.random_qr(10, 3)
    H, T, Q, Z, l = front.preprocess(A, B, nb=4)
    assert l == 0
    from oracle import househt as hh
    ref = hh.househt(A, B, nb=4)[:4]
    for a, b in zip(ref, (H, T, Q, Z)):
        assert np.array_equal(a, b)


FRONT_MUTATIONS = [
    # the front end's Q_B applied from the wrong side (Sec. 1)
    ("H, T, Qh, Z, _ = househt(Qb.T @ A, R, nb=nb)", "H, T, Qh, Z, _ = househt(Qb @ A, R, nb=nb)"),
    # Q_B left out of the accumulated Q
    ("return H, T, Qb @ Qh, Z", "return H, T, Qh, Z"),
    # zero columns moved to the back instead of the front (Sec. 3.4.1)
    ("perm = zc + [c for c in range(n) if c not in set(zc)]", "perm = [c for c in range(n) if c not in set(zc)] + zc"),
    # the first l rows of A miss Z22
    ("H[:l, l:] = A1[:l, l:] @ Z22", "H[:l, l:] = A1[:l, l:]"),
    # Z22 transposed on the first l rows of B
    ("T[:l, l:] = B1[:l, l:] @ Z22", "T[:l, l:] = B1[:l, l:] @ Z22.T"),
    # Q22 transposed in the accumulated Q
    ("Q[:, l:] = Q[:, l:] @ Q22", "Q[:, l:] = Q[:, l:] @ Q22.T"),
    # Q_1 applied to B from the wrong side
    ("B1 = Q1.T @ B0", "B1 = Q1 @ B0"),
]


def _front_mutant(old, new):
    import os
    import types
    src = open(os.path.join(os.path.dirname(front.__file__), "front.py")).read()
    assert src.count(old) == 1, old
    mod = types.ModuleType("oracle._front_mutant")
    mod.__dict__["__package__"] = "oracle"
    mod.__dict__["__name__"] = "oracle._front_mutant"
    exec(compile(src.replace(old, new), "front_mutant.py", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("idx", range(len(FRONT_MUTATIONS)))
def test_planted_front_mistake_is_caught(idx):
    mod = _front_mutant(*FRONT_MUTATIONS[idx])
    rng = np.random.default_rng(91)
    n = 14
    A, B = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    A2, B2 = _triu_with_zero_columns(12, [2, 5, 6, 11], 8)
    caught = False
    try:
        H, T, Q, Z = mod.general(A, B, nb=4)
        r = report(A, B, H, T, Q, Z)
        assert r["sh"] == 0 and r["st"] == 0 and max(r["oq"], r["oz"], r["ba"], r["bb"]) <= r["tol"], r
        H, T, Q, Z, l = mod.preprocess(A2, B2, nb=4)
        r = report(A2, B2, H, T, Q, Z)
        assert r["sh"] == 0 and r["st"] == 0 and max(r["oq"], r["oz"], r["ba"], r["bb"]) <= r["tol"], r
        assert not np.any(T[:, :l]) and not np.any(np.tril(H[:, :l], -1))
    except (AssertionError, ValueError, np.linalg.LinAlgError):
        caught = True
    assert caught, FRONT_MUTATIONS[idx][1]
