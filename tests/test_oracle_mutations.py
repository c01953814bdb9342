"""Planted mistakes: each plausible slip in the Algorithm 1 oracle (a sign, a
transposed factor, a dropped term, an index off by one) must be caught by the
invariant checks that pin the oracle.  The mutation is applied to a copy of
the oracle's source on the CPU; the real module is never modified."""
import importlib.util
import os
import sys
import types

import numpy as np
import pytest

import oracle
from oracle import checks
from paper_1710_08538_gb300 import pencils

SRC = os.path.join(os.path.dirname(oracle.__file__), "househt.py")

MUTATIONS = [
    # S growth sign (Sec. 3.2.2b)
    ("P.S[:k, k] = -beta * (P.S[:k, :k] @ (P.U[:, :k].T @ u))",
     "P.S[:k, k] = beta * (P.S[:k, :k] @ (P.U[:, :k].T @ u))"),
    # T growth transposed (Sec. 3.2.2d)
    ("P.Tw[:k, k] = -gamma * (P.Tw[:k, :k] @ vtv)", "P.Tw[:k, k] = -gamma * (P.Tw[:k, :k].T @ vtv)"),
    # dropped -Y V^T v term of the new Y column (Sec. 3.2.2d)
    ("P.Y[s + 1:, k] = gamma * (A[s + 1:, j + 1:] @ vv[j + 1:] - P.Y[s + 1:, :k] @ vtv)",
     "P.Y[s + 1:, k] = gamma * (A[s + 1:, j + 1:] @ vv[j + 1:])"),
    # S instead of S^T in the column update (Sec. 3.2.2a)
    ("A[s + 1:, j] -= Uk @ (P.S[:k, :k].T @ (Uk.T @ A[s + 1:, j]))",
     "A[s + 1:, j] -= Uk @ (P.S[:k, :k] @ (Uk.T @ A[s + 1:, j]))"),
    # deferred rows of Y off by one (Remark 3.1)
    ("A[:s + 1, s + 1:j] -= Y[:s + 1, :] @ P.V[s + 1:j, :k].T",
     "A[:s, s + 1:j] -= Y[:s, :] @ P.V[s + 1:j, :k].T"),
    # T instead of T^T in the enlarged solve (Sec. 3.2.2c step 3)
    ("y = yt - V @ (Tw.T @ (V.T @ yt))", "y = yt - V @ (Tw @ (V.T @ yt))"),
    # S^T instead of S in step 1 of the enlarged solve
    ("ct = ct - U @ (S @ (U.T @ ct))", "ct = ct - U @ (S.T @ (U.T @ ct))"),
    # right absorption rank-k correction with T^T (Sec. 3.3.1c step 3)
    ("X[:, s + 1:j + 1] -= W @ Tw @ V1.T", "X[:, s + 1:j + 1] -= W @ Tw.T @ V1.T"),
    # L-hat taken from the wrong rows (Sec. 3.3.1b)
    ("L1 = V2[p - k:, :]", "L1 = V2[:k, :]"),
    # left absorption uses S instead of S^T on B (Sec. 3.3.2c step 5)
    ("B[s + 1:j + k + 1, j + 1:] -= Ut @ S.T @ W.T", "B[s + 1:j + k + 1, j + 1:] -= Ut @ S @ W.T"),
    # Q update with S^T (Sec. 3.3.2d)
    ("Q[:, s + 1:j + k + 1] -= W @ S @ Ut.T", "Q[:, s + 1:j + k + 1] -= W @ S.T @ Ut.T"),
    # spike update skips the U2 part (Sec. 3.3.2c step 1)
    ("B[s + 1:j + 1, s + 1:j + 1] -= U1 @ S.T @ (Us.T @ B[s + 1:, s + 1:j + 1])",
     "B[s + 1:j + 1, s + 1:j + 1] -= U1 @ S.T @ (U1.T @ B[s + 1:j + 1, s + 1:j + 1])"),
    # restore RQ applied to A with the wrong side/transposition (Sec. 3.3.1e)
    ("A[:, c0:c1] = A[:, c0:c1] @ M", "A[:, c0:c1] = A[:, c0:c1] @ M.T"),
    # QR chain applied to Q with the transpose (Sec. 3.3.2d step 1)
    ("Q[:, q0:q1] = Q[:, q0:q1] @ Qm", "Q[:, q0:q1] = Q[:, q0:q1] @ Qm.T"),
    # column j of A not updated at absorption (Sec. 3.3.1e step 2)
    ("A[:, j] -= Y @ P.V[j, :k]", "A[s + 1:, j] -= Y[s + 1:] @ P.V[j, :k]"),
    # residual with S instead of S^T (Sec. 3.2.2c, residual step 3)
    ("w = w - U @ (S.T @ (U.T @ w))", "w = w - U @ (S @ (U.T @ w))"),
]


def _mutant(old: str, new: str) -> types.ModuleType:
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found exactly once: {old}"
    src = src.replace(old, new)
    mod = types.ModuleType("oracle._mutant")
    mod.__dict__["__package__"] = "oracle"
    mod.__dict__["__name__"] = "oracle._mutant"
    exec(compile(src, "househt_mutant.py", "exec"), mod.__dict__)
    return mod


def _substep_pins(mod):
    """The sub-step pins of test_oracle_pins, run against a module: the
    factored solve equals a dense solve of the explicit B~22 (Sec. 3.2.2c),
    its residual equals the explicit one, and a random pencil needs
    (almost) no iterative refinement (Sec. 4, Test Suite 1)."""
    n, nb = 30, 6
    A, B = pencils.random_qr(n, 12)
    B = np.triu(B)
    P = mod._Panel(n, nb)
    st = {"ir_steps": 0, "cols_with_ir": 0, "ir_failures": 0}
    k, _ = mod._panel(A.copy(), B, P, 0, nb, 2 * mod.U_ROUND * np.linalg.norm(B), 10, st, None)
    assert k == nb and st["ir_failures"] == 0 and st["ir_steps"] <= nb, st
    j = k - 1
    L = np.eye(n) - P.U[:, :k] @ P.S[:k, :k] @ P.U[:, :k].T
    R = np.eye(n) - P.V[:, :k - 1] @ P.Tw[:k - 1, :k - 1] @ P.V[:, :k - 1].T
    Bt = L.T @ B @ R
    c = np.random.default_rng(1).standard_normal(n - j - 1)
    x, sigma = mod._factored_solve(B, P, 0, j, k, k - 1, c)
    assert np.allclose(x, np.linalg.solve(Bt[j + 1:, j + 1:], sigma * c), rtol=1e-10, atol=1e-12)
    r = mod._residual(B, P, 0, j, k, k - 1, sigma * c, x)
    assert np.allclose(r, sigma * c - Bt[j + 1:, j + 1:] @ x, atol=1e-13)


@pytest.mark.parametrize("idx", range(len(MUTATIONS)))
def test_planted_mistake_is_caught(oracle_lib, idx):
    old, new = MUTATIONS[idx]
    mod = _mutant(old, new)
    caught = False
    errors = (AssertionError, ValueError, np.linalg.LinAlgError, FloatingPointError, IndexError)
    for kind, n, nb in (("random_qr", 40, 8), ("near_infinite", 40, 8), ("random_qr", 37, 5)):
        A, B = pencils.make(kind, n, 99)
        try:
            with np.errstate(all="ignore"):
                H, T, Q, Z, _ = mod.househt(A, B, nb=nb)
            checks.assert_invariants(A, B, H, T, Q, Z)
        except errors:
            caught = True
            break
    if not caught:
        try:
            with np.errstate(all="ignore"):
                _substep_pins(mod)
        except errors:
            caught = True
    assert caught, f"mutation not detected: {new}"


def test_unmutated_source_passes(oracle_lib):
    mod = _mutant("U_ROUND = 2.0 ** -53", "U_ROUND = 2.0 ** -53")
    A, B = pencils.random_qr(40, 99)
    H, T, Q, Z, _ = mod.househt(A, B, nb=8)
    checks.assert_invariants(A, B, H, T, Q, Z)
    _substep_pins(mod)
