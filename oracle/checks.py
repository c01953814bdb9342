"""Invariants of an HT reduction (TEST INFRASTRUCTURE ONLY).

The paper checks each result by its structure and by ||H - Q^T A Z||_F and
||T - Q^T B Z||_F (Sec. 4); Theorem A.1 and the corollary after it give the
O(u) bounds on the backward errors and on the loss of orthogonality.

All products here are plain FP64 numpy matmuls on the CPU.
"""
from __future__ import annotations

import numpy as np

EPS64 = 2.0 ** -52


def structure_violations(H: np.ndarray, T: np.ndarray) -> tuple[int, int]:
    """Count entries that must be exact zeros but are not: H(i, j) for
    i > j + 1 and T(i, j) for i > j (-0.0 counts as zero)."""
    n = H.shape[0]
    il_h = np.tril_indices(n, -2)
    il_t = np.tril_indices(n, -1)
    return int(np.count_nonzero(H[il_h])), int(np.count_nonzero(T[il_t]))


def orthogonality(M: np.ndarray) -> float:
    """||M^T M - I||_F."""
    n = M.shape[0]
    return float(np.linalg.norm(M.T @ M - np.eye(n)))


def backward_errors(A, B, H, T, Q, Z) -> tuple[float, float]:
    """||Q H Z^T - A||_F / ||A||_F and ||Q T Z^T - B||_F / ||B||_F."""
    Bu = np.triu(B)
    ra = np.linalg.norm(Q @ H @ Z.T - A) / max(np.linalg.norm(A), np.finfo(float).tiny)
    rb = np.linalg.norm(Q @ T @ Z.T - Bu) / max(np.linalg.norm(Bu), np.finfo(float).tiny)
    return float(ra), float(rb)


def invariant_report(A, B, H, T, Q, Z) -> dict:
    n = A.shape[0]
    sh, st = structure_violations(H, T)
    ra, rb = backward_errors(A, B, H, T, Q, Z)
    return {
        "n": n,
        "h_nonzeros_below_subdiag": sh,
        "t_nonzeros_below_diag": st,
        "orth_q": orthogonality(Q),
        "orth_z": orthogonality(Z),
        "bwd_a": ra,
        "bwd_b": rb,
        "q_e1": float(np.linalg.norm(Q[:, 0] - np.eye(n)[:, 0])) if n else 0.0,
        "tol": 20.0 * n * EPS64,
    }


def assert_invariants(A, B, H, T, Q, Z, bwd_tol: float | None = None, orth_tol: float | None = None) -> dict:
    """Invariants (i)-(iii): exact zeros, orthogonality <= 20 n eps and
    relative backward errors <= 20 n eps (or the given tolerances)."""
    rep = invariant_report(A, B, H, T, Q, Z)
    n = rep["n"]
    tol = 20.0 * max(n, 1) * EPS64
    bt = tol if bwd_tol is None else bwd_tol
    ot = tol if orth_tol is None else orth_tol
    assert rep["h_nonzeros_below_subdiag"] == 0, rep
    assert rep["t_nonzeros_below_diag"] == 0, rep
    assert rep["orth_q"] <= ot and rep["orth_z"] <= ot, rep
    assert rep["bwd_a"] <= bt and rep["bwd_b"] <= bt, rep
    assert rep["q_e1"] == 0.0, rep
    return rep


def sign_normalize(H, T, Q, Z):
    """Fix the diagonal sign freedom (Q, Z) -> (Q D1, Z D2) so that Q e1 = e1,
    T has a nonnegative diagonal and H a nonnegative subdiagonal.  Two
    correct reductions of the same pencil agree after this (implicit-Q
    argument) as long as no subdiagonal of H and no diagonal of T is zero."""
    n = H.shape[0]
    d1 = np.ones(n)
    d2 = np.ones(n)
    for i in range(n):
        if i > 0:
            h = H[i, i - 1] * d2[i - 1]
            d1[i] = -1.0 if h < 0 else 1.0
        t = d1[i] * T[i, i]
        d2[i] = -1.0 if t < 0 else 1.0
    Hn = (d1[:, None] * H) * d2[None, :]
    Tn = (d1[:, None] * T) * d2[None, :]
    return Hn, Tn, Q * d1[None, :], Z * d2[None, :]
