"""The QZ front end (Sec. 1) and the preprocessing of zero columns of B
(Sec. 3.4.1), each followed by Algorithm 1 (``househt``).  TEST
INFRASTRUCTURE ONLY: plain numpy, explicit dense orthogonal factors.

* ``general(A, B)``: B is a general matrix.  B = Q_B R by Householder QR
  (DLARFG rule, Sec. 2.1), then Algorithm 1 on (Q_B^T A, R) with Q starting
  from Q_B, so that H = Q^T A Z and T = Q^T B Z for the input pencil.
* ``preprocess(A, B)``: B upper triangular with l > 1 zero columns.  The
  steps of Sec. 3.4.1 in the paper's order: Z_0 moves the zero columns to the
  front (Q_0 = Z_0 when B is diagonal, else I); A_0 = Q_0^T A Z_0 and
  B_0 = Q_0^T B Z_0; the QR A_0(:, 1:l) = Q_1 [A11; 0] gives
  A_1 = [A11 A12; 0 A22] and B_1 = [0 B12; 0 B22]; the trailing pencil
  (A22, B22) then takes the front end and Algorithm 1 (Q22, Z22), and the
  first l rows take Z22 from the right.
"""
from __future__ import annotations

import numpy as np

from .househt import househt, qr_factor


def general(A, B, nb: int = 16):
    """(H, T, Q, Z) of the pencil (A, B) with a general B."""
    A = np.array(A, dtype=np.float64)
    B = np.array(B, dtype=np.float64)
    Qb, R = qr_factor(B)
    R = np.triu(R)
    H, T, Qh, Z, _ = househt(Qb.T @ A, R, nb=nb)
    return H, T, Qb @ Qh, Z


def zero_columns(B) -> list[int]:
    """Columns c of the upper triangle of B with B(0:c+1, c) = 0."""
    B = np.triu(np.asarray(B, dtype=np.float64))
    return [c for c in range(B.shape[0]) if not np.any(B[:c + 1, c])]


def preprocess(A, B, nb: int = 16):
    """(H, T, Q, Z, l) of Sec. 3.4.1; l = 0 when there is nothing to deflate
    (at most one zero column: the pencil is reduced as it is)."""
    A = np.array(A, dtype=np.float64)
    B = np.triu(np.array(B, dtype=np.float64))
    n = A.shape[0]
    zc = zero_columns(B)
    l = len(zc)
    if l <= 1 or n <= 2:
        H, T, Q, Z, _ = househt(A, B, nb=nb)
        return H, T, Q, Z, 0
    perm = zc + [c for c in range(n) if c not in set(zc)]
    Z0 = np.eye(n)[:, perm]
    diag = not np.any(np.triu(B, 1))
    Q0 = Z0 if diag else np.eye(n)
    A0 = Q0.T @ A @ Z0
    B0 = Q0.T @ B @ Z0
    Q1, _ = qr_factor(A0[:, :l])
    A1 = Q1.T @ A0
    B1 = Q1.T @ B0
    A1[l:, :l] = 0.0
    A1[:l, :l] = np.triu(A1[:l, :l])
    B1[:, :l] = 0.0
    m2 = n - l
    H, T = A1.copy(), B1.copy()
    Q22, Z22 = np.eye(m2), np.eye(m2)
    if m2 > 0:
        H22, T22, Q22, Z22 = general(A1[l:, l:], B1[l:, l:], nb=nb)
        H[l:, l:], T[l:, l:] = H22, T22
        H[:l, l:] = A1[:l, l:] @ Z22
        T[:l, l:] = B1[:l, l:] @ Z22
    Q = Q0 @ Q1
    Q[:, l:] = Q[:, l:] @ Q22
    Z = Z0.copy()
    Z[:, l:] = Z[:, l:] @ Z22
    return H, T, Q, Z, l
