"""Seeded synthetic pencils (A, B) shaped like the paper's workloads.

This module only draws inputs; it holds none of the reduction's arithmetic.
It is shared by the tests (which feed the same bits to the CPU oracle and to
the CUDA library) and by ``bench.py``.  Every generator uses
``numpy.random.Generator(PCG64(seed))`` and returns Fortran-ordered float64
arrays with B upper triangular.

Workloads
  ``random_qr``      A ~ N(0,1); B = R factor of the QR of an N(0,1) matrix
                     with a positive diagonal (the paper's Test Suite 1).
  ``near_infinite``  A ~ N(0,1); B upper triangular with N(0,1) strict upper
                     part, diagonal U[0.5, 2] except round(0.1 n) positions
                     set to 1e-12 (near-infinite eigenvalues; IR-heavy like
                     Test Suites 2 and 4).
  ``shifted_triu``   A ~ N(0,1); B = triu(N(0,1)) + 4 I.
  ``graded``         A = D1 G1 D2, B = triu(D3 G2 D4), log10 diag(Di) ~ U[-4, 4].
  ``saddle_point``   A = [X Y; Y^T 0], B = [I 0; 0 0], X SPD, dim X = 3n/4
                     (Test Suite 4; B singular).
  ``batch_sizes``    sizes n ~ U{lo..hi} for the batched workload.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _normal(rng: np.random.Generator, n: int) -> np.ndarray:
    return np.asfortranarray(rng.standard_normal((n, n)))


def random_qr(n: int, seed: int):
    rng = _rng(seed)
    A = _normal(rng, n)
    G = _normal(rng, n)
    if n == 0:
        return A, G
    R = np.linalg.qr(G, mode="r")
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    B = np.asfortranarray(np.triu(d[:, None] * R))
    return A, B


def near_infinite(n: int, seed: int, frac: float = 0.1, tiny: float = 1e-12):
    rng = _rng(seed)
    A = _normal(rng, n)
    B = np.triu(_normal(rng, n), 1)
    diag = rng.uniform(0.5, 2.0, size=n)
    cnt = int(round(frac * n))
    if cnt:
        pos = rng.choice(n, size=cnt, replace=False)
        diag[pos] = tiny
    B[np.arange(n), np.arange(n)] = diag
    return A, np.asfortranarray(B)


def shifted_triu(n: int, seed: int, shift: float = 4.0):
    rng = _rng(seed)
    A = _normal(rng, n)
    B = np.triu(_normal(rng, n))
    B[np.arange(n), np.arange(n)] += shift
    return A, np.asfortranarray(B)


def graded(n: int, seed: int, decades: float = 4.0):
    rng = _rng(seed)
    d = [10.0 ** rng.uniform(-decades, decades, size=n) for _ in range(4)]
    G1 = _normal(rng, n)
    G2 = _normal(rng, n)
    A = (d[0][:, None] * G1) * d[1][None, :]
    B = np.triu((d[2][:, None] * G2) * d[3][None, :])
    return np.asfortranarray(A), np.asfortranarray(B)


def saddle_point(n: int, seed: int):
    rng = _rng(seed)
    nx = (3 * n) // 4
    ny = n - nx
    G = rng.standard_normal((nx, nx))
    X = G @ G.T / max(nx, 1) + np.eye(nx)
    Yb = rng.standard_normal((nx, ny))
    A = np.zeros((n, n))
    A[:nx, :nx] = X
    A[:nx, nx:] = Yb
    A[nx:, :nx] = Yb.T
    B = np.zeros((n, n))
    B[np.arange(nx), np.arange(nx)] = 1.0
    return np.asfortranarray(A), np.asfortranarray(B)


def batch_sizes(count: int, seed: int, lo: int = 64, hi: int = 1024) -> np.ndarray:
    return _rng(seed).integers(lo, hi + 1, size=count)


WORKLOADS = {
    "random_qr": random_qr,
    "near_infinite": near_infinite,
    "shifted_triu": shifted_triu,
    "graded": graded,
    "saddle_point": saddle_point,
}


def make(kind: str, n: int, seed: int):
    return WORKLOADS[kind](n, seed)
