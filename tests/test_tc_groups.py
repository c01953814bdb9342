"""Grouped windows of the emulated chain applications (tcgen05 sweep).

The emulated sweeps apply the product G = G_t0 G_t0+1 ... of g = max(1, 64/k - 1)
consecutive window transforms of a chain (Sec. 3.3, Remark 3.2) as one dense
product on the union of their rows.  The sweep kernel holds G and a stripe of
lines in fixed 64-wide tiles, and it assumes the union is contiguous.  These
CPU tests check both assumptions against the window geometry of the oracle
(written from the paper independently of the CUDA path), for every chain kind
and k <= 32.  They also check that applying the group's product once equals
applying its windows one by one, on random chains of Householder windows.
"""
import numpy as np
import pytest

from oracle import househt as hh

TW = 64  # widest group (rows of the union) of the sweep kernel


def group(k):
    """Windows per group of the tcgen05 sweep for chains of k reflectors."""
    return max(1, TW // k - 1)


def chain_windows(kind, p, k):
    """(offset, width, reflectors) of every window of one chain, in the order
    the sweeps apply them: 0 QL chain, 1 QR chain, 2 RQ restore (right blocks,
    bottom to top), 3 QR restore (left blocks, top to bottom)."""
    if kind == 0:
        return [(a, b - a, k) for a, b in hh.ql_windows(p, k)]
    if kind == 1:
        return [(a, b - a, k) for a, b in hh.qr_windows(p, k)]
    if kind == 2:
        blocks = hh.right_blocks(p, k)
        out = []
        for t in range(len(blocks) - 1):
            bb = len(blocks) - 1 - t
            (c0, _), (d0, d1) = blocks[bb - 1], blocks[bb]
            out.append((c0, d1 - c0, d1 - d0))
        return out
    blocks = hh.left_blocks(p, k)
    out = []
    for t, (r0, r1) in enumerate(blocks):
        e1 = blocks[t + 1][1] if t + 1 < len(blocks) else r1
        out.append((r0, e1 - r0, r1 - r0))
    return out


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
@pytest.mark.parametrize("k", list(range(1, 33)))
def test_group_fits_the_tiles(kind, k):
    g = group(k)
    for p in list(range(1, 200)) + [257, 1000, 4093, 16382]:
        wins = chain_windows(kind, p, k)
        for m0 in range(0, len(wins), g):
            grp = wins[m0:m0 + g]
            lo = min(o for o, _, _ in grp)
            hi = max(o + w for o, w, _ in grp)
            assert hi - lo <= TW, (kind, k, p, m0, hi - lo)
            # contiguous union: every row of [lo, hi) is in some window
            covered = np.zeros(hi - lo, dtype=bool)
            for o, w, _ in grp:
                covered[o - lo:o - lo + w] = True
            assert covered.all(), (kind, k, p, m0)


def _householder_window(rng, w, k):
    """G = I - V W^T of k reflectors on w rows (W = V T^T, eq. (1) for T)."""
    X = rng.standard_normal((w, k))
    V = np.zeros((w, k))
    tau = np.zeros(k)
    for q in range(k):
        x = X[q:, q]
        alpha = -np.copysign(np.linalg.norm(x), x[0])
        v = x.copy()
        v[0] -= alpha
        v /= v[0]
        tau[q] = 2.0 / (v @ v)
        V[q:, q] = v
        X[q:, :] -= tau[q] * np.outer(v, v @ X[q:, :])
    T = np.zeros((k, k))
    for q in range(k):
        T[q, q] = tau[q]
        T[:q, q] = -tau[q] * T[:q, :q] @ (V[:, :q].T @ V[:, q])
    return V, V @ T.T


@pytest.mark.parametrize("k", [1, 2, 3, 7, 16, 21, 32])
def test_group_product_reproduces_the_chain(k):
    rng = np.random.default_rng(100 + k)
    p = 23 * k + 5
    g = group(k)
    wins = [(o, w, _householder_window(rng, w, r)) for o, w, r in chain_windows(0, p, k) if r <= w]
    X = rng.standard_normal((7, p))
    ref = X.copy()
    for o, w, (V, W) in wins:
        seg = ref[:, o:o + w]
        ref[:, o:o + w] = seg - (seg @ V) @ W.T
    got = X.copy()
    for m0 in range(0, len(wins), g):
        grp = wins[m0:m0 + g]
        lo = min(o for o, _, _ in grp)
        hi = max(o + w for o, w, _ in grp)
        G = np.eye(hi - lo)
        for o, w, (V, W) in grp:
            Gi = np.eye(hi - lo)
            Gi[o - lo:o - lo + w, o - lo:o - lo + w] -= V @ W.T
            G = G @ Gi
        got[:, lo:hi] = got[:, lo:hi] @ G
    assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
