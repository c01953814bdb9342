"""Algorithm 1 (HouseHT) of Bujanovic, Karlsson, Kressner (arXiv 1710.08538),
written out step by step in numpy.  TEST INFRASTRUCTURE ONLY.

Indices are 0-based; the paper's 1-based column j is column j-1 here.  With
s the first unreduced column of A and k = j - s delayed reflectors:
  * left reflector i (i = 0..k-1) reduces column s+i of A and acts on rows
    s+i+1..n-1;
  * right reflector i reduces column s+i+1 of B~ and acts on columns
    s+i+1..n-1;
  * V1 = V[s+1:j+1] and U1 = U[s+1:j+1] are k x k lower triangular,
    V2 = V[j+1:] and U2 = U[j+1:] have p = n-j-1 rows.

Every orthogonal factor of the absorption chains is formed as an explicit
dense matrix (no WY blocking): this module is for checking, not speed.

Readings where the paper is silent:
  * Householder sign: DLARFG rule (alpha = -sign(x0)||x||, identity when the
    tail is exactly zero).
  * IR tolerance 2u||B||_F with u = 2^-53 and ||B||_F of the input B; "abort
    after ten iterations" = at most ``max_ir`` correction solves; a failure
    with k = 0 delayed reflectors is accepted (the k = 0 solve is backward
    stable, Sec. 3.2.2c).
  * A zero on the diagonal of the trailing B is replaced by 2 u rho ||B||_F
    at the start of each panel (Sec. 3.2.1, Remark 2.2), rho from the
    counter-based generator keyed by (seed, panel start s, diagonal index).
  * Panel width k <= min(nb, (n-s-1)//2) so that V2 and U2 keep at least k
    rows; windows follow Remark 3.2 (first window k~ rows, k < k~ <= 2k, or
    a single window of p rows when p <= 2k).
  * After the top-to-bottom QR restore of Sec. 3.3.2f the last diagonal block
    is still full; one more QR of that block finishes the triangular form.
  * Rows 0..s of Y are formed after the panel (Remark 3.1), and rows 0..s of
    the panel columns s+1..j-1 are updated with them at absorption.
"""
from __future__ import annotations

import numpy as np

from . import philox_normal

U_ROUND = 2.0 ** -53


# --------------------------------------------------------------------------
# Householder reflectors and small factorizations (Sec. 2.1, 2.4)
# --------------------------------------------------------------------------
def house(x: np.ndarray):
    """(v, beta, alpha): v[0] = 1, (I - beta v v^T) x = alpha e1 (DLARFG rule)."""
    x = np.asarray(x, dtype=np.float64)
    m = x.size
    v = np.zeros(m)
    if m == 0:
        return v, 0.0, 0.0
    v[0] = 1.0
    x0 = x[0]
    tail2 = float(np.dot(x[1:], x[1:]))
    if tail2 == 0.0:
        return v, 0.0, float(x0)
    nrm = np.sqrt(x0 * x0 + tail2)
    a = -nrm if x0 >= 0.0 else nrm
    v[1:] = x[1:] / (x0 - a)
    beta = 2.0 / float(np.dot(v, v))
    return v, beta, float(a)


def _reflector_matrix(m: int, v: np.ndarray, beta: float) -> np.ndarray:
    return np.eye(m) - beta * np.outer(v, v)


def qr_factor(X: np.ndarray):
    """X (M x k, M >= k) = Qm @ R, R upper triangular in its top k rows."""
    X = np.array(X, dtype=np.float64)
    M, k = X.shape
    Qm = np.eye(M)
    for c in range(min(k, M)):
        v, beta, alpha = house(X[c:, c])
        H = _reflector_matrix(M - c, v, beta)
        X[c:, c:] = H @ X[c:, c:]
        X[c, c] = alpha
        X[c + 1:, c] = 0.0
        Qm[:, c:] = Qm[:, c:] @ H
    return Qm, X


def ql_factor(X: np.ndarray):
    """X (M x k, M >= k) = Qm @ L, L zero in rows 0..M-k-1 and lower
    triangular in its bottom k x k block."""
    X = np.array(X, dtype=np.float64)
    M, k = X.shape
    Qm = np.eye(M)
    for c in range(k - 1, -1, -1):
        t = M - k + c
        v_rev, beta, alpha = house(X[t::-1, c])
        v = v_rev[::-1]
        H = _reflector_matrix(t + 1, v, beta)
        X[:t + 1, :c + 1] = H @ X[:t + 1, :c + 1]
        X[t, c] = alpha
        X[:t, c] = 0.0
        Qm[:, :t + 1] = Qm[:, :t + 1] @ H
    return Qm, X


def rq_factor(X: np.ndarray):
    """X (k x K, K >= k): returns (M, R) with X @ M = R = [0 R1], R1 upper
    triangular k x k in the last k columns (M orthogonal)."""
    X = np.array(X, dtype=np.float64)
    k, K = X.shape
    M = np.eye(K)
    for c in range(k - 1, -1, -1):
        t = K - k + c
        v_rev, beta, alpha = house(X[c, t::-1])
        v = v_rev[::-1]
        H = _reflector_matrix(t + 1, v, beta)
        X[:c + 1, :t + 1] = X[:c + 1, :t + 1] @ H
        X[c, t] = alpha
        X[c, :t] = 0.0
        M[:, :t + 1] = M[:, :t + 1] @ H
    return M, X


# --------------------------------------------------------------------------
# Window / block layout of the absorption chains (Sec. 3.3, Remark 3.2)
# --------------------------------------------------------------------------
def first_window(p: int, k: int) -> int:
    """Rows k~ of the first QL (top) / QR (bottom) window."""
    if p <= 2 * k:
        return p
    return p - k * (-(-(p - 2 * k) // k))


def ql_windows(p: int, k: int):
    """Row ranges (relative to V2) of the top-to-bottom QL chain."""
    kt = first_window(p, k)
    wins = [(0, kt)]
    r0 = kt - k
    while r0 + 2 * k <= p and kt < p:
        wins.append((r0, r0 + 2 * k))
        r0 += k
    return wins


def qr_windows(p: int, k: int):
    """Row ranges (relative to U2) of the bottom-to-top QR chain."""
    kt = first_window(p, k)
    wins = [(p - kt, p)]
    r1 = p - kt + k
    while r1 - 2 * k >= 0 and kt < p:
        wins.append((r1 - 2 * k, r1))
        r1 -= k
    return wins


def right_blocks(p: int, k: int):
    """Column blocks of B(:, j+1:n) after the QL chain (small block first)."""
    if p <= k:
        return [(0, p)]
    b0 = first_window(p, k) - k
    return [(0, b0)] + [(b0 + i * k, b0 + (i + 1) * k) for i in range((p - b0) // k)]


def left_blocks(p: int, k: int):
    """Row blocks of B(j+1:n, :) after the QR chain (small block last)."""
    if p <= k:
        return [(0, p)]
    bl = first_window(p, k) - k
    nfull = (p - bl) // k
    return [(i * k, (i + 1) * k) for i in range(nfull)] + [(nfull * k, p)]


# --------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------
class _Panel:
    def __init__(self, n: int, kmax: int):
        self.U = np.zeros((n, kmax))
        self.V = np.zeros((n, kmax))
        self.Y = np.zeros((n, kmax))
        self.S = np.zeros((kmax, kmax))
        self.Tw = np.zeros((kmax, kmax))


_BIG = 2.0 ** 500   # rescale threshold of the scaled backward substitution


def _pow2_scale(target: float, value: float) -> float:
    """Largest power of two f <= target / value (value > 0, target > 0)."""
    m, e = np.frexp(target / value)
    return float(np.ldexp(1.0, int(e) - 1))


def _back_substitute(R: np.ndarray, c: np.ndarray):
    """Solve R y = sigma c (R upper triangular) by backward substitution.

    sigma in (0, 1] is a power of two chosen so that no |y_i| exceeds 2^500
    (the paper is silent on overflow; this follows the scaled triangular
    solve idea of LAPACK DLATRS).  Only the direction of the solution matters
    to an opposite reflector (Sec. 2.2), and the IR test is scale-free."""
    m = c.size
    y = np.array(c, dtype=np.float64)
    sigma = 1.0
    for i in range(m - 1, -1, -1):
        t = y[i] - np.dot(R[i, i + 1:], y[i + 1:])
        d = abs(R[i, i])
        if abs(t) > _BIG * d:
            f = _pow2_scale(_BIG * d, abs(t))
            y *= f
            t *= f
            sigma *= f
        y[i] = t / R[i, i]
    return y, sigma


def _factored_solve(B, P: _Panel, s: int, j: int, kl: int, kr: int, c: np.ndarray):
    """Solve B~22 x = sigma c through the enlarged system (Sec. 3.2.2c,
    steps 1-4); kl left and kr right reflectors are active.  Returns
    (x, sigma) with the scale sigma of the backward substitution."""
    n = B.shape[0]
    U, S, V, Tw = P.U[s + 1:, :kl], P.S[:kl, :kl], P.V[s + 1:, :kr], P.Tw[:kr, :kr]
    ct = np.zeros(n - s - 1)
    ct[j - s:] = c
    ct = ct - U @ (S @ (U.T @ ct))                    # (I - U S U^T) [0; c]
    yt, sigma = _back_substitute(B[s + 1:, s + 1:], ct)   # B y~ = sigma c~
    y = yt - V @ (Tw.T @ (V.T @ yt))                  # (I - V T V^T)^T y~
    return y[j - s:], sigma


def _normalize(x: np.ndarray, sigma: float):
    """Scale x by a power of two so that max |x_i| lies in [1, 2)."""
    mx = float(np.max(np.abs(x))) if x.size else 0.0
    if mx == 0.0 or not np.isfinite(mx):
        return x, sigma
    f = float(np.ldexp(1.0, -int(np.frexp(mx)[1]) + 1))
    return x * f, sigma * f


def _solve_ok(r: np.ndarray, x: np.ndarray, tol: float) -> bool:
    """IR stopping test ||r||_2 / ||x||_2 <= 2 u ||B||_F (Sec. 2.3); a
    non-finite residual or solution never passes."""
    nr = float(np.linalg.norm(r))
    nx = float(np.linalg.norm(x))
    return bool(np.isfinite(nr) and np.isfinite(nx) and nx > 0.0 and nr <= tol * nx)


def _residual(B, P: _Panel, s: int, j: int, kl: int, kr: int, c: np.ndarray, x: np.ndarray) -> np.ndarray:
    """r = c - B~22 x through the four steps of Sec. 3.2.2c."""
    n = B.shape[0]
    U, S, V, Tw = P.U[s + 1:, :kl], P.S[:kl, :kl], P.V[s + 1:, :kr], P.Tw[:kr, :kr]
    w = np.zeros(n - s - 1)
    w[j - s:] = x
    w = w - V @ (Tw @ (V.T @ w))                      # (I - V T V^T) [0; x]
    w = B[s + 1:, s + 1:] @ w                          # B w (B triangular)
    w = w - U @ (S.T @ (U.T @ w))                     # (I - U S^T U^T) w
    return c - w[j - s:]


def _panel(A, B, P: _Panel, s: int, kmax: int, tol: float, max_ir: int, stats: dict, fail_cols):
    """Reduce up to kmax columns starting at s (Sec. 3.2).  Returns the number
    k of accumulated left/right reflector pairs and whether IR failed."""
    n = A.shape[0]
    for k in range(kmax):
        j = s + k
        a_saved = A[:, j].copy()
        # (a) update column j with the k delayed right and left reflectors
        if k > 0:
            A[s + 1:, j] -= P.Y[s + 1:, :k] @ P.V[j, :k]
            Uk = P.U[s + 1:, :k]
            A[s + 1:, j] -= Uk @ (P.S[:k, :k].T @ (Uk.T @ A[s + 1:, j]))
        # (b) left reflector, S update
        v, beta, alpha = house(A[j + 1:, j])
        u = np.zeros(n)
        u[j + 1:] = v
        A[j + 1, j] = alpha
        A[j + 2:, j] = 0.0
        if k > 0:
            P.S[:k, k] = -beta * (P.S[:k, :k] @ (P.U[:, :k].T @ u))
        P.S[k, k] = beta
        P.U[:, k] = u
        # (c) factored solve of B~22 x = e1 with iterative refinement; the
        # iterate satisfies B~22 x ~ sigma e1 for a power-of-two sigma.
        p = n - j - 1
        e1 = np.zeros(p)
        e1[0] = 1.0
        x, sigma = _normalize(*_factored_solve(B, P, s, j, k + 1, k, e1))
        r = _residual(B, P, s, j, k + 1, k, sigma * e1, x)
        it = 0
        forced = fail_cols is not None and j in fail_cols and k > 0
        while (forced or not _solve_ok(r, x, tol)) and it < max_ir:
            d, t = _factored_solve(B, P, s, j, k + 1, k, r)
            x, sigma = _normalize(t * x + d, t * sigma)
            r = _residual(B, P, s, j, k + 1, k, sigma * e1, x)
            it += 1
        stats["ir_steps"] += it
        stats["cols_with_ir"] += int(it > 0)
        ok = (not forced) and _solve_ok(r, x, tol)
        if not ok and k > 0:
            # undo the left reflector and stop the panel (Algorithm 1)
            A[:, j] = a_saved
            P.U[:, k] = 0.0
            P.S[:, k] = 0.0
            P.S[k, :] = 0.0
            stats["ir_failures"] += 1
            return k, True
        # (d) right reflector, T and Y updates
        w, gamma, _ = house(x)
        vv = np.zeros(n)
        vv[j + 1:] = w
        vtv = P.V[:, :k].T @ vv
        if k > 0:
            P.Tw[:k, k] = -gamma * (P.Tw[:k, :k] @ vtv)
        P.Tw[k, k] = gamma
        P.Y[s + 1:, k] = gamma * (A[s + 1:, j + 1:] @ vv[j + 1:] - P.Y[s + 1:, :k] @ vtv)
        P.V[:, k] = vv
    return kmax, False


def _absorb(A, B, Q, Z, P: _Panel, s: int, k: int):
    """Absorb k right and k left reflectors (Sec. 3.3.1 and 3.3.2)."""
    n = A.shape[0]
    j = s + k
    p = n - j - 1
    V1 = P.V[s + 1:j + 1, :k].copy()
    V2 = P.V[j + 1:, :k].copy()
    U1 = P.U[s + 1:j + 1, :k].copy()
    U2 = P.U[j + 1:, :k].copy()
    S = P.S[:k, :k].copy()
    Tw = P.Tw[:k, :k].copy()
    Y = P.Y[:, :k]
    # Remark 3.1: rows 0..s of Y = A V T from the (still unmodified) rows 0..s.
    Y[:s + 1, :] = A[:s + 1, s + 1:] @ P.V[s + 1:, :k] @ Tw

    # ---- right reflectors (Sec. 3.3.1) --------------------------------------
    A[:s + 1, s + 1:j] -= Y[:s + 1, :] @ P.V[s + 1:j, :k].T    # deferred rows of panel columns
    A[:, j] -= Y @ P.V[j, :k]                                  # (e) step 2
    for (r0, r1) in ql_windows(p, k):                          # (b) V2 = Q1..Qr L
        Qm, Lw = ql_factor(V2[r0:r1])
        V2[r0:r1] = Lw
        c0, c1 = j + 1 + r0, j + 1 + r1
        B[:, c0:c1] = B[:, c0:c1] @ Qm                          # (c) step 1
        Z[:, c0:c1] = Z[:, c0:c1] @ Qm                          # (d) step 1
        A[:, c0:c1] = A[:, c0:c1] @ Qm                          # (e) step 1
    L1 = V2[p - k:, :]
    for X in (B, Z):                                           # (c)/(d) steps 2-4
        W = X[:, s + 1:j + 1] @ V1 + X[:, n - k:] @ L1
        X[:, s + 1:j + 1] -= W @ Tw @ V1.T
        X[:, n - k:] -= W @ Tw @ L1.T
    A[:, n - k:] -= Y @ L1.T                                   # (e) step 3
    blocks = right_blocks(p, k)                                # partial restore, bottom to top
    for b in range(len(blocks) - 1, 0, -1):
        r0, r1 = j + 1 + blocks[b][0], j + 1 + blocks[b][1]
        c0, c1 = j + 1 + blocks[b - 1][0], r1
        M, R = rq_factor(B[r0:r1, c0:c1])
        B[:r0, c0:c1] = B[:r0, c0:c1] @ M
        B[r0:r1, c0:c1] = R
        A[:, c0:c1] = A[:, c0:c1] @ M
        Z[:, c0:c1] = Z[:, c0:c1] @ M

    # ---- left reflectors (Sec. 3.3.2) ---------------------------------------
    Us = P.U[s + 1:, :k]
    B[s + 1:j + 1, s + 1:j + 1] -= U1 @ S.T @ (Us.T @ B[s + 1:, s + 1:j + 1])   # (c) step 1
    B[j + 1:, s + 1:j + 1] = 0.0                                                # (c) step 2
    for c in range(s + 1, j + 1):                       # spike columns are triangular (Fact 3)
        B[c + 1:j + 1, c] = 0.0
    for (r0, r1) in qr_windows(p, k):                   # (b) U2 = Q1..Qr R
        Qm, Rw = qr_factor(U2[r0:r1])
        U2[r0:r1] = Rw
        q0, q1 = j + 1 + r0, j + 1 + r1
        B[q0:q1, j + 1:] = Qm.T @ B[q0:q1, j + 1:]        # (c) step 3
        A[q0:q1, j:] = Qm.T @ A[q0:q1, j:]                # (e) step 1
        Q[:, q0:q1] = Q[:, q0:q1] @ Qm                    # (d) step 1
    Ut = np.vstack([U1, U2[:k, :]])                       # [U1; R1]
    W = B[s + 1:j + k + 1, j + 1:].T @ Ut                 # (c) steps 4-5
    B[s + 1:j + k + 1, j + 1:] -= Ut @ S.T @ W.T
    W = Q[:, s + 1:j + k + 1] @ Ut                        # (d) steps 2-3
    Q[:, s + 1:j + k + 1] -= W @ S @ Ut.T
    W = A[s + 1:j + k + 1, j:].T @ Ut                     # (e) steps 2-3
    A[s + 1:j + k + 1, j:] -= Ut @ S.T @ W.T
    lb = left_blocks(p, k)                                # (f) restore, top to bottom
    for b in range(len(lb)):
        r0 = j + 1 + lb[b][0]
        r1 = j + 1 + (lb[b + 1][1] if b + 1 < len(lb) else lb[b][1])
        c0, c1 = j + 1 + lb[b][0], j + 1 + lb[b][1]
        Qm, R = qr_factor(B[r0:r1, c0:c1])
        B[r0:r1, c1:] = Qm.T @ B[r0:r1, c1:]
        B[r0:r1, c0:c1] = R
        A[r0:r1, j:] = Qm.T @ A[r0:r1, j:]
        Q[:, r0:r1] = Q[:, r0:r1] @ Qm


def househt(A, B, nb: int = 16, max_ir: int = 10, seed: int = 0, ir_tol_scale: float = 1.0, fail_cols=None):
    """Algorithm 1.  Returns ``(H, T, Q, Z, stats)``.

    ``fail_cols`` (a set of 0-based columns) declares the solve failed at
    those columns when k >= 1, to drive the early-absorption path in tests.
    """
    A = np.array(A, dtype=np.float64, copy=True)
    B = np.triu(np.array(B, dtype=np.float64, copy=True))
    n = A.shape[0]
    Q = np.eye(n)
    Z = np.eye(n)
    stats = {"panels": 0, "ir_steps": 0, "cols_with_ir": 0, "ir_failures": 0, "perturbed": 0}
    if n <= 2:
        return A, B, Q, Z, stats
    bnorm = float(np.linalg.norm(B))
    tol = ir_tol_scale * 2.0 * U_ROUND * bnorm
    s = 0
    while s <= n - 3:
        for i in range(s + 1, n):                       # Remark 2.2 / Sec. 3.2.1
            if B[i, i] == 0.0:
                B[i, i] = 2.0 * U_ROUND * philox_normal(seed, s, i) * bnorm
                stats["perturbed"] += 1
        kmax = min(nb, (n - s - 1) // 2)
        P = _Panel(n, kmax)
        k, failed = _panel(A, B, P, s, kmax, tol, max_ir, stats, fail_cols)
        if k > 0:
            _absorb(A, B, Q, Z, P, s, k)
        stats["panels"] += 1
        s += max(k, 1) if not failed else k
    return A, B, Q, Z, stats
