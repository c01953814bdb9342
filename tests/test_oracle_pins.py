"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Nothing here uses a GPU.  Each test names the passage it checks.  The oracle
(oracle/) is checked against: exact special cases (n <= 2, idempotence, B = I
vs a library Hessenberg reduction), brute-force determinant polynomials for
n <= 4, Lemma 2.1, eq. (1), eqs. (5) and (7), the fill pattern printed in the
paper's figure for Sec. 3.3.1c, library generalized eigenvalues, and
agreement of three independent oracles modulo the diagonal sign freedom.
"""
import os

import mpmath
import numpy as np
import pytest
import scipy.linalg as sla
from scipy.optimize import linear_sum_assignment

import oracle
from oracle import checks
from oracle import househt as hh
from paper_1710_08538_gb300 import pencils

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = 2.0 ** -52


def _all_oracles(A, B, nb=4):
    return {
        "basic": oracle.basic_househt(A, B)[:4],
        "givens": oracle.givens_ht(A, B),
        "househt": hh.househt(A, B, nb=nb)[:4],
    }


def _read_pattern(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([ch == "x" for ch in line])
    return np.array(rows)


# --------------------------------------------------------------------------
# Householder reflector (Sec. 2.1) and the counter-based generator
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m", [1, 2, 3, 7, 40])
def test_house_reduces_vector(oracle_lib, m):
    rng = np.random.default_rng(m)
    for trial in range(5):
        x = rng.standard_normal(m)
        if trial == 1:
            x[0] = 0.0
        if trial == 2:
            x[0] = -abs(x[0]) - 1.0
        for impl in (oracle.house, hh.house):
            v, beta, alpha = impl(x)
            assert v[0] == 1.0
            Hx = x - beta * v * np.dot(v, x)
            assert abs(abs(alpha) - np.linalg.norm(x)) <= 4 * EPS * np.linalg.norm(x)
            assert np.allclose(Hx[0], alpha, rtol=4 * EPS * m, atol=0)
            if m > 1:
                assert np.max(np.abs(Hx[1:])) <= 8 * m * EPS * np.linalg.norm(x)
            if m > 1:
                # DLARFG sign rule: alpha = -sign(x0) ||x||, sign(0) = +
                assert np.sign(alpha) == (-1.0 if x[0] >= 0 else 1.0)
                # orthogonality of I - beta v v^T: beta = 2 / v^T v
                assert abs(beta * np.dot(v, v) - 2.0) <= 8 * EPS
        v1, b1, a1 = oracle.house(x)
        v2, b2, a2 = hh.house(x)
        assert np.allclose(v1, v2, rtol=1e-14, atol=1e-15) and abs(b1 - b2) <= 1e-14 and abs(a1 - a2) <= 1e-14 * abs(a1)


def test_house_identity_when_tail_zero(oracle_lib):
    for x in ([3.0, 0.0, 0.0], [-2.0, 0.0], [0.0, 0.0, 0.0], [5.0]):
        for impl in (oracle.house, hh.house):
            v, beta, alpha = impl(np.array(x))
            assert beta == 0.0 and alpha == x[0]


def test_philox_normal_is_standard_normal(oracle_lib):
    from scipy import stats
    z = np.array([oracle.philox_normal(7, c, i) for c in range(50) for i in range(400)])
    assert abs(z.mean()) < 0.03 and abs(z.var() - 1.0) < 0.05
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # deterministic and counter-based
    assert oracle.philox_normal(7, 3, 9) == oracle.philox_normal(7, 3, 9)
    assert oracle.philox_normal(7, 3, 9) != oracle.philox_normal(8, 3, 9)


def _philox_kat():
    rows = []
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    for ln in open(path):
        ln = ln.split("#")[0].split()
        if ln:
            w = [int(x, 16) for x in ln]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox4x32_10_known_answers(oracle_lib):
    """The counter-based generator behind the Remark 2.2 perturbation is
    Philox4x32-10: its raw blocks equal the published known-answer vectors
    (a wrong multiplier, Weyl constant, round count or word order fails)."""
    kat = _philox_kat()
    assert len(kat) == 3
    for ctr, key, out in kat:
        assert oracle.philox4x32_10(ctr, key) == out


def test_philox_normal_uses_first_two_words(oracle_lib):
    """Seed 0, column 0, index 0 is the all-zero counter and key of the first
    known-answer vector; the sample is Box-Muller on its words 0 and 1."""
    ctr, key, out = _philox_kat()[0]
    assert ctr == [0, 0, 0, 0] and key == [0, 0]
    u1 = (out[0] + 1.0) * 2.0 ** -32
    u2 = out[1] * 2.0 ** -32
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    assert abs(oracle.philox_normal(0, 0, 0) - z) <= 1e-15 * max(1.0, abs(z))


# --------------------------------------------------------------------------
# Exact special cases
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [0, 1, 2])
def test_tiny_n_is_identity(oracle_lib, n):
    """The loop j = 1:n-2 of Algorithms 1 and 2 is empty for n <= 2."""
    A, B = pencils.random_qr(n, 5)
    for name, (H, T, Q, Z) in _all_oracles(A, B).items():
        if name == "givens" and n == 0:
            continue
        assert np.array_equal(H, A) and np.array_equal(T, np.triu(B)), name
        assert np.array_equal(Q, np.eye(n)) and np.array_equal(Z, np.eye(n)), name


@pytest.mark.parametrize("n", [3, 6, 17])
def test_idempotent_on_ht_form(oracle_lib, n):
    """An input already in HT form is left alone: every left reflector sees a
    zero tail and every solve with triangular B gives x = e1 / b, so each
    reflector is the identity (DLARFG rule)."""
    rng = np.random.default_rng(n)
    A = np.triu(rng.standard_normal((n, n)), -1)
    B = np.triu(rng.standard_normal((n, n))) + 3 * np.eye(n)
    for name in ("basic", "househt"):
        H, T, Q, Z = _all_oracles(A, B)[name]
        assert np.array_equal(Q, np.eye(n)) and np.array_equal(Z, np.eye(n)), name
        assert np.array_equal(H, A) and np.array_equal(T, B), name


@pytest.mark.parametrize("n", [5, 16, 40])
def test_identity_B_gives_hessenberg_of_A(oracle_lib, n):
    """B = I: T = Q^T Z is triangular and orthogonal, hence diag(+-1), and H
    is the Hessenberg form of A with Q e1 = e1 (compare with LAPACK's
    reduction through scipy, modulo signs)."""
    rng = np.random.default_rng(100 + n)
    A = rng.standard_normal((n, n))
    B = np.eye(n)
    Hs, Qs = sla.hessenberg(A, calc_q=True)
    for name, (H, T, Q, Z) in _all_oracles(A, B).items():
        assert np.allclose(np.abs(np.diag(T)), 1.0, atol=50 * n * EPS), name
        assert np.max(np.abs(np.triu(T, 1))) <= 50 * n * EPS, name
        d = np.sign(np.diag(T))
        assert np.allclose(Z, Q * d[None, :], atol=50 * n * EPS), name
        Hn, Tn, Qn, Zn = checks.sign_normalize(H, T, Q, Z)
        Hsn, _, Qsn, _ = checks.sign_normalize(Hs, np.eye(n), Qs, Qs)
        assert np.allclose(Hn, Hsn, atol=1e-11 * np.linalg.norm(A)), name


# --------------------------------------------------------------------------
# Brute force for n <= 4: det(A - lambda B) = +-det(H - lambda T)
# --------------------------------------------------------------------------
def _det_poly(A, B):
    """Coefficients of det(A - lambda B) (degree n), by exact-ish interpolation
    in 50-digit arithmetic at n+1 points."""
    mpmath.mp.dps = 50
    n = A.shape[0]
    pts = [mpmath.mpf(i) - mpmath.mpf(n) / 2 for i in range(n + 1)]
    vals = []
    for lam in pts:
        M = mpmath.matrix([[mpmath.mpf(float(A[i, j])) - lam * mpmath.mpf(float(B[i, j])) for j in range(n)]
                           for i in range(n)])
        vals.append(mpmath.det(M))
    V = mpmath.matrix([[p ** d for d in range(n + 1)] for p in pts])
    c = mpmath.lu_solve(V, mpmath.matrix(vals))
    return np.array([float(c[i]) for i in range(n + 1)])


@pytest.mark.parametrize("n", [3, 4])
@pytest.mark.parametrize("kind", ["random_qr", "shifted_triu", "graded"])
def test_bruteforce_det_polynomial(oracle_lib, n, kind):
    A, B = pencils.make(kind, n, 31 + n)
    B = np.triu(B)
    ref = _det_poly(A, B)
    scale = np.max(np.abs(ref))
    for name, (H, T, Q, Z) in _all_oracles(A, B, nb=1).items():
        got = _det_poly(H, T)
        sgn = np.sign(np.linalg.det(Q) * np.linalg.det(Z))
        assert np.max(np.abs(sgn * got - ref)) <= 1e-12 * scale, (name, got, ref)
        # and the roots (generalized eigenvalues) agree as multisets
        r1 = np.roots(ref[::-1]) if abs(ref[-1]) > 1e-300 else np.array([])
        r2 = np.roots((sgn * got)[::-1]) if abs(got[-1]) > 1e-300 else np.array([])
        if r1.size and r1.size == r2.size:
            C = np.abs(r1[:, None] - r2[None, :])
            i, j = linear_sum_assignment(C)
            assert np.all(C[i, j] <= 1e-6 * (1 + np.abs(r1[i]))), (name, r1, r2)


# --------------------------------------------------------------------------
# Invariants (i)-(iii) on every workload, three oracles
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind", list(pencils.WORKLOADS))
@pytest.mark.parametrize("n,nb", [(5, 2), (13, 3), (32, 8), (70, 16)])
def test_invariants_all_oracles(oracle_lib, kind, n, nb):
    A, B = pencils.make(kind, n, 1000 + n)
    for name, (H, T, Q, Z) in _all_oracles(A, B, nb=nb).items():
        checks.assert_invariants(A, B, H, T, Q, Z)


@pytest.mark.parametrize("n", [8, 24])
def test_three_oracles_agree_modulo_signs(oracle_lib, n):
    """By the implicit-Q argument (H T^-1 is the Hessenberg form of A B^-1
    with Q e1 = e1) the reductions agree up to diagonal signs."""
    A, B = pencils.random_qr(n, 77 + n)
    outs = {k: checks.sign_normalize(*v) for k, v in _all_oracles(A, B, nb=3).items()}
    ref = outs["basic"]
    for name in ("givens", "househt"):
        for a, b in zip(ref, outs[name]):
            assert np.max(np.abs(a - b)) <= 1e-11, name


def test_generalized_eigenvalues_match_lapack(oracle_lib):
    """Invariant (iv): eig(H, T) = eig(A, B) to 1e-8 relative on a
    well-conditioned pencil (LAPACK dggev through scipy as the library)."""
    n = 64
    A, B = pencils.random_qr(n, 4242)
    ev = sla.eigvals(A, B)
    for name, (H, T, Q, Z) in _all_oracles(A, B, nb=8).items():
        eh = sla.eigvals(H, T)
        C = np.abs(ev[:, None] - eh[None, :]) / (1 + np.abs(ev[:, None]))
        i, j = linear_sum_assignment(C)
        assert np.max(C[i, j]) <= 1e-8, name


# --------------------------------------------------------------------------
# Lemma 2.1: the opposite Householder reflector
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [5, 30, 100])
def test_lemma_2_1_opposite_reflector(oracle_lib, n):
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n))
    e1 = np.eye(n)[:, 0]
    x = np.linalg.solve(B, e1)                 # backward stable solve
    v, beta, _ = hh.house(x)
    C = B - np.outer(B @ v, beta * v)          # step 2
    bn = np.linalg.norm(B)
    below = np.linalg.norm(C[1:, 0])
    assert below <= 10 * n * EPS * bn          # column 1 is reduced ...
    C[1:, 0] = 0.0                             # ... and step 3 zeros it
    Hm = np.eye(n) - beta * np.outer(v, v)
    assert np.linalg.norm(C - B @ Hm) <= 10 * n * EPS * bn


# --------------------------------------------------------------------------
# Sub-steps of Algorithm 1
# --------------------------------------------------------------------------
def _run_one_panel(A, B, nb):
    n = A.shape[0]
    A = np.array(A, copy=True)
    B = np.triu(B)
    P = hh._Panel(n, nb)
    stats = {"ir_steps": 0, "cols_with_ir": 0, "ir_failures": 0}
    tol = 2 * hh.U_ROUND * np.linalg.norm(B)
    A0 = A.copy()
    k, failed = hh._panel(A, B, P, 0, nb, tol, 10, stats, None)
    return A0, A, B, P, k


def test_eq1_compact_wy_growth(oracle_lib):
    """eq. (1) and the S/T growth rules of Sec. 3.2.2b/d:
    prod (I - beta_i u_i u_i^T) = I - U S U^T, same for V and T."""
    n, nb = 40, 8
    A, B = pencils.random_qr(n, 9)
    _, _, _, P, k = _run_one_panel(A, B, nb)
    assert k == nb
    left = np.eye(n)
    right = np.eye(n)
    for i in range(k):
        left = left @ (np.eye(n) - P.S[i, i] * np.outer(P.U[:, i], P.U[:, i]))
        right = right @ (np.eye(n) - P.Tw[i, i] * np.outer(P.V[:, i], P.V[:, i]))
    assert np.allclose(left, np.eye(n) - P.U @ P.S @ P.U.T, atol=1e-14)
    assert np.allclose(right, np.eye(n) - P.V @ P.Tw @ P.V.T, atol=1e-14)
    assert np.allclose(np.triu(P.S), P.S) and np.allclose(np.triu(P.Tw), P.Tw)


def test_panel_reduces_factored_pencil(oracle_lib):
    """After a panel: Y = A V T on rows s+1..n (Sec. 3.2.1), columns s..j-1
    of A are reduced, and B~ = (I-USU^T)^T B (I-VTV^T) is upper triangular
    in its first j+1 columns (Fact 3)."""
    n, nb = 48, 8
    A, B = pencils.random_qr(n, 10)
    A0, A1, B1, P, k = _run_one_panel(A, B, nb)
    U, S, V, Tw = P.U[:, :k], P.S[:k, :k], P.V[:, :k], P.Tw[:k, :k]
    assert np.allclose(P.Y[1:, :k], (A0 @ V @ Tw)[1:], atol=1e-13)
    L = np.eye(n) - U @ S @ U.T
    R = np.eye(n) - V @ Tw @ V.T
    Bt = L.T @ B1 @ R
    assert np.max(np.abs(np.tril(Bt[:, :k + 1], -1))) <= 1e-13
    At = L.T @ A0 @ R
    for c in range(k):
        assert np.max(np.abs(At[c + 2:, c])) <= 1e-13
        assert np.allclose(A1[1:, c], At[1:, c], atol=1e-13)


def test_factored_solve_matches_dense_solve(oracle_lib):
    """Steps 1-4 of Sec. 3.2.2c solve B~22 x = c (compared with a dense
    solve of the explicitly formed B~22 on a well-conditioned pencil)."""
    n, nb = 30, 6
    A, B = pencils.random_qr(n, 12)
    _, _, B1, P, k = _run_one_panel(A, B, nb)
    s, j = 0, k - 1      # reuse the panel factors with kl = k, kr = k - 1
    L = np.eye(n) - P.U[:, :k] @ P.S[:k, :k] @ P.U[:, :k].T
    R = np.eye(n) - P.V[:, :k - 1] @ P.Tw[:k - 1, :k - 1] @ P.V[:, :k - 1].T
    Bt = L.T @ B1 @ R
    c = np.random.default_rng(1).standard_normal(n - j - 1)
    x, sigma = hh._factored_solve(B1, P, s, j, k, k - 1, c)
    xd = np.linalg.solve(Bt[j + 1:, j + 1:], sigma * c)
    assert np.allclose(x, xd, rtol=1e-10, atol=1e-12)
    r = hh._residual(B1, P, s, j, k, k - 1, sigma * c, x)
    assert np.allclose(r, sigma * c - Bt[j + 1:, j + 1:] @ x, atol=1e-13)


@pytest.mark.parametrize("p,k", [(15, 3), (16, 3), (17, 3), (3, 3), (4, 3), (6, 3), (64, 8), (70, 8), (9, 1)])
def test_eq5_eq7_chains_and_windows(oracle_lib, p, k):
    """eq. (5): V2 = Qhat_1..Qhat_r Lhat with Lhat = [0; L1]; eq. (7):
    U2 = Qtil_1..Qtil_r Rtil with Rtil = [R1; 0]; windows per Remark 3.2
    (first window k < k~ <= 2k rows, the rest 2k rows, overlaps of k)."""
    rng = np.random.default_rng(p * 31 + k)
    V2 = rng.standard_normal((p, k))
    wins = hh.ql_windows(p, k)
    assert wins[0][0] == 0 and wins[-1][1] == p
    for (a0, a1), (b0, b1) in zip(wins, wins[1:]):
        assert b0 == a1 - k and b1 - b0 == 2 * k
    assert k < wins[0][1] <= 2 * k or (p <= k and wins[0][1] == p)
    W = V2.copy()
    prod = np.eye(p)
    for (r0, r1) in wins:
        Qm, Lw = hh.ql_factor(W[r0:r1])
        W[r0:r1] = Lw
        G = np.eye(p)
        G[r0:r1, r0:r1] = Qm
        prod = prod @ G
    assert np.all(W[:p - k] == 0.0) and np.all(np.triu(W[p - k:], 1) == 0.0)
    assert np.allclose(prod @ W, V2, atol=1e-13)
    U2 = rng.standard_normal((p, k))
    wins = hh.qr_windows(p, k)
    assert wins[0][1] == p and wins[-1][0] == 0
    W = U2.copy()
    prod = np.eye(p)
    for (r0, r1) in wins:
        Qm, Rw = hh.qr_factor(W[r0:r1])
        W[r0:r1] = Rw
        G = np.eye(p)
        G[r0:r1, r0:r1] = Qm
        prod = prod @ G
    assert np.all(W[k:] == 0.0) and np.all(np.tril(W[:k], -1) == 0.0)
    assert np.allclose(prod @ W, U2, atol=1e-13)


def test_figure_fill_pattern_of_B(oracle_lib):
    """The paper's figure for Sec. 3.3.1c (k = 3, n - j = 15): B(:, j+1:n)
    times the QL chain is block upper Hessenberg with full diagonal blocks;
    also the final shapes of V2 and U2 printed in Sec. 3.3.1b and 3.3.2b."""
    k, p = 3, 15
    rng = np.random.default_rng(3)
    Bt = np.triu(rng.standard_normal((p, p)))
    V2 = rng.standard_normal((p, k))
    for (r0, r1) in hh.ql_windows(p, k):
        Qm, Lw = hh.ql_factor(V2[r0:r1])
        V2[r0:r1] = Lw
        Bt[:, r0:r1] = Bt[:, r0:r1] @ Qm
    assert np.array_equal(Bt != 0.0, _read_pattern("fig_fillinB_k3_p15.txt"))
    assert np.array_equal(V2 != 0.0, _read_pattern("fig_reduceV_k3_p15.txt"))
    U2 = rng.standard_normal((p, k))
    for (r0, r1) in hh.qr_windows(p, k):
        Qm, Rw = hh.qr_factor(U2[r0:r1])
        U2[r0:r1] = Rw
    assert np.array_equal(U2 != 0.0, _read_pattern("fig_reduceU_k3_p15.txt"))


def test_rq_factor(oracle_lib):
    rng = np.random.default_rng(5)
    for k, K in [(3, 6), (3, 4), (4, 4), (1, 2)]:
        X = rng.standard_normal((k, K))
        M, R = hh.rq_factor(X)
        assert np.allclose(M.T @ M, np.eye(K), atol=1e-14)
        assert np.allclose(X @ M, R, atol=1e-13)
        assert np.all(R[:, :K - k] == 0.0) and np.all(np.tril(R[:, K - k:], -1) == 0.0)


# --------------------------------------------------------------------------
# Early absorption (Algorithm 1 "solve failed" branch) and singular B
# --------------------------------------------------------------------------
def test_forced_ir_failures_still_reduce(oracle_lib):
    """Declaring failure at every third column, or making the IR tolerance 0
    (every solve with k >= 1 fails), exercises the undo + early absorption
    path; progress is guaranteed by the k = 0 solve (Sec. 3.2.2c)."""
    A, B = pencils.random_qr(45, 8)
    H, T, Q, Z, st = hh.househt(A, B, nb=8, fail_cols=set(range(1, 45, 3)))
    assert st["ir_failures"] > 5
    checks.assert_invariants(A, B, H, T, Q, Z)
    H, T, Q, Z, st = hh.househt(A, B, nb=8, ir_tol_scale=0.0)
    assert st["ir_failures"] >= 20
    checks.assert_invariants(A, B, H, T, Q, Z)


def test_singular_B_perturbation(oracle_lib):
    """Remark 2.2 / Sec. 3.2.1: exact zeros on B's diagonal are replaced by
    2 u rho ||B||_F; the reduction of the saddle-point pencil of Test Suite 4
    is still backward stable."""
    A, B = pencils.saddle_point(48, 2)
    H, T, Q, Z, st = hh.househt(A, B, nb=8, seed=3)
    assert st["perturbed"] > 0
    checks.assert_invariants(A, B, H, T, Q, Z)
    H, T, Q, Z, npert = oracle.basic_househt(A, B, seed=3)
    checks.assert_invariants(A, B, H, T, Q, Z)


def test_near_infinite_eigenvalues_need_ir(oracle_lib):
    """Sec. 4: pencils with (near-)infinite eigenvalues need iterative
    refinement on a sizeable fraction of columns, random ones almost none."""
    A, B = pencils.near_infinite(128, 5)
    _, _, _, _, st = hh.househt(A, B, nb=16)
    A2, B2 = pencils.random_qr(128, 5)
    _, _, _, _, st2 = hh.househt(A2, B2, nb=16)
    assert st["cols_with_ir"] > 10 * max(st2["cols_with_ir"], 1) or st["ir_failures"] > st2["ir_failures"]
