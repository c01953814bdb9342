"""CPU oracle for the Householder-based Hessenberg-triangular reduction
(Bujanovic, Karlsson, Kressner, arXiv 1710.08538).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library and never calls it.

Modules
  ``ht_oracle.c``  plain C: Householder reflector (Sec. 2.1), Algorithm 2
                   (BasicHouseHT, Appendix A), unblocked Givens HT reduction
                   (Moler-Stewart, Sec. 1/4), Philox4x32-10 normal samples
                   (Remark 2.2 perturbation).
  ``househt``      numpy, Algorithm 1 (HouseHT) step by step: panel
                   reduction (Sec. 3.2), absorption (Sec. 3.3).
  ``checks``       the invariants the paper's Sec. 4 and Appendix A fix.

Parity pins live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ht_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``ht_oracle.c`` into ``oracle/_build/liboracle.so`` (plain gcc -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_house.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, dp]
            lib.oracle_house.restype = None
            lib.oracle_basic_househt.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int,
                                                 dp, ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]
            lib.oracle_basic_househt.restype = ctypes.c_int
            lib.oracle_givens_ht.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int,
                                             dp, ctypes.c_int]
            lib.oracle_givens_ht.restype = ctypes.c_int
            lib.oracle_philox_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
            lib.oracle_philox_normal.restype = ctypes.c_double
            lib.oracle_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                                 ctypes.POINTER(ctypes.c_uint32)]
            lib.oracle_philox4x32_10.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fortran(a) -> np.ndarray:
    return np.array(a, dtype=np.float64, order="F", copy=True)


def house(x):
    """Householder reflector of Sec. 2.1 with the DLARFG sign rule.

    Returns ``(v, beta, alpha)`` with ``v[0] == 1`` and
    ``(I - beta v v^T) x = alpha e1``; ``beta == 0`` when ``x[1:]`` is exactly 0.
    """
    v = np.array(x, dtype=np.float64, copy=True)
    beta = ctypes.c_double()
    alpha = ctypes.c_double()
    _load().oracle_house(v.size, _ptr(v), 1, ctypes.byref(beta), ctypes.byref(alpha))
    v[0] = 1.0
    return v, beta.value, alpha.value


def basic_househt(A, B, seed: int = 0):
    """Algorithm 2 (BasicHouseHT, Appendix A).  Returns ``(H, T, Q, Z, n_perturbed)``."""
    H = _fortran(A)
    T = _fortran(B)
    n = H.shape[0]
    Q = np.zeros((n, n), order="F")
    Z = np.zeros((n, n), order="F")
    npert = ctypes.c_int(0)
    ld = max(1, n)
    rc = _load().oracle_basic_househt(n, _ptr(H), ld, _ptr(T), ld, _ptr(Q), ld, _ptr(Z), ld,
                                      ctypes.c_uint64(seed), ctypes.byref(npert))
    if rc != 0:
        raise RuntimeError(f"oracle_basic_househt failed: {rc}")
    return H, T, Q, Z, npert.value


def givens_ht(A, B):
    """Unblocked Givens (Moler-Stewart) HT reduction.  Returns ``(H, T, Q, Z)``."""
    H = _fortran(A)
    T = _fortran(B)
    n = H.shape[0]
    Q = np.zeros((n, n), order="F")
    Z = np.zeros((n, n), order="F")
    ld = max(1, n)
    rc = _load().oracle_givens_ht(n, _ptr(H), ld, _ptr(T), ld, _ptr(Q), ld, _ptr(Z), ld)
    if rc != 0:
        raise RuntimeError(f"oracle_givens_ht failed: {rc}")
    return H, T, Q, Z


def philox_normal(seed: int, column: int, index: int) -> float:
    """N(0,1) sample used for the singular-B perturbation (Remark 2.2)."""
    return _load().oracle_philox_normal(ctypes.c_uint64(seed), ctypes.c_uint32(column), ctypes.c_uint32(index))


def philox4x32_10(counter, key):
    """Raw Philox4x32-10 block (Salmon et al. 2011) for the known-answer pin."""
    c = (ctypes.c_uint32 * 4)(*counter)
    k = (ctypes.c_uint32 * 2)(*key)
    out = (ctypes.c_uint32 * 4)()
    _load().oracle_philox4x32_10(c, k, out)
    return [int(x) for x in out]
