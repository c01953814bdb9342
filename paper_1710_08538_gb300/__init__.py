"""Python binding of libht, the GB300 (sm_103a) Householder-based
Hessenberg-triangular reduction of Bujanovic, Karlsson and Kressner
(arXiv 1710.08538).

This module only marshals arguments to the C ABI declared in
``include/ht.h``; every step of the reduction runs in the CUDA library.  If
the library has not been built, every call raises (there is no CPU path).

Matrices are FP64 torch CUDA tensors in column-major layout (stride(0) == 1),
e.g. ``colmajor(np_array)``; A and B are overwritten in place by H and T.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libht.so")

HT_OK = 0
HT_ERR_CUDA = 1001
HT_ERR_NOMEM = 1002
HT_ERR_TIMEOUT = 1003
HT_ERR_NONFINITE = 1004
HT_ERR_NOT_IMPLEMENTED = 1005
HT_ERR_INTERNAL = 1006
HT_ERR_TOO_LARGE = 1007
HT_NOALLOC_NMAX = 512
HT_PREC_FP64 = 0
HT_PREC_EMU = 1

EXPORTED = ["ht_reduce", "ht_reduce_ex", "ht_reduce_general", "ht_reduce_batched", "ht_reduce_noalloc",
            "ht_last_device_status", "ht_finalize", "ht_status_string", "ht_version", "ht_philox4x32_10"]


class HtOptions(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("max_ir", ctypes.c_int), ("ir_tol_scale", ctypes.c_double),
                ("precision", ctypes.c_int), ("emu_slices", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("profile", ctypes.c_int), ("wait_polls", ctypes.c_int), ("preprocess", ctypes.c_int),
                ("emu_check", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


class HtStats(ctypes.Structure):
    _fields_ = [("panels", ctypes.c_int), ("early_absorptions", ctypes.c_int), ("ir_steps", ctypes.c_longlong),
                ("cols_with_ir", ctypes.c_longlong), ("perturbed_pivots", ctypes.c_int),
                ("ms_panel", ctypes.c_double), ("ms_absorb", ctypes.c_double), ("flops_nominal", ctypes.c_double),
                ("ms_by_class", ctypes.c_double * 8), ("flops_by_class", ctypes.c_double * 8),
                ("launches_by_class", ctypes.c_longlong * 8), ("panel_phase_ms", ctypes.c_double * 24),
                ("emu_bwd_est", ctypes.c_double * 2), ("emu_fallback", ctypes.c_int)]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


CLASS_NAMES = ["panel", "chain_factor", "restore", "sweep", "rankk", "gemm", "other", "side"]


class HtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libht error {code}: {msg}")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """Load libht.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libht is not built ({LIB_PATH} missing); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p
        L.ht_reduce.argtypes = [ip, dp, ip, dp, ip, dp, dp, ip, vp]
        L.ht_reduce.restype = ctypes.c_int
        L.ht_reduce_ex.argtypes = [ip, dp, ip, dp, ip, dp, ip, dp, ip, ip, ctypes.POINTER(HtOptions),
                                   ctypes.POINTER(HtStats), vp]
        L.ht_reduce_ex.restype = ctypes.c_int
        L.ht_reduce_general.argtypes = L.ht_reduce_ex.argtypes
        L.ht_reduce_general.restype = ctypes.c_int
        L.ht_reduce_batched.argtypes = [ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p), ip, vp]
        L.ht_reduce_batched.restype = ctypes.c_int
        L.ht_reduce_noalloc.argtypes = [ip, dp, ip, dp, ip, dp, ip, dp, ip, ip, vp]
        L.ht_reduce_noalloc.restype = ctypes.c_int
        L.ht_last_device_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        L.ht_last_device_status.restype = ctypes.c_int
        L.ht_finalize.argtypes = []
        L.ht_finalize.restype = ctypes.c_int
        L.ht_status_string.argtypes = [ctypes.c_int]
        L.ht_status_string.restype = ctypes.c_char_p
        L.ht_philox4x32_10.argtypes = [ip, vp, vp, vp]
        L.ht_philox4x32_10.restype = ctypes.c_int
        L.ht_version.argtypes = []
        L.ht_version.restype = ctypes.c_char_p
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().ht_status_string(code).decode()


def _check(rc: int):
    if rc != HT_OK:
        raise HtError(rc, status_string(rc))


def colmajor(a, device="cuda"):
    """FP64 column-major (stride(0) == 1) torch tensor on `device` from a numpy array."""
    import torch
    a = np.asarray(a, dtype=np.float64)
    n0, n1 = a.shape
    t = torch.empty((n1, n0), dtype=torch.float64, device=device).t()
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return t


def _ld(t) -> int:
    if t.dtype.__repr__() != "torch.float64":
        raise TypeError("libht works on float64 tensors")
    if t.dim() != 2 or t.shape[0] != t.shape[1]:
        raise ValueError("square matrix expected")
    if t.shape[0] > 0 and t.stride(0) != 1:
        raise ValueError("column-major tensor expected (stride(0) == 1); use colmajor()")
    return max(1, t.stride(1) if t.shape[0] > 1 else t.shape[0])


def _stream_ptr(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def options(nb: int = 0, max_ir: int = 0, ir_tol_scale: float = 0.0, precision: int = HT_PREC_FP64,
            emu_slices: int = 0, seed: int = 0, profile: int = 0, wait_polls: int = 0,
            preprocess: int = 0, emu_check: int = 0) -> HtOptions:
    o = HtOptions()
    o.nb, o.max_ir, o.ir_tol_scale, o.precision, o.emu_slices, o.seed = nb, max_ir, ir_tol_scale, precision, \
        emu_slices, seed
    o.profile = profile
    o.wait_polls = wait_polls
    o.preprocess = preprocess
    o.emu_check = emu_check
    return o


def reduce(A, B, Q=None, Z=None, want_qz: bool = True, opts: HtOptions | None = None, stream=None,
           with_stats: bool = False):
    """ht_reduce_ex on torch tensors.  Returns a stats dict when with_stats."""
    n = A.shape[0]
    st = HtStats()
    qp = Q.data_ptr() if (want_qz and Q is not None) else None
    zp = Z.data_ptr() if (want_qz and Z is not None) else None
    ldq = _ld(Q) if (want_qz and Q is not None) else max(1, n)
    ldz = _ld(Z) if (want_qz and Z is not None) else max(1, n)
    rc = lib().ht_reduce_ex(n, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), qp, ldq, zp, ldz, int(want_qz),
                            ctypes.byref(opts) if opts is not None else None,
                            ctypes.byref(st) if with_stats else None, _stream_ptr(stream))
    _check(rc)
    return st.as_dict() if with_stats else None


def reduce_general(A, B, Q=None, Z=None, want_qz: bool = True, opts: HtOptions | None = None, stream=None,
                   with_stats: bool = False):
    """ht_reduce_general (B a general matrix: QR front end, then Algorithm 1) on torch tensors."""
    n = A.shape[0]
    st = HtStats()
    qp = Q.data_ptr() if (want_qz and Q is not None) else None
    zp = Z.data_ptr() if (want_qz and Z is not None) else None
    ldq = _ld(Q) if (want_qz and Q is not None) else max(1, n)
    ldz = _ld(Z) if (want_qz and Z is not None) else max(1, n)
    rc = lib().ht_reduce_general(n, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), qp, ldq, zp, ldz, int(want_qz),
                                 ctypes.byref(opts) if opts is not None else None,
                                 ctypes.byref(st) if with_stats else None, _stream_ptr(stream))
    _check(rc)
    return st.as_dict() if with_stats else None


def reduce_plain(n: int, A_ptr: int, lda: int, B_ptr: int, ldb: int, Q_ptr: int | None, Z_ptr: int | None,
                 want_qz: int, stream_ptr: int) -> int:
    """ht_reduce with raw pointers; returns the status code."""
    return lib().ht_reduce(n, A_ptr, lda, B_ptr, ldb, Q_ptr, Z_ptr, want_qz, stream_ptr)


def reduce_noalloc(A, B, Q=None, Z=None, want_qz: bool = True, stream=None):
    """ht_reduce_noalloc (n <= HT_NOALLOC_NMAX, no device allocation) on torch tensors."""
    n = A.shape[0]
    qp = Q.data_ptr() if (want_qz and Q is not None) else None
    zp = Z.data_ptr() if (want_qz and Z is not None) else None
    ldq = _ld(Q) if (want_qz and Q is not None) else max(1, n)
    ldz = _ld(Z) if (want_qz and Z is not None) else max(1, n)
    _check(lib().ht_reduce_noalloc(n, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), qp, ldq, zp, ldz, int(want_qz),
                                   _stream_ptr(stream)))


def reduce_batched(As, Bs, Qs=None, Zs=None, want_qz: bool = True, stream=None):
    """ht_reduce_batched over lists of column-major tensors."""
    cnt = len(As)
    n = (ctypes.c_int * cnt)(*[a.shape[0] for a in As])
    lda = (ctypes.c_int * cnt)(*[_ld(a) for a in As])
    ldb = (ctypes.c_int * cnt)(*[_ld(b) for b in Bs])
    pa = (ctypes.c_void_p * cnt)(*[a.data_ptr() for a in As])
    pb = (ctypes.c_void_p * cnt)(*[b.data_ptr() for b in Bs])
    pq = (ctypes.c_void_p * cnt)(*[q.data_ptr() for q in Qs]) if want_qz else None
    pz = (ctypes.c_void_p * cnt)(*[z.data_ptr() for z in Zs]) if want_qz else None
    rc = lib().ht_reduce_batched(cnt, n, pa, lda, pb, ldb, pq, pz, int(want_qz), _stream_ptr(stream))
    _check(rc)


def philox4x32_10(blocks, stream=None):
    """Raw Philox4x32-10 blocks computed by the device generator: ``blocks``
    is a list of (counter[4], key[2]); returns a list of output[4]."""
    import torch
    cnt = len(blocks)
    flat = [int(w) & 0xFFFFFFFF for c, k in blocks for w in list(c) + list(k)]
    flat = [w - (1 << 32) if w >= (1 << 31) else w for w in flat]  # the same 32 bits as int32
    dev_in = torch.tensor(flat, dtype=torch.int32, device="cuda")
    dev_out = torch.zeros(4 * cnt, dtype=torch.int32, device="cuda")
    _check(lib().ht_philox4x32_10(cnt, dev_in.data_ptr(), dev_out.data_ptr(), _stream_ptr(stream)))
    torch.cuda.synchronize()
    out = [int(x) & 0xFFFFFFFF for x in dev_out.cpu().tolist()]
    return [out[4 * i:4 * i + 4] for i in range(cnt)]


def finalize():
    _check(lib().ht_finalize())
