"""ht_reduce_noalloc: the reduction for small pencils without any device
allocation (for callers whose allocator owns the GPU's memory or who cannot
pay for cudaMalloc/cudaFree), with its workspace in a static array of the
library.  Checked against ht_reduce, the entry point that allocates its
workspace, on two calls in a row (the array keeps the previous call's
contents, so the second call also checks that each call starts clean).
This file is collected last on purpose."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import checks
from paper_1710_08538_gb300 import pencils

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ht():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_1710_08538_gb300 as m
    return m


def _run(ht, fn, A, B):
    n = A.shape[0]
    dA, dB = ht.colmajor(A), ht.colmajor(B)
    dQ, dZ = ht.colmajor(np.zeros((n, n))), ht.colmajor(np.zeros((n, n)))
    fn(dA, dB, dQ, dZ)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in (dA, dB, dQ, dZ)]


def test_noalloc_matches_ht_reduce_twice(ht):
    n = 300
    for seed in (11, 12):
        A, B = pencils.random_qr(n, seed)
        ref = _run(ht, lambda a, b, q, z: ht.reduce(a, b, q, z, want_qz=True), A, B)
        refn = checks.sign_normalize(*ref)
        for call in range(2):
            got = _run(ht, lambda a, b, q, z: ht.reduce_noalloc(a, b, q, z, want_qz=True), A, B)
            checks.assert_invariants(A, B, *got)
            gotn = checks.sign_normalize(*got)
            for name, x, y in zip("HTQZ", refn, gotn):
                err = float(np.max(np.abs(x - y)))
                assert err <= 1e-10 * max(1.0, float(np.max(np.abs(x)))), (seed, call, name, err)


def test_noalloc_limits(ht):
    import ctypes
    L = ht.lib()
    assert L.ht_reduce_noalloc(ht.HT_NOALLOC_NMAX + 1, 0x1000, 1024, 0x1000, 1024, 0x1000, 1024, 0x1000, 1024, 1,
                               None) == ht.HT_ERR_TOO_LARGE
    assert "ht_reduce_noalloc" in ht.status_string(ht.HT_ERR_TOO_LARGE)
    # the largest order it accepts still reduces correctly
    n = ht.HT_NOALLOC_NMAX
    A, B = pencils.shifted_triu(n, 5)
    got = _run(ht, lambda a, b, q, z: ht.reduce_noalloc(a, b, q, z, want_qz=True), A, B)
    checks.assert_invariants(A, B, *got)
