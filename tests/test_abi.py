"""The C ABI without a GPU: every function declared in include/ht.h is
exported by libht.so, and host-side argument errors come back synchronously
as LAPACK-style negative codes before any CUDA call."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def htlib():
    import __graft_entry__ as g
    from paper_1710_08538_gb300 import _build
    _build.build()
    import paper_1710_08538_gb300 as ht
    return ht


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "ht.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(ht_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("ht_reduce", "ht_reduce_batched", "ht_reduce_ex", "ht_last_device_status", "ht_finalize"):
        assert required in names


def test_every_declared_symbol_is_exported(htlib):
    L = htlib.lib()
    for name in _declared_functions():
        assert hasattr(L, name), name
    assert set(htlib.EXPORTED) >= set(_declared_functions())


def test_version_and_status_strings(htlib):
    assert b"sm_103a" in htlib.lib().ht_version()
    assert htlib.status_string(0) == "success"
    assert "NaN" in htlib.status_string(htlib.HT_ERR_NONFINITE)
    assert htlib.status_string(-3) == "invalid argument"


@pytest.mark.parametrize("args,code", [
    ((-1, 8, 8, 1), -1),    # n < 0
    ((10, 5, 10, 1), -3),   # lda < n
    ((10, 10, 9, 1), -5),   # ldb < n
])
def test_argument_errors(htlib, args, code):
    n, lda, ldb, want = args
    fake = 0x1000  # never dereferenced: the arguments are rejected first
    rc = htlib.lib().ht_reduce(n, fake, lda, fake, ldb, fake, fake, want, None)
    assert rc == code


def test_null_pointers_rejected(htlib):
    L = htlib.lib()
    assert L.ht_reduce(4, None, 4, 0x1000, 4, 0x1000, 0x1000, 1, None) == -2
    assert L.ht_reduce(4, 0x1000, 4, None, 4, 0x1000, 0x1000, 1, None) == -4
    assert L.ht_reduce(4, 0x1000, 4, 0x1000, 4, None, 0x1000, 1, None) == -6
    assert L.ht_reduce_batched(-1, None, None, None, None, None, None, None, 0, None) == -1


def test_options_rejected_before_device_work(htlib):
    opts = htlib.options(nb=128)
    L = htlib.lib()
    import ctypes
    rc = L.ht_reduce_ex(4, 0x1000, 4, 0x1000, 4, 0x1000, 4, 0x1000, 4, 1, ctypes.byref(opts), None, None)
    assert rc == htlib.HT_ERR_NOT_IMPLEMENTED


def test_last_device_status_is_per_stream(htlib):
    """ht_last_device_status reads the status of the last call on the given
    stream; a stream without calls reports HT_OK (no CUDA call is made)."""
    import ctypes
    st = ctypes.c_int(-7)
    assert htlib.lib().ht_last_device_status(ctypes.c_void_p(0x7777), ctypes.byref(st)) == htlib.HT_OK
    assert st.value == htlib.HT_OK
    assert htlib.lib().ht_last_device_status(None, None) == -2


def test_struct_layouts_match_the_header(htlib, tmp_path):
    """The Python binding's ht_options and ht_stats have the sizes and field
    offsets of the C declarations in include/ht.h (compiled here with gcc)."""
    import ctypes
    import subprocess
    src = tmp_path / "sz.c"
    fields_o = ["nb", "max_ir", "ir_tol_scale", "precision", "emu_slices", "seed", "profile", "wait_polls",
                "preprocess", "emu_check"]
    fields_s = ["panels", "ir_steps", "ms_panel", "flops_nominal", "ms_by_class", "launches_by_class",
                "panel_phase_ms", "emu_bwd_est", "emu_fallback"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ht.h"', "int main(void) {",
             '  printf("%zu %zu\\n", sizeof(ht_options), sizeof(ht_stats));']
    lines += [f'  printf("%zu\\n", offsetof(ht_options, {f}));' for f in fields_o]
    lines += [f'  printf("%zu\\n", offsetof(ht_stats, {f}));' for f in fields_s]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(htlib.HtOptions) and out[1] == ctypes.sizeof(htlib.HtStats)
    got = [getattr(htlib.HtOptions, f).offset for f in fields_o] + [getattr(htlib.HtStats, f).offset for f in fields_s]
    assert out[2:] == got
