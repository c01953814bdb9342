"""The autotuner's table (csrc/ht_tuned.h) on CPU: the committed header
compiles and maps every order to a supported panel width of its class, and
the generator writes a header of the same form for new measurements."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1710_08538_gb300", "csrc")


def _lookup(header_dir, orders, tmp_path):
    src = tmp_path / "t.cc"
    src.write_text('#include <cstdio>\n#include "ht_tuned.h"\nint main() {\n' +
                   "".join(f'  std::printf("%d\\n", ht_tuned_nb({n}));\n' for n in orders) + "  return 0;\n}\n")
    exe = tmp_path / "t"
    subprocess.run(["g++", "-std=c++17", "-I", str(header_dir), str(src), "-o", str(exe)], check=True)
    return [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]


def test_committed_table(tmp_path):
    orders = [3, 64, 128, 129, 256, 257, 512, 513, 1024, 20000]
    got = _lookup(CSRC, orders, tmp_path)
    assert all(nb in (1, 2, 4, 8, 16, 32, 64) for nb in got), got


def test_generator_writes_the_measured_widths(tmp_path):
    from paper_1710_08538_gb300 import tune_batched as tb
    rows = [{"nmax": 128, "nb": 16}, {"nmax": 256, "nb": 32}, {"nmax": 512, "nb": 64}, {"nmax": 1 << 30, "nb": 32}]
    d = tmp_path / "hdr"
    d.mkdir()
    (d / "ht_tuned.h").write_text(tb.header(rows))
    assert _lookup(d, [100, 128, 129, 256, 400, 512, 513, 5000], tmp_path) == [16, 16, 32, 32, 64, 64, 32, 32]
