"""The CUDA path's chain geometry (Remark 3.2 windows and the restore blocks,
host/device functions of csrc/ht_common.cuh) against the oracle's, on CPU.

A small host program is compiled from the header with the system C++ compiler
and prints every window and block for a range of (p, k); the oracle computes
the same lists independently from the paper.
"""
import os
import shutil
import subprocess

import pytest

from oracle import househt as hh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r'''
#include <cstdio>
#include "paper_1710_08538_gb300/csrc/ht_common.cuh"
int main() {
  for (int k = 1; k <= KMAX; ++k)
    for (int p = 1; p <= PMAX; ++p) {
      std::printf("P %d %d\n", p, k);
      const int nw = ht_num_windows(p, k);
      for (int i = 0; i < nw; ++i) {
        int a, b, c, d;
        ht_ql_window(p, k, i, &a, &b);
        ht_qr_window(p, k, i, &c, &d);
        std::printf("W %d %d %d %d\n", a, b, c, d);
      }
      const int nr = ht_num_right_blocks(p, k);
      for (int i = 0; i < nr; ++i) { int a, b; ht_right_block(p, k, i, &a, &b); std::printf("R %d %d\n", a, b); }
      const int nl = ht_num_left_blocks(p, k);
      for (int i = 0; i < nl; ++i) { int a, b; ht_left_block(p, k, i, &a, &b); std::printf("L %d %d\n", a, b); }
    }
  return 0;
}
'''


@pytest.fixture(scope="module")
def cuda_geometry(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx or not os.path.isdir(CUDA_INC):
        pytest.skip("no C++ compiler or CUDA headers")
    d = tmp_path_factory.mktemp("geom")
    src, exe = d / "geom.cpp", d / "geom"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-O1", "-std=c++17", "-DKMAX=40", "-DPMAX=200", f"-I{ROOT}", f"-I{CUDA_INC}", str(src),
                    "-o", str(exe)], check=True, capture_output=True, timeout=300)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=300).stdout
    geo = {}
    cur = None
    for line in out.splitlines():
        f = line.split()
        if f[0] == "P":
            cur = {"ql": [], "qr": [], "right": [], "left": []}
            geo[(int(f[1]), int(f[2]))] = cur
        elif f[0] == "W":
            a, b, c, d_ = map(int, f[1:])
            cur["ql"].append((a, b))
            cur["qr"].append((c, d_))
        elif f[0] == "R":
            cur["right"].append((int(f[1]), int(f[2])))
        else:
            cur["left"].append((int(f[1]), int(f[2])))
    return geo


def test_windows_and_blocks_match_the_oracle(cuda_geometry):
    assert len(cuda_geometry) == 40 * 200
    for (p, k), g in cuda_geometry.items():
        assert g["ql"] == [tuple(w) for w in hh.ql_windows(p, k)], ("ql", p, k)
        assert g["qr"] == [tuple(w) for w in hh.qr_windows(p, k)], ("qr", p, k)
        assert g["right"] == [tuple(b) for b in hh.right_blocks(p, k)], ("right", p, k)
        assert g["left"] == [tuple(b) for b in hh.left_blocks(p, k)], ("left", p, k)
