"""Autotuner of ht_reduce_batched's panel width per size class.

For every size class (orders up to 128, 256, 512 and above) and candidate
panel width, times one ht_reduce_ex call (FP64, Q and Z; best of three) on
pencils of the batched workload's generator at the class's representative
orders, and writes the fastest width per class into csrc/ht_tuned.h, which
the library compiles into ht_reduce_batched.  Needs a GPU.

    python -m paper_1710_08538_gb300.tune_batched [--write]
"""
from __future__ import annotations

import argparse
import json
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CLASSES = [(128, [96, 128]), (256, [192, 256]), (512, [384, 512]), (1 << 30, [768, 1024])]
CANDIDATES = [16, 32, 64]


def measure() -> list[dict]:
    import torch
    import paper_1710_08538_gb300 as ht
    from paper_1710_08538_gb300 import pencils
    out = []
    for nmax, orders in CLASSES:
        times = {}
        for nb in CANDIDATES:
            tot = 0.0
            for i, n in enumerate(orders):
                A, B = pencils.random_qr(n, 7000 + i)
                A0, B0 = ht.colmajor(A), ht.colmajor(B)
                best = None
                for _ in range(3):
                    dA, dB = A0.clone(), B0.clone()
                    dQ, dZ = torch.empty_like(dA), torch.empty_like(dA)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    ht.reduce(dA, dB, dQ, dZ, opts=ht.options(nb=nb))
                    torch.cuda.synchronize()
                    dt = time.perf_counter() - t0
                    best = dt if best is None else min(best, dt)
                tot += best
            times[nb] = tot
        nb_best = min(times, key=times.get)
        out.append({"nmax": nmax, "orders": orders, "seconds_by_nb": times, "nb": nb_best})
    return out


def header(rows: list[dict]) -> str:
    nmax = ", ".join("1 << 30" if r["nmax"] >= (1 << 30) else str(r["nmax"]) for r in rows)
    nbs = ", ".join(str(r["nb"]) for r in rows)
    with open(os.path.join(HERE, "csrc", "ht_tuned.h")) as f:
        src = f.read()
    head = src.split("constexpr int HT_TUNED_NMAX")[0]
    tail = src.split("inline int ht_tuned_nb")[1]
    return (head + f"constexpr int HT_TUNED_NMAX[HT_TUNED_CLASSES] = {{{nmax}}};\n"
            f"constexpr int HT_TUNED_NB[HT_TUNED_CLASSES] = {{{nbs}}};\n\ninline int ht_tuned_nb" + tail)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--write", action="store_true", help="rewrite csrc/ht_tuned.h with the measured widths")
    args = ap.parse_args()
    import __graft_entry__ as g
    g.build()
    rows = measure()
    print(json.dumps(rows), flush=True)
    if args.write:
        text = header(rows)
        with open(os.path.join(HERE, "csrc", "ht_tuned.h"), "w") as f:
            f.write(text)


if __name__ == "__main__":
    main()
