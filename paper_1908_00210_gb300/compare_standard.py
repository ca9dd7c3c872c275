"""GDI (Algorithm 3) against the paper's standard annealer (Algorithm 2) on the GPU, by graph size.

Both run on the CTA-resident path of libgdi.so with the paper's P_f schedule: GDI reads the
decoupled magnetisation G, the standard annealer sums all n spins for every spin's balance term
(GDI_FLAG_STANDARD; its P_f five times GDI's, the paper's tuning note).  Graphs are shaped like the
paper's Table 1 inputs: Erdos-Renyi with density 1-2 % for n <= 2000 and 4-regular tori up to
20,000 vertices.  For each graph and method: GPU milliseconds of the anneal kernel, raw |G| and the
repaired cut (median over the replicas).

    python -m paper_1908_00210_gb300.compare_standard [--sweeps 1000] [--replicas 8]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1908_00210_gb300 import _binding as B  # noqa: E402


def graphs():
    from gdi_synth import erdos_renyi, torus2d
    out = [(f"ER n=800 p=0.02", erdos_renyi(800, 0.02, 1801), None),
           (f"ER n=1000 p=0.01", erdos_renyi(1000, 0.01, 1802), None),
           (f"ER n=2000 p=0.01", erdos_renyi(2000, 0.01, 1803), None)]
    for L in (32, 50, 71, 100, 141):
        t = torus2d(L, 1900 + L, signed=False)
        out.append((f"torus {L}x{L} (n={L * L})", t, t.color))
    return out


def run(sweeps: int, replicas: int, pf0: float, pf1: float, W: int):
    import torch
    rows = []
    for name, g, color in graphs():
        row = {"graph": name, "n": g.n, "nnz": g.nnz}
        for method, flags, scale in (("gdi", 0, 1.0), ("standard", B.GDI_FLAG_STANDARD, 5.0)):
            ann = B.Annealer(g, A=1, B=4, W=W, replicas=replicas, color=color)
            ann.configure(path=B.GDI_PATH_CTA)
            sch = B.Schedule(sweeps=sweeps, mode=B.GDI_PAPER_PF, pf0=min(0.49, pf0 * scale),
                             pf1=min(0.49, pf1 * scale))
            ann.anneal(sch, 1, flags=flags)           # warm-up
            ann.results()
            ann.anneal(sch, 2, flags=flags)
            res = ann.results()
            ms, _ = ann.kernel_ms()
            ann.close()
            row[method] = {"kernel_ms": ms, "raw_absG_median": float(np.median(np.abs(res["raw_G"][0]))),
                           "cut_median": float(np.median(res["final_cut"][0]))}
        row["speedup"] = row["standard"]["kernel_ms"] / row["gdi"]["kernel_ms"]
        rows.append(row)
        print(json.dumps(row), flush=True)
    torch.cuda.synchronize()
    return rows


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--sweeps", type=int, default=200)
    ap.add_argument("--replicas", type=int, default=8)
    ap.add_argument("--pf0", type=float, default=0.02)
    ap.add_argument("--pf1", type=float, default=0.0002)
    ap.add_argument("--W", type=int, default=0, help="window (0 = whole colour class)")
    args = ap.parse_args()
    run(args.sweeps, args.replicas, args.pf0, args.pf1, args.W)


if __name__ == "__main__":
    main()
