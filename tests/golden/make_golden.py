"""Writes tests/golden/*.json from the FP64 oracle only (no CUDA path).

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle  # noqa: E402
from paper_1805_06124_gb300 import synth  # noqa: E402


def main():
    N, M, seed, tol, kmax = 64, 96, 1, 1e-10, 96
    S = synth.chirps(N, M, seed)
    r = oracle.rb_greedy(S, tol, kmax)
    out = dict(
        what="RB-greedy (Alg. 3) on the synthetic chirp family, FP64 oracle",
        N=N, M=M, seed=seed, tol=tol, kmax=kmax, status=int(r["status"]), k=int(r["k"]),
        pivots=[int(p) for p in r["pivots"]],
        err_curve=[float(e) for e in r["err_curve"]],
        rdiag=[float(d) for d in r["rdiag"]],
    )
    with open(os.path.join(HERE, "chirp_64x96_seed1.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
