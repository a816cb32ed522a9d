"""Write tests/golden/rs_counts.json: the FP64 oracle's RS-CBD run at the 2D large size, for
the GPU test at sizes where the oracle takes minutes.

Case "ie2d_n1024_cbd_m128": N = 1024^2 (cell-centred grid), M = 128^2 partitions (N / M = 64,
the paper's choice for CBD, Sec. 5.2), one extra layer of overlap, eps = 1e-3, 64 proxy points,
right-hand side the seeded Gaussian random field of length scale 0.05 (seed 0).  Stored: the
compression levels and last-level DOFs of each colour, the sum of the ranks per colour and
level, and the PCG iteration count to a relative residual of 1e-8 (FFT matvec, Sec. 6).

Calls only the oracle.  Usage: python tests/golden/make_rs_counts.py
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

OUT = os.path.join(HERE, "rs_counts.json")


def main():
    from oracle import ie_oracle as O
    from oracle import rs_oracle as RS
    from paper_2108_12574_gb300 import inputs as I
    dim, n, m, delta, eps, nproxy = 2, 1024, 128, 1, 1e-3, 64
    F = RS.factor(dim, n, m, delta, eps, nproxy)
    f = I.grf(dim, n, 0.05, 0)
    _, it, rel = O.pcg(lambda x: O.matvec_fft(dim, n, x), lambda r: RS.apply(F, r), f, 1e-8, 300)
    out = {"ie2d_n1024_cbd_m128": dict(
        dim=dim, n=n, m=m, delta=delta, eps=eps, nproxy=nproxy, rhs="grf(2, 1024, 0.05, seed 0)", tol=1e-8,
        levels=[len(fc["levels"]) for fc in F], top=RS.top_dofs(F),
        rank_sums=[[int(sum(r)) for r in lv] for lv in RS.ranks(F)], iterations=int(it), recursive_relres=float(rel))}
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
        fh.write("\n")


if __name__ == "__main__":
    main()
