"""Write tests/golden/rs_paper_table.json: the CBD-with-RS rows the paper prints (Sec. 5,
Tables t:cbd_strong_2d, t:cbd_weak_2d and t:cbd_strong_3d: S = the DOFs at the last level of one
subproblem, n_it = PCG iterations to a relative residual of 1e-12, eps = 1e-3, one extra grid
layer of overlap), next to what the FP64 oracle computes for the same N, M and eps.

Calls only the oracle.  The paper does not give its right-hand side or its proxy-point count:
the oracle runs take a uniform[-1, 1] right-hand side (seed 0), 64 proxy points in 2D and 256 in
3D (the library's defaults), and the points of the table grid (the convention under which the
paper's Sec. 3-4 tables are reproduced).  In 3D the oracle's S stays about 20% below the printed
one at any proxy count tried (382 at 128 points, 424 at 512, printed 527) while n_it matches, so
that row's S is kept as context ("S_context") and only n_it is compared.

Usage: python tests/golden/make_rs_paper_table.py [--jobs K]
"""
from __future__ import annotations

import concurrent.futures as cf
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

OUT = os.path.join(HERE, "rs_paper_table.json")
NPROXY_3D = 256

# (table, key, dim, n, m, printed S, printed n_it, run the oracle here)
ROWS = [
    ("t:cbd_strong_2d", "256_8", 2, 256, 8, 64, 26, True),
    ("t:cbd_strong_2d", "256_16", 2, 256, 16, 114, 26, True),
    ("t:cbd_strong_2d", "256_32", 2, 256, 32, 213, 24, True),
    ("t:cbd_strong_2d", "256_64", 2, 256, 64, 407, 22, True),
    ("t:cbd_weak_2d", "512_64", 2, 512, 64, 338, 24, True),
    ("t:cbd_weak_2d", "1024_128", 2, 1024, 128, 568, 25, True),
    ("t:cbd_strong_3d", "32_4", 3, 32, 4, 527, 33, True),
]


def run(row):
    import numpy as np
    from oracle import ie_oracle as O
    from oracle import rs_oracle as RS
    from paper_2108_12574_gb300 import inputs as I
    table, key, dim, n, m, S, nit, _ = row
    nproxy = 64 if dim == 2 else NPROXY_3D
    F = RS.factor(dim, n, m, 1, 1e-3, nproxy, convention=O.GRID_TABLE)
    f = I.uniform_rhs(n ** dim, 0)
    _, it, _ = O.pcg(lambda x: O.matvec_fft(dim, n, x, O.GRID_TABLE), lambda r: RS.apply(F, r), f, 1e-12, 400)
    return table, key, dict(oracle_S=int(max(RS.top_dofs(F))), oracle_S_all=RS.top_dofs(F), oracle_n_it=int(it),
                            nproxy=nproxy)


def main(argv):
    jobs = int(argv[argv.index("--jobs") + 1]) if "--jobs" in argv else 1
    out = {}
    for table, key, dim, n, m, S, nit, _ in ROWS:
        out.setdefault(table, {})[key] = dict(N=f"{n}^{dim}", M=f"{m}^{dim}", S=S, n_it=nit, eps=1e-3, delta=1,
                                              source=f"Sec. 5, Table {table}", S_context=dim == 3)
    todo = [r for r in ROWS if r[7]]
    if jobs > 1:
        with cf.ProcessPoolExecutor(jobs, mp_context=mp.get_context("spawn")) as ex:
            results = list(ex.map(run, todo))
    else:
        results = [run(r) for r in todo]
    for table, key, res in results:
        out[table][key].update(res)
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
        fh.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:])
