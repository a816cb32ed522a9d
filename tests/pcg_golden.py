"""Stored oracle PCG iteration counts (tests/golden/pcg_counts.json) and the checks built on them.

The counts are written by tests/golden/make_pcg_counts.py, which calls only the oracle.  Each
case holds a tolerance at which the oracle's count is well conditioned (see that script), the
FP64 count there per column and whether the perturbed-oracle ensemble agreed on it (``stable``),
and the counts of the FP64 oracle and of the ensemble at the workloads' tolerance 1e-8.
"""
from __future__ import annotations

import json
import os

import numpy as np

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "pcg_counts.json")


def load():
    with open(PATH) as fh:
        return json.load(fh)


def case(name):
    return load()[name]


def rhs(c):
    """The case's right-hand sides (N, ncol) from the seeded generators."""
    from paper_2108_12574_gb300 import inputs as I
    dim, n, spec = c["dim"], c["n"], c["rhs"]
    if spec["kind"] == "grf":
        return np.stack([I.grf(dim, n, spec["ell"], s) for s in spec["seeds"]], axis=1)
    return I.uniform_rhs_batch(n ** dim, spec["seeds"])


def band_at_1e8(c, col=0):
    """[lo, hi]: the iteration counts the FP64 oracle and its perturbed versions reach at 1e-8,
    widened by one.  At 1e-8 the count of these problems is not always well conditioned (the
    residual norm of single iterations is hypersensitive; see make_pcg_counts.py), so a correct
    implementation can land anywhere the ensemble does."""
    vals = [c["it_fp64_at_1e-8"][col]] + [v for v in c["ensemble_at_1e-8"][col].values() if v is not None]
    return min(vals) - 1, max(vals) + 1


def check_counts_at_stable_tol(c, iterations):
    """+-1 of the oracle's FP64 count at the case's stable tolerance for every column the ensemble
    agreed on; the others within the ensemble's counts +-1.  ``iterations``: per-column GPU counts."""
    bad = []
    for k, (it, col) in enumerate(zip(iterations, c["columns"])):
        ref = col["it_fp64"]
        if col["stable"]:
            ok = abs(it - ref) <= 1
        else:
            vals = [ref] + [v for v in col["ensemble"].values() if v is not None]
            ok = min(vals) - 1 <= it <= max(vals) + 1
        if not ok:
            bad.append((k, it, ref, col["stable"]))
    assert not bad, f"tol {c['tol']:.0e}: (column, GPU, oracle, stable) {bad}"
