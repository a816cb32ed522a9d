"""Stored oracle PCG iteration counts (tests/golden/pcg_counts.json) and the checks built on them.

The counts are written by tests/golden/make_pcg_counts.py, which calls only the oracle.  Each
case holds a tolerance at which the oracle's FP64 count is well conditioned (its rounding-level
variants ``p64a``, ``p64b``, ``mvn64``, ``f64n``, ``mvd64`` span at most two consecutive counts there), and per column the FP64
count, every ensemble member's count and whether the column is stable.  The FP32-level members
(``m32``, ``c32``, ``c32p``, ``c32q``, ``c32w``, ``c32s``, ``c32d``; ``mv32``, ``mv32e`` in 3D) are the oracle with FP32 subdomain inverses
(and, for ``mv32``, an FP32-class matvec): the counts a mixed-precision implementation of the
method can be expected to reach.
"""
from __future__ import annotations

import json
import os

import numpy as np

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "pcg_counts.json")
FP64_LEVEL = ("p64a", "p64b", "mvn64", "f64n", "mvd64")


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


def _vals(members):
    return [v for v in members.values() if v is not None]


# How far above the FP32-level members a path with the library's FP32 explicit inverses may land.
# Those inverses come from tensor-core GEMMs with FP32 accumulation, W = L^{-1} stored in FP32 and
# M = W^T W formed in FP32: measured on single blocks, ||I - A_i M_i|| is 1.7x (2D, 256 points)
# and 6x (3D, 512 points) that of the c32s member (FP32 LAPACK factor, W and M in FP32
# arithmetic) and 45x / 120x that of c32; the ensemble brackets the count from below, and such an
# inverse costs up to two iterations more than its worst member (measured on every stored case).
FP32_INVERSE_EXCESS = 2


def band_at_1e8(c, col=0):
    """[lo, hi]: the counts the FP64 oracle and every perturbed version reach at 1e-8, one below
    the lowest and FP32_INVERSE_EXCESS above the highest.  At 1e-8 the count of these problems is
    not always well conditioned (the residual norm of single iterations is hypersensitive; see
    make_pcg_counts.py), and FP32 subdomain inverses cost iterations, so a correct mixed-precision
    implementation lands anywhere the ensemble does, or up to FP32_INVERSE_EXCESS above it."""
    vals = [c["it_fp64_at_1e-8"][col]] + _vals(c["ensemble_at_1e-8"][col])
    return min(vals) - 1, max(vals) + FP32_INVERSE_EXCESS


def fp64_level_range(c, col=0):
    """[lo, hi] of the FP64-level counts (the oracle and its rounding-level variants) at the
    stable tolerance: the spread of counts that correct FP64 implementations reach there."""
    e = c["columns"][col]
    vals = [e["it_fp64"]] + [e["ensemble"][k] for k in FP64_LEVEL if e["ensemble"].get(k) is not None]
    return min(vals), max(vals)


def check_fp64_counts(c, iterations):
    """FP64-class paths (FP64 factors, an FP64-class matvec): within the oracle's FP64-level counts
    +-1 at the stable tolerance, in every stable column."""
    bad = []
    for k, (it, col) in enumerate(zip(iterations, c["columns"])):
        lo, hi = fp64_level_range(c, k)
        if col["stable"] and not (lo - 1 <= it <= hi + 1):
            bad.append((k, it, (lo, hi)))
    assert not bad, f"tol {c['tol']:.0e}: (column, GPU, oracle FP64-level range) {bad}"


def check_mixed_counts(c, iterations):
    """Paths with the library's FP32 subdomain inverses: within the counts of the whole ensemble
    (FP64-level and FP32-level members) at the stable tolerance, from one below the lowest to
    FP32_INVERSE_EXCESS above the highest, in every column."""
    bad = []
    for k, (it, col) in enumerate(zip(iterations, c["columns"])):
        vals = [col["it_fp64"]] + _vals(col["ensemble"])
        if not (min(vals) - 1 <= it <= max(vals) + FP32_INVERSE_EXCESS):
            bad.append((k, it, (min(vals), max(vals))))
    assert not bad, f"tol {c['tol']:.0e}: (column, GPU, ensemble range) {bad}"
