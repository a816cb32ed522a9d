"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each case patches one plausible slip into the oracle -- a dropped term, a wrong factor,
a one-sided overlap, a missing triangular solve, a wrong sign -- and checks that the
pin against the paper's printed eigenvalues (Table t:schwarz, Sec. 3.1) or against a
dense direct solve now fails.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import ie_oracle as O
from paper_2108_12574_gb300 import inputs as I

# Table t:schwarz (Sec. 3.1), 2D, N = 16^2, D = 4^2: Schwarz lambda_max / lambda_min
PRINTED = (8.8046, 0.9112)


def _schwarz_16():
    n = 16
    A = O.dense_matrix(2, n, O.GRID_TABLE)
    blocks = O.partition(2, n, 4, 1, O.SCHWARZ)
    F = O.factor(2, n, blocks, O.GRID_TABLE)
    ev = O.preconditioned_spectrum(A, O.preconditioner_matrix(F, blocks, n * n))
    return ev[-1], ev[0]


def _matches_print():
    try:
        lmax, lmin = _schwarz_16()
    except O.NotSPD:  # the slip made A (or a block) indefinite
        return False
    return abs(lmax - PRINTED[0]) < 1.5e-4 and abs(lmin - PRINTED[1]) < 1.5e-4


def test_unmutated_oracle_matches_print():
    assert _matches_print()


def test_dropped_diagonal_term_is_caught(monkeypatch):
    orig = O.self_cell_integral

    def bad(dim, h):
        if dim == 2:  # drop the pi/2 of int ln(s^2+t^2) over the unit square
            return -(h * h / (4 * math.pi)) * (2 * math.log(h / 2) + math.log(2) - 3)
        return orig(dim, h)
    monkeypatch.setattr(O, "self_cell_integral", bad)
    assert not _matches_print()


def test_log_r_squared_instead_of_log_r_is_caught(monkeypatch):
    monkeypatch.setattr(O, "kernel", lambda dim, r: -np.log(np.asarray(r) ** 2) / (2 * math.pi))
    assert not _matches_print()


def test_one_sided_overlap_is_caught(monkeypatch):
    orig = O.partition

    def bad(dim, n, m, delta, kind):
        # extend only towards larger indices
        w = n // m
        out = []
        for b in orig(dim, n, m, 0, O.JACOBI):
            hi = set()
            for i in b:
                r, c = divmod(int(i), n)
                for dr in range(0, delta + 1):
                    for dc in range(0, delta + 1):
                        if r + dr < n and c + dc < n:
                            hi.add((r + dr) * n + c + dc)
            out.append(np.array(sorted(hi)))
        return out if kind == O.SCHWARZ else orig(dim, n, m, delta, kind)
    monkeypatch.setattr(O, "partition", bad)
    assert not _matches_print()


def test_missing_transpose_solve_is_caught(monkeypatch):
    def bad_pm(factors, blocks, N):
        T = np.zeros((N, N))
        for L, b in zip(factors, blocks):  # L^{-1} alone instead of L^{-T} L^{-1}
            T[np.ix_(b, b)] += scipy.linalg.solve_triangular(L, np.eye(L.shape[0]), lower=True)
        return 0.5 * (T + T.T)
    monkeypatch.setattr(O, "preconditioner_matrix", bad_pm)
    assert not _matches_print()


def test_wrong_sign_operator_is_caught():
    n = 16
    P = O.Problem(2, n, 4, 1, O.SCHWARZ, matvec="dense")
    f = I.uniform_rhs(n * n, 0)
    ref = scipy.linalg.solve(P.A, f, assume_a="pos")

    def bad_matvec(x):  # the kernel's sign flipped
        return -(P.A @ x)
    u, it, rel = O.pcg(bad_matvec, P.apply, f, 1e-10, 60)
    assert not np.linalg.norm(u - ref) < 1e-8 * np.linalg.norm(ref)
