"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each case patches one plausible slip into the oracle -- a dropped term, a wrong factor,
a one-sided overlap, a missing triangular solve, a wrong sign -- and checks that the
pin against the paper's printed eigenvalues (Table t:schwarz, Sec. 3.1) or against a
dense direct solve now fails.  The second half plants slips in every other stage (the
CBD colouring, the clipping of extended boxes, the overlap sum, the 3D weight and
self-cell scaling, Cholesky, the FFT embedding and the PCG recurrences) and runs the
named pin of test_oracle_pins.py that must catch each one.
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


# --- More planted slips, each checked against the pin that should catch it ------------------
#
# Every case below patches one slip into the oracle and runs one of the pins of
# test_oracle_pins.py against it: the pin must now fail.  The unmutated oracle passes the same
# pins in that file.

import itertools  # noqa: E402

import test_oracle_pins as pins  # noqa: E402

_PIN_FAILURES = (AssertionError, O.NotSPD, np.linalg.LinAlgError, FloatingPointError, ValueError)


def _fails(pin, *args):
    try:
        pin(*args)
    except _PIN_FAILURES:
        return True
    return False


def _row(table, dim, n):
    return next(r for r in pins.GOLDEN[table]["rows"] if r["dim"] == dim and r["n"] == n)


def test_checkerboard_colouring_is_caught(monkeypatch):
    # two colours by the parity of k_1 + k_2 instead of the 2^d parity vectors of Sec. 2.3
    orig = O.partition

    def bad(dim, n, m, delta, kind):
        if kind != O.CBD:
            return orig(dim, n, m, delta, kind)
        ext = orig(dim, n, m, delta, O.SCHWARZ)
        col = [sum(k) % 2 for k in itertools.product(range(m), repeat=dim)]
        return [np.unique(np.concatenate([b for b, c in zip(ext, col) if c == cc])) for cc in (0, 1)]
    monkeypatch.setattr(O, "partition", bad)
    assert _fails(pins.test_printed_cbd_table, _row("t_cbd", 2, 16))
    assert _fails(pins.test_cbd_lambda_max_multiplicity)


def test_periodic_extension_is_caught(monkeypatch):
    # extended boxes wrapped around the grid instead of clipped at its boundary
    orig = O.partition

    def bad(dim, n, m, delta, kind):
        if kind != O.SCHWARZ:
            return orig(dim, n, m, delta, kind)
        w = n // m
        out = []
        for k in itertools.product(range(m), repeat=dim):
            mesh = np.meshgrid(*[np.arange(kk * w - delta, (kk + 1) * w + delta) % n for kk in k],
                               indexing="ij")
            idx = np.zeros(mesh[0].shape, dtype=np.int64)
            for a in mesh:
                idx = idx * n + a
            out.append(np.unique(idx))
        return out
    monkeypatch.setattr(O, "partition", bad)
    assert _fails(pins.test_partition_box_geometry)
    assert _fails(pins.test_printed_schwarz_table, _row("t_schwarz", 2, 16))


def test_partition_of_unity_weights_are_caught(monkeypatch):
    # overlap contributions scaled by 1/multiplicity instead of the plain sum of Eq. e:ad
    def bad_pm(factors, blocks, N):
        mult = np.zeros(N)
        for b in blocks:
            mult[b] += 1
        T = np.zeros((N, N))
        for L, b in zip(factors, blocks):
            Linv = scipy.linalg.solve_triangular(L, np.eye(L.shape[0]), lower=True)
            T[np.ix_(b, b)] += (Linv.T @ Linv) / mult[b][:, None]
        return 0.5 * (T + T.T)
    monkeypatch.setattr(O, "preconditioner_matrix", bad_pm)
    assert _fails(pins.test_lambda_max_bounds, 2, 16, 2)
    assert not _matches_print()


def test_3d_weight_h_squared_is_caught(monkeypatch):
    # the 2D quadrature weight h^2 carried over to 3D (Eq. e:a_3d has h^3)
    orig = O.grid_geometry

    def bad(dim, n, convention=O.GRID_TEXT):
        s, o, w, h = orig(dim, n, convention)
        return (s, o, h * h, h) if dim == 3 else (s, o, w, h)
    monkeypatch.setattr(O, "grid_geometry", bad)
    assert _fails(pins.test_printed_schwarz_table, _row("t_schwarz", 3, 4))


def test_3d_self_cell_scaling_is_caught(monkeypatch):
    # the 3D self-cell integral scaled by h^3 (like the weight) instead of h^2
    orig = O.self_cell_integral

    def bad(dim, h):
        if dim == 3:
            return (h ** 3 / (2.0 * math.pi)) * O.inverse_distance_integral_unit_cube()
        return orig(dim, h)
    monkeypatch.setattr(O, "self_cell_integral", bad)
    assert _fails(pins.test_3d_self_cell_equals_direct_cell_quadrature)


def _slipped_cholesky(slip):
    def chol(A):
        A = np.asarray(A, dtype=np.float64)
        nb = A.shape[0]
        L = np.zeros_like(A)
        for j in range(nb):
            s = A[j, j] - L[j, :j] @ L[j, :j]
            if not s > 0.0:
                raise O.NotSPD(j)
            L[j, j] = s if slip == "no_sqrt" else math.sqrt(s)
            if j + 1 < nb:
                # "column": the update reads the (zero) upper triangle L[:j, j] for L[j, :j]
                lj = L[:j, j] if slip == "column" else L[j, :j]
                L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ lj) / L[j, j]
        return L
    return chol


@pytest.mark.parametrize("slip", ["no_sqrt", "column"])
def test_cholesky_slips_are_caught(monkeypatch, slip):
    monkeypatch.setattr(O, "cholesky", _slipped_cholesky(slip))
    assert _fails(pins.test_cholesky_reconstructs_and_matches_lapack)
    assert _fails(pins.test_subdomain_block_cholesky)


def test_fft_embedding_without_negative_offsets_is_caught(monkeypatch):
    # the circulant's first column built from offsets 0..2n-1 instead of 0..n-1, -n+1..-1
    def bad_fft(dim, n, x, convention=O.GRID_TEXT, a_shift=0.0):
        spacing, _, weight, _ = O.grid_geometry(dim, n, convention)
        size = 2 * n
        grids = np.meshgrid(*([np.arange(size, dtype=np.float64)] * dim), indexing="ij")
        r = spacing * np.sqrt(sum(g * g for g in grids))
        zero = r == 0.0
        r[zero] = 1.0
        c = weight * O.kernel(dim, r)
        c[zero] = O.diagonal(dim, n, a_shift)
        xp = np.zeros((size,) * dim)
        xp[tuple(slice(0, n) for _ in range(dim))] = np.asarray(x).reshape((n,) * dim)
        yp = np.fft.irfftn(np.fft.rfftn(c) * np.fft.rfftn(xp), s=(size,) * dim, axes=tuple(range(dim)))
        return yp[tuple(slice(0, n) for _ in range(dim))].reshape(-1)
    monkeypatch.setattr(O, "matvec_fft", bad_fft)
    assert _fails(pins.test_fft_matvec_equals_direct_sum, 2, 16)
    assert _fails(pins.test_printed_iteration_counts, _row("t_it_m48", 2, 16))


def _slipped_pcg(slip):
    """One right-hand side of the oracle's PCG loop with one slip planted."""
    def pcg(matvec, precond, f, tol, max_it, x0=None, history=None):
        f = np.asarray(f, dtype=np.float64)
        if f.ndim != 1:
            raise NotImplementedError("the slipped PCG takes one right-hand side")
        u = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64)
        r = f - matvec(u) if x0 is not None else f.copy()
        fnorm = np.linalg.norm(f)
        p = None
        rho_old = 1.0
        it = 0
        while np.linalg.norm(r) > tol * fnorm and it < max_it:
            z = precond(r)
            rho = r @ (r if slip == "rho_unpreconditioned" else z)
            if p is None:
                p = z.copy()
            else:
                beta = rho_old / rho if slip == "beta_inverted" else rho / rho_old
                p = z + beta * p
            rho_old = rho
            q = matvec(p)
            alpha = rho / (p @ p if slip == "alpha_pp" else p @ q)
            u = u - alpha * p if slip == "update_sign" else u + alpha * p
            r = r - alpha * q
            it += 1
        return u, it, float(np.linalg.norm(r) / fnorm)
    return pcg


@pytest.mark.parametrize("slip", ["beta_inverted", "alpha_pp", "rho_unpreconditioned", "update_sign"])
def test_pcg_slips_are_caught(monkeypatch, slip):
    monkeypatch.setattr(O, "pcg", _slipped_pcg(slip))
    assert (_fails(pins.test_pcg_matches_dense_solve)
            or _fails(pins.test_printed_iteration_counts, _row("t_it_m48", 2, 16)))


def test_unslipped_pcg_restatement_passes_the_pins(monkeypatch):
    # the harness itself: with no slip the restated loop passes the pins the slips fail
    monkeypatch.setattr(O, "pcg", _slipped_pcg(None))
    assert not _fails(pins.test_pcg_matches_dense_solve)
    assert not _fails(pins.test_printed_iteration_counts, _row("t_it_m48", 2, 16))
