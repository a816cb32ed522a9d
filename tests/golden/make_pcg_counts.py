"""Write tests/golden/pcg_counts.json: the oracle's PCG iteration counts for the mixed-precision
parity tests, at a tolerance where the count is well conditioned.

Calls only the FP64 oracle (``oracle/ie_oracle.py``) and the seeded input generators.  Run from
the repository root:  python tests/golden/make_pcg_counts.py [--jobs K] [case ...]

Why a tolerance has to be chosen.  PCG minimises the A-norm of the error, not the 2-norm of the
residual, and on these first-kind systems the residual norm of some iterations is extremely
sensitive: perturbing the FP64 Cholesky factors by 1e-13 relative moves single residuals of the
128^2 problem by up to 5x (1.25e-8 -> 6.9e-8) while its neighbours agree to three digits.  Where
the residual crosses the tolerance at or next to such an iteration, the count at that tolerance
is not a property of the method: two correct FP64 implementations can differ by two or three.
The +-1 criterion is therefore checked where the count is well conditioned.

How.  For each case the oracle is run as defined (FP64 factors, triangular solves, FFT matvec)
and, as an ensemble of perturbed but equally valid versions of the same method, with
  * ``p64a``, ``p64b``  the FP64 Cholesky factors perturbed by 2^-44 and 2^-40 relative (random
              signs), and ``mvn64``  every matvec perturbed by 2^-48 max |A x| (random signs): other
              FP64 implementations of the same method (another summation order or FP64 algorithm
              moves a factor of blocks with cond(A_i) ~ 1e4 by up to ~1e-12, and a matvec by
              ~1e-15 of max |A x|), and ``f64n`` the right-hand side perturbed by 2^-50 of its
              largest entry (the seeded Gaussian random fields come out of an FFT, whose last bits
              differ between machines); ``mvd64`` every matvec perturbed by 2^-52 (|A| |x|)_i
              (random signs): the error class of an FP64 evaluation of the defining direct sum
              (Eq. e:dis), whose roundings are at the scale of sum_j |A_ij| |x_j|, not of |(A x)_i|
              (at 1024^2 that is ~1e3 times larger: an exact-entry direct sum, like the tensor-core
              one, lands there, an FFT matvec does not);
  * ``m32``   the exact subdomain inverses A_i^{-1} stored in FP32 (storage rounding only);
  * ``c32``   inverses formed from an FP32 Cholesky of A_i (LAPACK spotrf), stored in FP32;
  * ``c32p``, ``c32q``  the same after symmetric relative perturbations of A_i by 2^-24 and 2^-23
              (other roundings of the same FP32 factor);
  * ``c32w``  W_i = L_i^{-1} of the FP32 factor rounded to FP32 and M_i = W_i^T W_i formed in FP32
              arithmetic (the explicit-inverse pipeline with FP32 rounding at every step);
  * ``c32s``  the same with W_i formed in FP32 arithmetic too (LAPACK strtrs on the FP32 factor);
  * ``c32d``  ``c32`` with the ``mvd64`` matvec (FP32 inverses with a direct-sum-class FP64 matvec);
  * ``mv32``  (3D only) ``c32`` with every matvec perturbed by 2^-23 |A| |x| per entry, the
              error class of an FP32-accumulated matvec;
  * ``mv32e`` (3D only) ``c32`` with a matvec whose entries carry a fixed relative error of up to
              2^-22 per lattice offset (the FP32 entries of a regenerated-entry matvec, the same at
              every product) on top of the ``mv32`` accumulation error.
A candidate tolerance (tried in the order 1e-8, 5e-9, 2e-9, 1e-9, 5e-10, 2e-10, 1e-10) is
*stable* for a column when the FP64-level counts (``fp64``, ``p64a``, ``p64b``, ``mvn64``,
``f64n``, ``mvd64``) span at most two consecutive values: there the FP64 count is a property of the method and not of its
rounding.
The candidate stable for the most columns (ties: the one where the FP64-level counts agree
exactly in the most columns, then the first) is stored with, per column, every member's count and
whether it is stable there; the counts of every member at every candidate are stored too.
The FP32-level members show what FP32 subdomain inverses cost at that tolerance (a few
iterations on the larger grids, even when the inverse is exact before its FP32 rounding).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np
import scipy.linalg

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import ie_oracle as O  # noqa: E402
from paper_2108_12574_gb300 import inputs as I  # noqa: E402

CANDIDATES = [1e-8, 5e-9, 2e-9, 1e-9, 5e-10, 2e-10, 1e-10]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pcg_counts.json")

# name -> (dim, n, m, delta, kind, rhs description); the right-hand sides come from inputs.py
CASES = {
    "ie2d_n64_m4_d1_grf": (2, 64, 4, 1, O.SCHWARZ, ("grf", 0.1, [0])),
    "ie3d_n16_m2_d1_uniform": (3, 16, 2, 1, O.SCHWARZ, ("uniform", None, [0])),
    "ie2d_n96_m6_d2_grf": (2, 96, 6, 2, O.SCHWARZ, ("grf", 0.1, [0])),
    "ie2d_n128_m8_d2_grf": (2, 128, 8, 2, O.SCHWARZ, ("grf", 0.1, [0])),
    "ie2d_n64_m4_d2_cbd_grf": (2, 64, 4, 2, O.CBD, ("grf", 0.1, [0])),
    "ie2d_n512_m32_d2_grf": (2, 512, 32, 2, O.SCHWARZ, ("grf", 0.1, [0])),
    "ie3d_n32_m4_d1_uniform64": (3, 32, 4, 1, O.SCHWARZ, ("uniform", None, list(range(64)))),
    "ie2d_n1024_m64_d2_grf": (2, 1024, 64, 2, O.SCHWARZ, ("grf", 0.05, [0])),
}


def rhs(dim, n, spec):
    kind, ell, seeds = spec
    N = n ** dim
    if kind == "grf":
        return np.stack([I.grf(dim, n, ell, s) for s in seeds], axis=1)
    return I.uniform_rhs_batch(N, seeds)


def count(h, tol):
    idx = np.nonzero(h <= tol)[0]
    return int(idx[0]) + 1 if idx.size else None


def history(matvec, precond, F, tol_min, max_it):
    h = []
    O.pcg(matvec, precond, F, tol_min, max_it, history=h)
    H = np.array(h)
    return H.reshape(H.shape[0], -1)


def fft_matvec_entry_error(dim, n, rel_bits, seed):
    """The oracle's FFT route (circulant embedding of the per-offset entries, Sec. 6) with every
    off-diagonal entry t(d) multiplied by (1 + 2^rel_bits u(|d|)), u uniform in [-1, 1] and fixed
    per offset: a fixed perturbation of A, like FP32 entries regenerated the same way each time."""
    spacing, _, weight, _ = O.grid_geometry(dim, n, O.GRID_TEXT)
    size = 2 * n
    off = np.arange(size)
    off = np.where(off < n, off, off - size)
    grids = np.meshgrid(*([off] * dim), indexing="ij")
    r2 = sum(g.astype(np.float64) ** 2 for g in grids)
    # |d| per axis, symmetric in sign (offset n is never reached by a product of the [0, n) window)
    key = sum(np.minimum(np.abs(g), n - 1) * n ** k for k, g in enumerate(grids))
    u = np.random.default_rng(seed).uniform(-1.0, 1.0, n ** dim)[key]
    zero = r2 == 0.0
    r = spacing * np.sqrt(np.where(zero, 1.0, r2))
    c = weight * O.kernel(dim, r) * (1.0 + 2.0 ** rel_bits * u)
    c[zero] = O.diagonal(dim, n)
    chat = np.fft.rfftn(c)

    def mv(x):
        x = np.asarray(x, dtype=np.float64)
        xm = x.reshape(n ** dim, -1)
        out = np.empty_like(xm)
        for k in range(xm.shape[1]):
            xp = np.zeros((size,) * dim)
            xp[tuple(slice(0, n) for _ in range(dim))] = xm[:, k].reshape((n,) * dim)
            yp = np.fft.irfftn(chat * np.fft.rfftn(xp), s=(size,) * dim, axes=tuple(range(dim)))
            out[:, k] = yp[tuple(slice(0, n) for _ in range(dim))].reshape(-1)
        return out.reshape(x.shape)
    return mv


def inverse_apply(blocks, inverses):
    def ap(r):
        z = np.zeros_like(r)
        for M, b in zip(inverses, blocks):
            z[b] += M @ r[b]
        return z
    return ap


def fp32(a):
    return a.astype(np.float32).astype(np.float64)


def inverse_from_lower(L):
    W = scipy.linalg.solve_triangular(L, np.eye(L.shape[0]), lower=True)
    return W.T @ W


def run_case(name):
    dim, n, m, delta, kind, spec = CASES[name]
    t0 = time.time()
    F = rhs(dim, n, spec)
    blocks = O.partition(dim, n, m, delta, kind)
    A_blocks = O.block_matrices(dim, n, blocks)
    L64 = [O.cholesky(A) for A in A_blocks]
    rng = np.random.default_rng(20210827)
    p64 = []
    for seed, lev in ((1, -44), (2, -40)):
        prng = np.random.default_rng(seed)
        p64.append([L * (1.0 + 2.0 ** lev * np.sign(prng.standard_normal(L.shape))) for L in L64])
    m32, c32, c32p, c32q, c32w, c32s = [], [], [], [], [], []
    for A, L in zip(A_blocks, L64):
        m32.append(fp32(inverse_from_lower(L)))
        L32 = np.linalg.cholesky(A.astype(np.float32)).astype(np.float64)
        c32.append(fp32(inverse_from_lower(L32)))
        W32 = scipy.linalg.solve_triangular(L32, np.eye(L32.shape[0]), lower=True).astype(np.float32)
        c32w.append((W32.T @ W32).astype(np.float64))
        L32f = L32.astype(np.float32)
        W32s = scipy.linalg.solve_triangular(L32f, np.eye(L32f.shape[0], dtype=np.float32), lower=True)
        assert W32s.dtype == np.float32
        c32s.append((W32s.T @ W32s).astype(np.float64))
        E = rng.uniform(-1.0, 1.0, A.shape)
        Ap = A * (1.0 + 2.0 ** -24 * 0.5 * (E + E.T))
        c32p.append(fp32(inverse_from_lower(np.linalg.cholesky(Ap.astype(np.float32)).astype(np.float64))))
        E = rng.uniform(-1.0, 1.0, A.shape)
        Aq = A * (1.0 + 2.0 ** -23 * 0.5 * (E + E.T))
        c32q.append(fp32(inverse_from_lower(np.linalg.cholesky(Aq.astype(np.float32)).astype(np.float64))))
    del A_blocks

    def mv(x):
        return O.matvec_fft(dim, n, x)

    noise_rng = np.random.default_rng(7)

    def mv_noisy(x):
        y = O.matvec_fft(dim, n, x)
        mag = O.matvec_fft(dim, n, np.abs(x))  # |A| |x| (A > 0 entrywise in 3D)
        return y + 2.0 ** -23 * mag * noise_rng.uniform(-1.0, 1.0, y.shape)

    def exact_apply(r):
        return O.apply(L64, blocks, r)

    rng64 = np.random.default_rng(11)

    def mv_fp64_noisy(x):
        y = O.matvec_fft(dim, n, x)
        Y = y.reshape(y.shape[0], -1)
        return y + (2.0 ** -48 * np.abs(Y).max(axis=0) * np.sign(rng64.standard_normal(Y.shape))).reshape(y.shape)

    rngd = np.random.default_rng(19)

    def mv_direct_noisy(x):
        y = O.matvec_fft(dim, n, x)
        mag = np.abs(O.matvec_fft(dim, n, np.abs(x)))  # (|A| |x|)_i, up to the sign of the far-field entries in 2D
        return y + 2.0 ** -52 * mag * np.sign(rngd.standard_normal(y.shape))

    tol_min, max_it = CANDIDATES[-1] / 4, 600
    H = {"fp64": history(mv, exact_apply, F, tol_min, max_it),
         "p64a": history(mv, lambda r: O.apply(p64[0], blocks, r), F, tol_min, max_it),
         "p64b": history(mv, lambda r: O.apply(p64[1], blocks, r), F, tol_min, max_it),
         "mvn64": history(mv_fp64_noisy, exact_apply, F, tol_min, max_it),
         "f64n": history(mv, exact_apply, F + 2.0 ** -50 * np.abs(F).max(axis=0) *
                         np.sign(np.random.default_rng(13).standard_normal(F.shape)), tol_min, max_it),
         "m32": history(mv, inverse_apply(blocks, m32), F, tol_min, max_it),
         "c32": history(mv, inverse_apply(blocks, c32), F, tol_min, max_it),
         "c32p": history(mv, inverse_apply(blocks, c32p), F, tol_min, max_it),
         "c32q": history(mv, inverse_apply(blocks, c32q), F, tol_min, max_it),
         "c32w": history(mv, inverse_apply(blocks, c32w), F, tol_min, max_it),
         "c32s": history(mv, inverse_apply(blocks, c32s), F, tol_min, max_it),
         "mvd64": history(mv_direct_noisy, exact_apply, F, tol_min, max_it),
         "c32d": history(mv_direct_noisy, inverse_apply(blocks, c32), F, tol_min, max_it)}
    if dim == 3:
        H["mv32"] = history(mv_noisy, inverse_apply(blocks, c32), F, tol_min, max_it)
        mv_e = fft_matvec_entry_error(dim, n, -22, 17)

        def mv_entry_noisy(x):
            y = mv_e(x)
            mag = O.matvec_fft(dim, n, np.abs(x))
            return y + 2.0 ** -23 * mag * noise_rng.uniform(-1.0, 1.0, y.shape)
        H["mv32e"] = history(mv_entry_noisy, inverse_apply(blocks, c32), F, tol_min, max_it)
    ncol = F.shape[1]

    def col_hist(key, c):
        h = H[key][:, c]
        return h

    per_tol, exact = {}, {}
    fp64_level = ("fp64", "p64a", "p64b", "mvn64", "f64n", "mvd64")
    for tol in CANDIDATES:
        cols, same = [], 0
        for c in range(ncol):
            k = count(col_hist("fp64", c), tol)
            ens = {key: count(col_hist(key, c), tol) for key in H if key != "fp64"}
            lvl = [k] + [ens[key] for key in fp64_level[1:]]
            ok = all(v is not None for v in lvl) and max(lvl) - min(lvl) <= 1
            same += int(ok and max(lvl) == min(lvl))
            cols.append({"it_fp64": k, "ensemble": ens, "stable": bool(ok)})
        per_tol[tol], exact[tol] = cols, same
    # the first candidate stable for the most columns, and among those the one whose FP64-level
    # counts agree exactly in the most columns
    best = max(CANDIDATES, key=lambda t: (sum(c["stable"] for c in per_tol[t]), exact[t], -CANDIDATES.index(t)))
    entry = {
        "dim": dim, "n": n, "m": m, "delta": delta,
        "kind": {O.JACOBI: "jacobi", O.SCHWARZ: "schwarz", O.CBD: "cbd"}[kind],
        "rhs": {"kind": spec[0], "ell": spec[1], "seeds": spec[2]},
        "tol": best,
        "columns": per_tol[best],
        "stable_columns_per_candidate": {f"{t:.0e}": sum(c["stable"] for c in per_tol[t]) for t in CANDIDATES},
        "counts_per_candidate": {f"{t:.0e}": [{key: count(col_hist(key, c), t) for key in H} for c in range(ncol)]
                                 for t in CANDIDATES},
        "it_fp64_at_1e-8": [count(col_hist("fp64", c), 1e-8) for c in range(ncol)],
        "ensemble_at_1e-8": [{key: count(col_hist(key, c), 1e-8) for key in H if key != "fp64"} for c in range(ncol)],
    }
    if ncol == 1:
        entry["history_fp64"] = [float(f"{v:.4e}") for v in col_hist("fp64", 0)]
    print(f"{name}: tol {best:.0e}, stable {entry['stable_columns_per_candidate']}, "
          f"{time.time() - t0:.0f} s", flush=True)
    return entry


def main(argv):
    """python tests/golden/make_pcg_counts.py [--jobs K] [case ...]: the cases (all by default), K
    of them at a time in separate processes; the file is rewritten as each one finishes."""
    jobs = 1
    if "--jobs" in argv:
        i = argv.index("--jobs")
        jobs = int(argv[i + 1])
        argv = argv[:i] + argv[i + 2:]
    names = argv or list(CASES)
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            data = json.load(fh)
    data["_about"] = ("Oracle PCG iteration counts (FP64, FFT matvec, stop on the recursive residual) "
                      "at a tolerance where the count is well conditioned; written by "
                      "tests/golden/make_pcg_counts.py, which calls only the oracle")

    def store(name, entry):
        data[name] = entry
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=1)

    if jobs <= 1:
        for name in names:
            store(name, run_case(name))
        return
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=jobs, mp_context=mp.get_context("spawn")) as ex:
        futs = {ex.submit(run_case, name): name for name in names}
        for fut in cf.as_completed(futs):
            store(futs[fut], fut.result())


if __name__ == "__main__":
    main(sys.argv[1:])
