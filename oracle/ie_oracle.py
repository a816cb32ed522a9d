"""Plain FP64 CPU oracle for PCG on the dense IE system with the additive overlapping
domain-decomposition preconditioner (Chen & Biros, arXiv 2108.12574).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this module.  It shares no code
with the CUDA library in ``paper_2108_12574_gb300/`` and never imports it.

Every function follows the paper's definition directly, in FP64, with no blocking or
reordering beyond what the definition states.  Library primitives used as single
steps: numpy matmul / dot, numpy FFT (the paper's own matvec route, Sec. 6), scipy
triangular solves and symmetric eigenvalues.  The O(N^2) direct sum is the plain
double loop of ``direct_sum.c``.

Readings of the paper where it is silent or inconsistent (each also listed in the
design notes):
  * Sec. 2.1 says "trapezoidal rule" but the nodes are cell centres with equal weights
    h^d; the weights of Eq. e:a_2d are used as printed (midpoint rule).
  * The diagonal "proper singular quadrature" is the exact self-cell integral, in
    closed form (``self_cell_integral``).
  * The 2D tables of Sec. 3-4 are reproduced only when the points sit on
    linspace(0, 1, n) (spacing 1/(n-1)) with weight 1/n^2 and the h = 1/n diagonal;
    that is ``GRID_TABLE``.  The text's cell-centred grid is ``GRID_TEXT``, the default.
  * Partitions are extended by ``delta`` grid layers and clipped at the boundary
    ("when possible", Sec. 2.2); index sets are in ascending global order.
  * PCG starts from x0 = 0 unless given, stops on the recursive residual
    ||r||_2 <= tol ||f||_2, and counts iterations as products q = A p.
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
import subprocess
import threading

import numpy as np
import scipy.linalg

GRID_TEXT = 0
GRID_TABLE = 1
JACOBI = 0
SCHWARZ = 1
CBD = 2


class NotSPD(ArithmeticError):
    """A non-positive pivot met in the Cholesky factorization."""

    def __init__(self, column):
        super().__init__(f"non-positive pivot at column {column}")
        self.column = column


# ---------------------------------------------------------------------------
# Discretization, Sec. 2.1 (Eqs. e:ie, e:k, e:a_2d, e:a_3d)
# ---------------------------------------------------------------------------

def kernel(dim: int, r):
    """Laplace fundamental solution K(r), Eq. e:k."""
    r = np.asarray(r, dtype=np.float64)
    if dim == 2:
        return -np.log(r) / (2.0 * math.pi)
    if dim == 3:
        return 1.0 / (4.0 * math.pi * r)
    raise ValueError("dim must be 2 or 3")


def log_integral_unit_square() -> float:
    """int_{[0,1]^2} ln(s^2 + t^2) ds dt = ln 2 - 3 + pi/2 (closed form)."""
    return math.log(2.0) - 3.0 + math.pi / 2.0


def inverse_distance_integral_unit_cube() -> float:
    """int_{[0,1]^3} 1/|x| dx = 3 ln(1 + sqrt 3) - (3/2) ln 2 - pi/4 (closed form)."""
    return 3.0 * math.log(1.0 + math.sqrt(3.0)) - 1.5 * math.log(2.0) - math.pi / 4.0


def self_cell_integral(dim: int, h: float) -> float:
    """Diagonal entry of Eqs. e:a_2d / e:a_3d: the integral of K over the h^d cell
    centred at the origin.

    2D: by symmetry 4 * int_{[0,h/2]^2} -(1/4pi) ln(x^2+y^2); scaling by a = h/2 gives
        -(h^2 / (4 pi)) (2 ln(h/2) + ln 2 - 3 + pi/2).
    3D: 8 * int_{[0,h/2]^3} 1/(4 pi |x|) = (h^2 / (2 pi)) * J, J = int_{[0,1]^3} 1/|x|.
    """
    if dim == 2:
        return -(h * h / (4.0 * math.pi)) * (2.0 * math.log(h / 2.0) + log_integral_unit_square())
    if dim == 3:
        return (h * h / (2.0 * math.pi)) * inverse_distance_integral_unit_cube()
    raise ValueError("dim must be 2 or 3")


def grid_geometry(dim: int, n: int, convention: int = GRID_TEXT):
    """(spacing, offset, weight, h) of the collocation grid.

    GRID_TEXT : p_j = h (j - 1/2), j = 1..n, h = 1/n (Sec. 2.1); weight h^d.
    GRID_TABLE: p_j = (j - 1)/(n - 1), weight (1/n)^d -- the convention under which the
                paper's 2D eigenvalue tables are reproduced (see module docstring).
    """
    h = 1.0 / n
    if convention == GRID_TEXT:
        return h, 0.5 * h, h ** dim, h
    if convention == GRID_TABLE:
        return 1.0 / (n - 1), 0.0, h ** dim, h
    raise ValueError("unknown grid convention")


def lattice(dim: int, n: int) -> np.ndarray:
    """Integer multi-indices (N, dim), row-major, last coordinate fastest."""
    axes = np.meshgrid(*([np.arange(n)] * dim), indexing="ij")
    return np.stack([a.reshape(-1) for a in axes], axis=1)


def points(dim: int, n: int, convention: int = GRID_TEXT) -> np.ndarray:
    """Collocation points (N, dim) in FP64."""
    spacing, offset, _, _ = grid_geometry(dim, n, convention)
    return offset + spacing * lattice(dim, n).astype(np.float64)


def diagonal(dim: int, n: int, a_shift: float = 0.0) -> float:
    """A_ii: the self-cell integral with h = 1/n, plus the second-kind shift a (Eq. e:int)."""
    return self_cell_integral(dim, 1.0 / n) + a_shift


def dense_matrix(dim: int, n: int, convention: int = GRID_TEXT, a_shift: float = 0.0,
                 index=None) -> np.ndarray:
    """A (or its principal sub-block A[index, index], Eq. e:ai) as a dense FP64 array."""
    _, _, weight, _ = grid_geometry(dim, n, convention)
    p = points(dim, n, convention)
    if index is not None:
        p = p[np.asarray(index)]
    diff = p[:, None, :] - p[None, :, :]
    r = np.sqrt((diff * diff).sum(axis=2))
    np.fill_diagonal(r, 1.0)
    A = weight * kernel(dim, r)
    np.fill_diagonal(A, diagonal(dim, n, a_shift))
    return A


# ---------------------------------------------------------------------------
# Matvec: plain direct sum (the definition) and the FFT route of Sec. 6
# ---------------------------------------------------------------------------

_LIB = None
_LIB_LOCK = threading.Lock()
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct_sum.c")
_SO = os.path.join(_HERE, "_build", "liboracle_direct.so")


def build_native(force: bool = False) -> str:
    """Compile direct_sum.c (plain -O2 FP64, OpenMP) into oracle/_build/."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _LIB
    with _LIB_LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build_native())
            lib.oracle_matvec_rows.restype = ctypes.c_int
            lib.oracle_matvec_rows.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                ctypes.c_double, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                ctypes.c_longlong, ctypes.c_void_p]
            _LIB = lib
    return _LIB


def matvec_direct(dim: int, n: int, x: np.ndarray, rows=None, convention: int = GRID_TEXT,
                  a_shift: float = 0.0) -> np.ndarray:
    """Rows of A x by the plain O(N) sum per row (Eq. e:dis).

    x: (N,) or (N, k).  Returns (len(rows),) or (len(rows), k); all rows if rows is None.
    """
    N = n ** dim
    x = np.asarray(x, dtype=np.float64)
    vec = x.ndim == 1
    xm = np.ascontiguousarray(x.reshape(N, -1))
    k = xm.shape[1]
    rows = np.arange(N, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    y = np.empty((rows.size, k), dtype=np.float64)
    spacing, offset, weight, _ = grid_geometry(dim, n, convention)
    st = _lib().oracle_matvec_rows(dim, n, spacing, offset, weight, diagonal(dim, n, a_shift),
                                   xm.ctypes.data, k, rows.ctypes.data, rows.size, y.ctypes.data)
    if st != 0:
        raise ValueError("oracle_matvec_rows: bad arguments")
    return y[:, 0] if vec else y


def matvec_fft(dim: int, n: int, x: np.ndarray, convention: int = GRID_TEXT,
               a_shift: float = 0.0) -> np.ndarray:
    """A x through the FFT (Sec. 6: the paper's matvec).

    A_ij depends only on the integer offset i - j on the uniform grid, so A is
    block-Toeplitz with Toeplitz blocks; it is embedded in a circulant on the (2n)^d
    periodic grid and applied by FFT.  x: (N,) or (N, k).
    """
    N = n ** dim
    x = np.asarray(x, dtype=np.float64)
    vec = x.ndim == 1
    xm = x.reshape(N, -1)
    spacing, _, weight, _ = grid_geometry(dim, n, convention)
    size = 2 * n
    off = np.arange(size)
    off = np.where(off < n, off, off - size).astype(np.float64)  # offset n is never used
    grids = np.meshgrid(*([off] * dim), indexing="ij")
    r = spacing * np.sqrt(sum(g * g for g in grids))
    zero = (r == 0.0)
    r[zero] = 1.0
    c = weight * kernel(dim, r)
    c[zero] = diagonal(dim, n, a_shift)
    chat = np.fft.rfftn(c)
    out = np.empty_like(xm)
    for k in range(xm.shape[1]):
        xp = np.zeros((size,) * dim)
        xp[tuple(slice(0, n) for _ in range(dim))] = xm[:, k].reshape((n,) * dim)
        yp = np.fft.irfftn(chat * np.fft.rfftn(xp), s=(size,) * dim, axes=tuple(range(dim)))
        out[:, k] = yp[tuple(slice(0, n) for _ in range(dim))].reshape(-1)
    return out[:, 0] if vec else out


# ---------------------------------------------------------------------------
# Domain decomposition, Sec. 2.2-2.3 (Eqs. e:dd, e:first, e:cbd, e:second; Table t:dd)
# ---------------------------------------------------------------------------

def partition(dim: int, n: int, m: int, delta: int, kind: int):
    """Index sets I_i of the subdomains, each in ascending global order.

    The grid is split into M = m^d boxes of w = n/m cells (Eq. e:dd).  JACOBI: the boxes
    themselves.  SCHWARZ: every box extended by ``delta`` layers in every direction,
    clipped to the grid (Eq. e:first, D = M).  CBD: box k gets colour (k_1 mod 2, ...,
    k_d mod 2) (the 2^d-colouring of Sec. 2.3's theorem) and each subdomain is the union
    of the extended boxes of one colour (Eq. e:cbd, D = 2^d).
    """
    if n % m != 0 or m < 1:
        raise ValueError("n must be a multiple of m")
    if delta < 0:
        raise ValueError("delta must be >= 0")
    w = n // m
    ext = 0 if kind == JACOBI else delta
    boxes = []
    colours = []
    for k in itertools.product(range(m), repeat=dim):
        ranges = [np.arange(max(kk * w - ext, 0), min((kk + 1) * w + ext, n)) for kk in k]
        mesh = np.meshgrid(*ranges, indexing="ij")
        idx = np.zeros(mesh[0].shape, dtype=np.int64)
        for a in mesh:
            idx = idx * n + a
        boxes.append(np.sort(idx.reshape(-1)))
        colours.append(tuple(kk % 2 for kk in k))
    if kind in (JACOBI, SCHWARZ):
        return boxes
    if kind == CBD:
        out = []
        for c in itertools.product(range(2), repeat=dim):
            members = [b for b, cc in zip(boxes, colours) if cc == c]
            if members:
                out.append(np.unique(np.concatenate(members)))
        return out
    raise ValueError("unknown decomposition kind")


# ---------------------------------------------------------------------------
# Subdomain factors and the additive preconditioner, Sec. 3 (Eqs. e:ai, e:ad)
# ---------------------------------------------------------------------------

def cholesky(A: np.ndarray) -> np.ndarray:
    """Lower-triangular L with A = L L^T, column by column (Cholesky-Crout).

    l_jj = sqrt(a_jj - sum_{k<j} l_jk^2),  l_ij = (a_ij - sum_{k<j} l_ik l_jk) / l_jj.
    Raises NotSPD at the first non-positive pivot.
    """
    A = np.asarray(A, dtype=np.float64)
    nb = A.shape[0]
    L = np.zeros_like(A)
    for j in range(nb):
        s = A[j, j] - L[j, :j] @ L[j, :j]
        if not s > 0.0:
            raise NotSPD(j)
        L[j, j] = math.sqrt(s)
        if j + 1 < nb:
            L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def block_matrices(dim: int, n: int, blocks, convention: int = GRID_TEXT, a_shift: float = 0.0):
    """A_i = R_i A R_i^T for each index set (Eq. e:ai)."""
    return [dense_matrix(dim, n, convention, a_shift, index=b) for b in blocks]


def factor(dim: int, n: int, blocks, convention: int = GRID_TEXT, a_shift: float = 0.0):
    """Cholesky factors L_i of every A_i."""
    return [cholesky(Ai) for Ai in block_matrices(dim, n, blocks, convention, a_shift)]


def apply(factors, blocks, r: np.ndarray) -> np.ndarray:
    """z = T^{-1} r = sum_i R_i^T A_i^{-1} R_i r (Eq. e:ad), A_i^{-1} = L_i^{-T} L_i^{-1}.

    A plain sum over the overlaps (no partition-of-unity weights).  r: (N,) or (N, k).
    """
    r = np.asarray(r, dtype=np.float64)
    z = np.zeros_like(r)
    for L, b in zip(factors, blocks):
        y = scipy.linalg.solve_triangular(L, r[b], lower=True)
        z[b] += scipy.linalg.solve_triangular(L.T, y, lower=False)
    return z


def preconditioner_matrix(factors, blocks, N: int) -> np.ndarray:
    """Dense T^{-1} = sum_i R_i^T A_i^{-1} R_i (Eq. e:ad), for spectra on small N."""
    T = np.zeros((N, N))
    for L, b in zip(factors, blocks):
        Linv = scipy.linalg.solve_triangular(L, np.eye(L.shape[0]), lower=True)
        T[np.ix_(b, b)] += Linv.T @ Linv
    return T


def preconditioned_spectrum(A: np.ndarray, Tinv: np.ndarray) -> np.ndarray:
    """Ascending eigenvalues of T^{-1} A (Eq. e:ta), via the similar symmetric C^T T^{-1} C
    with A = C C^T."""
    C = cholesky(A)
    S = C.T @ Tinv @ C
    S = 0.5 * (S + S.T)
    return scipy.linalg.eigvalsh(S)


# ---------------------------------------------------------------------------
# Preconditioned conjugate gradient (Sec. 6: PCG with the preconditioner of Eq. e:ad)
# ---------------------------------------------------------------------------

def pcg(matvec, precond, f: np.ndarray, tol: float, max_it: int, x0=None, history=None):
    """Hestenes-Stiefel PCG on A u = f, one independent recurrence per column.

    r_0 = f - A x0 (r_0 = f when x0 is None); per iteration z = T^{-1} r, rho = r^T z,
    p = z + (rho / rho_old) p, q = A p, alpha = rho / p^T q, u += alpha p, r -= alpha q.
    A column stops once ||r||_2 <= tol ||f||_2 and is frozen afterwards.  Returns
    (u, iterations per column, recursive relative residual per column).  ``history``,
    if a list, receives the per-iteration relative residuals.
    """
    f = np.asarray(f, dtype=np.float64)
    vec = f.ndim == 1
    F = f.reshape(f.shape[0], -1)
    k = F.shape[1]
    U = np.zeros_like(F) if x0 is None else np.array(np.asarray(x0, dtype=np.float64).reshape(F.shape))
    R = F - _cols(matvec, U) if x0 is not None else F.copy()
    fnorm = np.linalg.norm(F, axis=0)
    fnorm_safe = np.where(fnorm > 0, fnorm, 1.0)
    its = np.zeros(k, dtype=np.int64)
    active = np.linalg.norm(R, axis=0) > tol * fnorm
    P = np.zeros_like(F)
    rho = np.ones(k)
    first = True
    while active.any():
        Z = _cols(precond, R)
        rho_new = np.einsum("ij,ij->j", R, Z)
        if first:
            P = Z.copy()
            first = False
        else:
            beta = np.where(active, rho_new / np.where(active, rho, 1.0), 0.0)
            P = np.where(active, Z + beta * P, P)
        rho = np.where(active, rho_new, rho)
        Q = _cols(matvec, P)
        pq = np.einsum("ij,ij->j", P, Q)
        alpha = np.where(active, rho / np.where(active, pq, 1.0), 0.0)
        U = U + alpha * P
        R = R - alpha * Q
        its += active
        rel = np.linalg.norm(R, axis=0) / fnorm_safe
        if history is not None:
            history.append(rel.copy())
        active = active & (rel > tol) & (its < max_it)
    rel = np.linalg.norm(R, axis=0) / fnorm_safe
    if vec:
        return U[:, 0], int(its[0]), float(rel[0])
    return U, its, rel


def _cols(op, X):
    Y = op(X if X.shape[1] > 1 else X[:, 0])
    return np.asarray(Y).reshape(X.shape)


def true_relative_residual(dim: int, n: int, f: np.ndarray, u: np.ndarray,
                           matvec=None) -> np.ndarray:
    """||f - A u||_2 / ||f||_2 per column, with A u from ``matvec`` (FFT route by default)."""
    mv = matvec or (lambda v: matvec_fft(dim, n, v))
    F = np.asarray(f).reshape(f.shape[0], -1)
    R = F - np.asarray(mv(u)).reshape(F.shape)
    out = np.linalg.norm(R, axis=0) / np.linalg.norm(F, axis=0)
    return out if F.shape[1] > 1 else float(out[0])


class Problem:
    """Convenience bundle: discretization + decomposition + factors, for tests and the
    CPU baseline.  matvec: 'dense' (small N), 'direct' or 'fft'."""

    def __init__(self, dim, n, m, delta, kind=SCHWARZ, convention=GRID_TEXT, a_shift=0.0,
                 matvec="fft"):
        self.dim, self.n, self.N = dim, n, n ** dim
        self.convention, self.a_shift = convention, a_shift
        self.blocks = partition(dim, n, m, delta, kind)
        self.factors = factor(dim, n, self.blocks, convention, a_shift)
        if matvec == "dense":
            self.A = dense_matrix(dim, n, convention, a_shift)
            self.matvec = lambda x: self.A @ x
        elif matvec == "direct":
            self.matvec = lambda x: matvec_direct(dim, n, x, None, convention, a_shift)
        elif matvec == "fft":
            self.matvec = lambda x: matvec_fft(dim, n, x, convention, a_shift)
        else:
            raise ValueError(matvec)

    def apply(self, r):
        return apply(self.factors, self.blocks, r)

    def solve(self, f, tol, max_it=1000, x0=None, history=None):
        return pcg(self.matvec, self.apply, f, tol, max_it, x0, history)
