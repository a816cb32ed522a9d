"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module only makes inputs: it holds none of the solver's arithmetic (no kernel,
no discretization, no preconditioner).  Everything is generated on the host in FP64
so that both sides of a parity check see bit-identical data.

Generators
----------
* ``uniform_rhs``  -- i.i.d. uniform[-1, 1] entries from SplitMix64 (Steele, Lea and
  Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): state
  advances by the golden-gamma constant 0x9E3779B97F4A7C15, the output is the
  variant-13 mix, and the top 53 bits become a double in [0, 1).
* ``gaussian_noise`` -- standard normals from two SplitMix64 streams by Box-Muller.
* ``grf``          -- a stationary Gaussian random field on the cell-centred grid with
  squared-exponential covariance exp(-r^2 / (2 l^2)) (unit variance), made by
  circulant embedding on a (2n)^d periodic grid: the covariance is sampled at the
  wrapped offsets, its FFT gives the circulant eigenvalues (negative ones, which
  only appear from truncation, are clipped to 0), white noise is filtered by their
  square root and the [0, n)^d window is kept.  The window is then scaled to unit
  sample standard deviation.

Index order everywhere is row-major with the last coordinate fastest.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """First ``count`` outputs of SplitMix64 started from state ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def unit_doubles(seed: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64 outputs."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_rhs(n_points: int, seed: int) -> np.ndarray:
    """i.i.d. uniform[-1, 1] vector of length ``n_points`` from seed ``seed``."""
    return 2.0 * unit_doubles(seed, n_points) - 1.0


def uniform_rhs_batch(n_points: int, seeds) -> np.ndarray:
    """Column-major batch: column k is ``uniform_rhs(n_points, seeds[k])``."""
    return np.stack([uniform_rhs(n_points, s) for s in seeds], axis=1)


def gaussian_noise(count: int, seed: int) -> np.ndarray:
    """Standard normal samples by Box-Muller over two SplitMix64 streams."""
    u1 = unit_doubles(2 * seed + 1, count)
    u2 = unit_doubles(2 * seed + 2, count)
    u1 = 1.0 - u1  # (0, 1]: log stays finite
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def grf(dim: int, n: int, ell: float, seed: int) -> np.ndarray:
    """Unit-variance squared-exponential Gaussian random field, flattened (N,)."""
    h = 1.0 / n
    size = 2 * n
    off = np.arange(size)
    off = np.minimum(off, size - off) * h  # wrapped distance on the 2n torus
    grids = np.meshgrid(*([off] * dim), indexing="ij")
    r2 = sum(g * g for g in grids)
    cov = np.exp(-r2 / (2.0 * ell * ell))
    lam = np.fft.fftn(cov).real
    lam = np.maximum(lam, 0.0)
    w = gaussian_noise(size ** dim, seed).reshape((size,) * dim)
    field = np.fft.ifftn(np.sqrt(lam) * np.fft.fftn(w)).real
    window = field[tuple(slice(0, n) for _ in range(dim))]
    window = window / window.std()
    return np.ascontiguousarray(window.reshape(-1))


def grf_batch(dim: int, n: int, ells, seeds) -> np.ndarray:
    """Column-major batch of GRFs, column k with length scale ells[k], seed seeds[k]."""
    return np.stack([grf(dim, n, l, s) for l, s in zip(ells, seeds)], axis=1)


# Named workloads (the synthetic stand-ins for the paper's uniform-grid problems).
WORKLOADS = {
    # 2D plain FP64 method, 64^2, uniform RHS seed 0, Schwarz 4x4 partitions, 1-cell overlap.
    "ie2d_n64_schwarz_m4_d1": dict(dim=2, n=64, m=4, delta=1, rhs="uniform", seeds=(0,), tol=1e-8),
    # 2D mixed precision, 512^2, GRF l=0.1 seed 0, Schwarz 32x32 partitions (16x16 cells), 2-cell overlap.
    "ie2d_n512_schwarz_m32_d2": dict(dim=2, n=512, m=32, delta=2, rhs="grf", ell=0.1, seeds=(0,),
                                     tol=1e-8, replace_every=50),
    # 3D batched, 32^3, 64 uniform RHS seeds 0..63, Schwarz 4x4x4 partitions, 1-cell overlap.
    "ie3d_n32_schwarz_m4_d1_rhs64": dict(dim=3, n=32, m=4, delta=1, rhs="uniform",
                                         seeds=tuple(range(64)), tol=1e-8),
    # 2D large, 1024^2, GRF l=0.05 seed 0, Schwarz 64x64 partitions, 2-cell overlap.
    "ie2d_n1024_schwarz_m64_d2": dict(dim=2, n=1024, m=64, delta=2, rhs="grf", ell=0.05, seeds=(0,),
                                      tol=1e-8),
    # 2D warm-start workload, 256^2, Schwarz 16x16 partitions, 2-cell overlap.
    "ie2d_n256_schwarz_m16_d2": dict(dim=2, n=256, m=16, delta=2, rhs="grf", ell=0.1, seeds=(0,),
                                     tol=1e-8),
}


def workload_rhs(name: str) -> np.ndarray:
    """The RHS of a named workload: (N,) for one seed, (N, k) column-major batch otherwise."""
    w = WORKLOADS[name]
    N = w["n"] ** w["dim"]
    if w["rhs"] == "uniform":
        cols = [uniform_rhs(N, s) for s in w["seeds"]]
    else:
        cols = [grf(w["dim"], w["n"], w["ell"], s) for s in w["seeds"]]
    return cols[0] if len(cols) == 1 else np.stack(cols, axis=1)
