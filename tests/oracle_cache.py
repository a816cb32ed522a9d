"""Oracle solves too slow to run inside one test, computed in a background process.

The 1024^2 workload's FP64 oracle solve (its own column Cholesky of 4096 blocks and an FFT-matvec
PCG) and the 64^3 solve (512 blocks of up to 1000 points) take minutes on the host.  When a pytest
session has collected a test that needs one, ``conftest.py`` starts it at the beginning of the
session (``start``), so that it overlaps the GPU tests before it; the test then waits for it
(``result``).  The background job is a separate
Python process started with subprocess (fork + exec), so it shares no state with the CUDA
context of the test process.  It calls only the oracle and the seeded input generators.

  python tests/oracle_cache.py NAME OUT.npz   (what the background process runs)
"""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

# name -> (dim, n, m, delta, GRF length scale (None: uniform[-1,1]), seeds, tolerance)
JOBS = {"ie2d_n1024_m64_d2_grf": (2, 1024, 64, 2, 0.05, [0], 1e-8),
        "ie3d_n64_m8_d1_uniform": (3, 64, 8, 1, None, [0, 1], 1e-8)}
# test node-id fragments that need each job
NEEDED_BY = {"ie2d_n1024_m64_d2_grf": "test_pcg_full_size_1024_mixed",
             "ie3d_n64_m8_d1_uniform": "test_3d_n64_batched_matvec_and_solve"}

_procs: dict = {}


def _out(name: str) -> str:
    d = os.environ.get("IEDD_ORACLE_CACHE") or os.path.join(tempfile.gettempdir(), f"iedd_oracle_{os.getpid()}")
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, f"{name}.npz")


def start(name: str) -> None:
    """Start the background solve of ``name`` (once per session)."""
    if name in _procs:
        return
    out = _out(name)
    log = open(out + ".log", "w")
    _procs[name] = (subprocess.Popen([sys.executable, os.path.abspath(__file__), name, out], cwd=ROOT,
                                     stdout=log, stderr=subprocess.STDOUT), out)


def result(name: str, timeout: float = 3600.0):
    """(u, iterations, recursive relative residual, history) of the oracle solve of ``name``
    (per column when the job has several right-hand sides); starts it if nothing has, then waits
    for it.  Jobs in 3D return a fifth entry: the iterations of the first column's solve with an
    FP32-class matvec (every product perturbed by 2^-23 |A| |x|)."""
    start(name)
    proc, out = _procs[name]
    proc.wait(timeout=timeout)
    if proc.returncode != 0:
        raise RuntimeError(f"oracle job {name} failed: " + open(out + ".log").read()[-2000:])
    z = np.load(out)
    its = z["iterations"]
    its = int(its) if its.ndim == 0 else its
    res = (z["u"], its, z["relres"], z["history"])
    return res + ((z["its_mv32"],) if "its_mv32" in z else ())


def stop_all() -> None:
    for proc, _ in _procs.values():
        if proc.poll() is None:
            proc.kill()
            proc.wait()


def _compute(name: str, out: str) -> None:
    sys.path.insert(0, ROOT)
    from oracle import ie_oracle as O
    from paper_2108_12574_gb300 import inputs as I

    dim, n, m, delta, ell, seeds, tol = JOBS[name]
    t0 = time.time()
    if ell is None:
        F = I.uniform_rhs_batch(n ** dim, seeds)
    else:
        F = np.stack([I.grf(dim, n, ell, s) for s in seeds], axis=1)
    f = F[:, 0] if F.shape[1] == 1 else F
    P = O.Problem(dim, n, m, delta, O.SCHWARZ, matvec="fft")
    hist: list = []
    u, its, rel = P.solve(f, tol, history=hist)
    extra = {}
    if dim == 3:
        rng = np.random.default_rng(7)

        def mv32(x):
            y = O.matvec_fft(dim, n, x)
            return y + 2.0 ** -23 * O.matvec_fft(dim, n, np.abs(x)) * rng.uniform(-1.0, 1.0, y.shape)
        _, its32, _ = O.pcg(mv32, P.apply, F[:, :1], tol, 1000)
        extra["its_mv32"] = np.atleast_1d(its32)
    tmp = out + ".tmp.npz"
    np.savez(tmp, u=u, iterations=its, relres=rel, history=np.array(hist).reshape(len(hist), -1), **extra)
    os.replace(tmp, out)
    print(f"{name}: {its} iterations, {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    _compute(sys.argv[1], sys.argv[2])
