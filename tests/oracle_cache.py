"""Oracle solves too slow to run inside one test, computed in a background process.

The 1024^2 workload's FP64 oracle solve (its own column Cholesky of 4096 blocks and an FFT-matvec
PCG) takes minutes on the host.  When a pytest session has collected a test that needs it,
``conftest.py`` starts it at the beginning of the session (``start``), so that it overlaps the
GPU tests before it; the test then waits for it (``result``).  The background job is a separate
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

# name -> (dim, n, m, delta, GRF length scale, seed, tolerance)
JOBS = {"ie2d_n1024_m64_d2_grf": (2, 1024, 64, 2, 0.05, 0, 1e-8)}
# test node-id fragments that need each job
NEEDED_BY = {"ie2d_n1024_m64_d2_grf": "test_pcg_full_size_1024_mixed"}

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
    """(u, iterations, recursive relative residual, history) of the oracle solve of ``name``;
    starts it if nothing has, then waits for it."""
    start(name)
    proc, out = _procs[name]
    proc.wait(timeout=timeout)
    if proc.returncode != 0:
        raise RuntimeError(f"oracle job {name} failed: " + open(out + ".log").read()[-2000:])
    z = np.load(out)
    return z["u"], int(z["iterations"]), float(z["relres"]), z["history"]


def stop_all() -> None:
    for proc, _ in _procs.values():
        if proc.poll() is None:
            proc.kill()
            proc.wait()


def _compute(name: str, out: str) -> None:
    sys.path.insert(0, ROOT)
    from oracle import ie_oracle as O
    from paper_2108_12574_gb300 import inputs as I

    dim, n, m, delta, ell, seed, tol = JOBS[name]
    t0 = time.time()
    f = I.grf(dim, n, ell, seed)
    P = O.Problem(dim, n, m, delta, O.SCHWARZ, matvec="fft")
    hist: list = []
    u, its, rel = P.solve(f, tol, history=hist)
    tmp = out + ".tmp.npz"
    np.savez(tmp, u=u, iterations=its, relres=rel, history=np.array(hist).reshape(-1))
    os.replace(tmp, out)
    print(f"{name}: {its} iterations, {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    _compute(sys.argv[1], sys.argv[2])
