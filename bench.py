#!/usr/bin/env python
"""Benchmark: PCG time to a 1e-8 true relative residual on the 2D 1024^2 workload.

Workload (synthetic stand-in for the paper's uniform-grid problems): 2D Laplace first-kind
IE, 1024 x 1024 cell-centred grid (N = 1048576, 1.1e12 kernel pairs per matvec), f a Gaussian
random field (squared-exponential covariance, length scale 0.05, seed = rank), Schwarz
preconditioner with 64 x 64 partitions of 16 x 16 cells extended by 2 cells (4096 blocks of up
to 400 points); subdomain Cholesky and explicit FP32 inverses on the tensor cores, applied with
double-float products; the exact direct-sum matvec on the tensor cores (the FP64 per-offset
entries and x cut into six BF16 digits, 21 digit products summed exactly); FP64 CG vectors and
scalars; the FP64 FFT matvec for the true residual, which replaces the recursive one every 50
iterations and at convergence; tolerance 1e-8 on the true residual.

One step = the whole hot path for one right-hand side: ie_discretize, dd_partition, dd_factor,
pcg_solve (inputs already in HBM).  N > 1 GPUs run independent replicas (weak scaling).
The other workloads (--workload) are timed the same way; the 512^2 one is also reported as an
extra leg of the default run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "ie2d_n1024_schwarz_m64_d2"
TOL, REPLACE_EVERY = 1e-8, 50
# every workload the benchmark can time (--workload); the default is the 1024^2 one, the
# largest that the workloads define
WORKLOADS = {
    "ie2d_n64_schwarz_m4_d1": dict(dim=2, n=64, m=4, delta=1, rhs="uniform", seeds=1, precision="fp64",
                                   factor="fp64"),
    "ie2d_n512_schwarz_m32_d2": dict(dim=2, n=512, m=32, delta=2, rhs="grf", ell=0.1, seeds=1, precision="mixed",
                                     factor="mixed"),
    "ie3d_n32_schwarz_m4_d1_rhs64": dict(dim=3, n=32, m=4, delta=1, rhs="uniform", seeds=64, precision="mixed",
                                         factor="mixed"),
    "ie2d_n1024_schwarz_m64_d2": dict(dim=2, n=1024, m=64, delta=2, rhs="grf", ell=0.05, seeds=1, precision="mixed",
                                      factor="mixed"),
    "ie2d_n256_schwarz_m16_d2": dict(dim=2, n=256, m=16, delta=2, rhs="grf", ell=0.1, seeds=1, precision="mixed",
                                     factor="mixed"),
    # the paper's CBD preconditioner with recursive-skeletonization subdomain factors (Sec. 4.3) at
    # N / M = 64, one layer of overlap, eps = 1e-3 (Sec. 5.2), the FP64 FFT matvec (Sec. 6)
    "ie2d_n1024_cbd_rs_m128_d1": dict(dim=2, n=1024, m=128, delta=1, rhs="grf", ell=0.05, seeds=1, precision="fp64",
                                      factor="rs", eps=1e-3, inner="fft"),
    # the same beyond the dense-CBD limit: the paper's weak-scaling rows (Sec. 5, N / M = 64 in 2D, 512 in 3D)
    "ie2d_n2048_cbd_rs_m256_d1": dict(dim=2, n=2048, m=256, delta=1, rhs="grf", ell=0.05, seeds=1, precision="fp64",
                                      factor="rs", eps=1e-3, inner="fft"),
    "ie3d_n64_cbd_rs_m8_d1": dict(dim=3, n=64, m=8, delta=1, rhs="uniform", seeds=1, precision="fp64", factor="rs",
                                  eps=1e-3, inner="fft"),
}
METRIC = "PCG time-to-1e-8 true relative residual (s)"
L2_FLUSH_BYTES = 512 << 20
# FP32-pipe operations per pair of the exact double-float matvec (k2_accurate_2d, x split hi/lo):
# FMUL, FADD, FADD, 3 FFMA, FADD, plus the Fast2Sum renormalisation (3 ops every 4 pairs)
FP32_OPS_PER_PAIR_K2 = 7.75
FP32_LANES_PER_SM = 128

# DRAM traffic per launch of the dominant kernel from an ncu capture, valid only for the
# source it was measured on (k2_source_hash: the 2D exact kernel's source text); otherwise the
# bench reports null.
NCU_TRAFFIC = {"24904137a1834c92": 4624128}  # k2_accurate_2d<true,1>, n = 512, bytes per launch
# ncu figures of the exact tensor-core matvec per (tc_exact_source_hash(), grid side n): DRAM
# bytes per launch and the tensor pipe's active fraction (sm__pipe_tensor_cycles_active)
NCU_KZ = {("e2d6b85e8691647a", 1024): {"traffic": 1782236976, "tensor_pipe": 0.620}}
# the same for the batched tensor-core matvec per (tc_matvec_source_hash(), grid side n), 3D
NCU_K1W = {("c8970434ed8bad33", 32): {"traffic": 83382784, "tensor_pipe": 0.430}}
# BF16 digit products per pair of the exact tensor-core matvec (six digits per factor, levels 0..5)
KZ_PRODUCTS_PER_PAIR = 21
# ncu figures of the RS factor's level-1 launches per rs_source_hash(), 2D 256^2 with M = 32^2 (the
# same region shapes as 1024^2): FP64 pipe activity of rs_id / rs_elim and their DRAM bytes
NCU_RS = {"ae5a2a3237e2c633": {"fp64_pipe": {"rs_id": 0.737, "rs_elim": 0.698},
                               "dram_bytes_256": {"rs_id": 1516905437, "rs_elim": 398942244}}}
# GB300's FP64 rate (nominal; no FP64 peak is measured on this machine)
FP64_NOMINAL_TFLOPS = 1.25


TF32_PER_BF16 = 1.1 / 2.25  # nominal dense tensor rates per GPU


def measured_peak(key: str, fallback: float) -> float:
    """A peak from MEASURED_PEAKS.json at the repository root (driver-written), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key])
    except (OSError, KeyError, ValueError, TypeError):
        return fallback


def k2_source_hash() -> str:
    """sha256 (16 hex digits) of the 2D exact kernel's source text (from its patch constants to
    the 3D kernel's comment), the key under which its ncu DRAM traffic is recorded."""
    src = open(os.path.join(ROOT, "paper_2108_12574_gb300", "csrc", "matvec.cu")).read()
    a, b = src.index("constexpr int kP1"), src.index("// 3D: 4 x 8 x 8 patches")
    return hashlib.sha256(src[a:b].encode()).hexdigest()[:16]


def tc_matvec_source_hash() -> str:
    """sha256 (16 hex digits) of the batched tensor-core matvec's source file."""
    src = open(os.path.join(ROOT, "paper_2108_12574_gb300", "csrc", "tc_matvec.cu")).read()
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def tc_exact_source_hash() -> str:
    """sha256 (16 hex digits) of the exact tensor-core matvec's source file."""
    src = open(os.path.join(ROOT, "paper_2108_12574_gb300", "csrc", "tc_exact.cu")).read()
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def rs_source_hash() -> str:
    """sha256 (16 hex digits) of the RS factor kernels' source text (the entry lookup, rs_proxy_table,
    rs_id, the tiled products and rs_elim: up to the first apply kernel), the key of their ncu
    figures."""
    src = open(os.path.join(ROOT, "paper_2108_12574_gb300", "csrc", "rs.cu")).read()
    a, b = src.index("__device__ __forceinline__ double a_entry"), src.index("__global__ void rs_gather")
    return hashlib.sha256(src[a:b].encode()).hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=WORKLOAD)
    ap.add_argument("--no-extras", action="store_true", help="skip FP64-plain and CPU-baseline legs")
    ap.add_argument("--kernel", choices=["k1", "k2", "kd", "tc", "kz", "stored", "fft", "apply", "factor", "rs", "rs_apply", "ws_train",
                                         "ws_predict"], default=None,
                    help="profiling case: run one hot operation twice on a --dim/--n/--nrhs problem and exit")
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--nrhs", type=int, default=1)
    return ap.parse_args()


def kernel_case(args):
    """A single hot operation, launched twice (warm-up + the one to capture with ncu -s/-c)."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_12574_gb300 import iedd
    from paper_2108_12574_gb300 import inputs as I

    N = args.n ** args.dim
    prob = iedd.ie_discretize(args.dim, args.n)
    if args.kernel in ("ws_train", "ws_predict"):
        # the warm-start network: one training step (forward, backward, Adam) or one prediction
        # on --nrhs Gaussian random fields of a 2D --n grid
        model = iedd.ws_create(0, 1)
        F = torch.from_numpy(np.stack([I.grf(2, args.n, 0.1, s) for s in range(args.nrhs)])).cuda()
        U = torch.from_numpy(np.stack([I.grf(2, args.n, 0.2, s + 50) for s in range(args.nrhs)])).cuda()
        for _ in range(2):
            if args.kernel == "ws_train":
                model.train_step(prob, F, U, 1e-4)
            else:
                model.predict(prob, F, U)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_case": args.kernel, "dim": 2, "n": args.n, "nrhs": args.nrhs, "ok": True}))
        return 0
    X = torch.from_numpy(I.uniform_rhs_batch(N, range(args.nrhs)).T.copy()).cuda()
    Y = torch.zeros_like(X)
    if args.kernel in ("rs", "rs_apply"):
        # the RS factor of a CBD partition into boxes of 8^d points, one layer of overlap, eps = 1e-3
        # (the paper's N / M = 64 in 2D, 512 in 3D); rs_apply then applies it
        part = iedd.dd_partition(prob, args.n // 8, 1, iedd.DD_CBD)
        for _ in range(2):
            fac = iedd.dd_factor_rs(prob, part, eps=1e-3)
            if args.kernel == "rs_apply":
                iedd.dd_apply(fac, X, Y)
            torch.cuda.synchronize()
            levels, top, st = iedd.dd_rs_info(fac, stats=True)
            fac.close()
        print(json.dumps({"kernel_case": args.kernel, "dim": args.dim, "n": args.n, "levels": levels, "top": top,
                          "stats": st, "ok": True}))
        return 0
    m = args.n // 16 if args.dim == 2 else args.n // 8
    for _ in range(2):
        if args.kernel in ("k1", "k2", "kd", "tc", "kz", "stored", "fft"):
            prec = {"k1": iedd.IE_MIXED, "k2": iedd.IE_ACCURATE, "kd": iedd.IE_FP64, "tc": iedd.IE_TENSOR,
                    "kz": iedd.IE_TENSOR_EXACT, "stored": iedd.IE_STORED, "fft": iedd.IE_FFT}[args.kernel]
            if args.kernel == "stored":
                iedd.ie_store_matrix(prob)
            iedd.ie_matvec(prob, X, Y, prec)
        else:
            part = iedd.dd_partition(prob, m, 2 if args.dim == 2 else 1, iedd.DD_SCHWARZ)
            fac = iedd.dd_factor(prob, part, iedd.IE_MIXED)
            if args.kernel == "apply":
                iedd.dd_apply(fac, X, Y)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": args.kernel, "dim": args.dim, "n": args.n, "nrhs": args.nrhs, "ok": True}))
    return 0


PRECISION_TEXT = {
    "mixed2d": ("mixed (exact direct-sum matvec on the tcgen05 tensor cores: FP64 entries and x cut into six "
                "BF16 digits, 21 digit products summed exactly; FP32 explicit subdomain inverses with "
                "double-float products; FP64 scalars and vectors; the FP64 true residual and replacements by "
                "the FP64 FFT matvec)"),
    "mixed3d": ("mixed (3xTF32 tcgen05 batched matvec with FP32 accumulation; FP32 explicit subdomain "
                "inverses; FP64 scalars and vectors; the FP64 true residual by the FP64 FFT matvec)"),
    "fp64": "FP64 (entries regenerated in FP64, FP64 Cholesky factors and triangular solves)",
}


def config_dict(name: str = WORKLOAD) -> dict:
    W = WORKLOADS[name]
    rhs = (f"GRF l={W['ell']} seed=rank" if W["rhs"] == "grf" else
           f"uniform[-1,1] seeds rank*{W['seeds']}..+{W['seeds'] - 1}" if W["seeds"] > 1 else "uniform[-1,1] seed=rank")
    prec = "fp64" if W["precision"] == "fp64" else f"mixed{W['dim']}d"
    out = {"workload": name, "dim": W["dim"], "n": W["n"], "N": W["n"] ** W["dim"], "m": W["m"],
           "delta": W["delta"], "nrhs": W["seeds"], "rhs": rhs, "tol": TOL, "decomposition": "schwarz",
           "precision": PRECISION_TEXT[prec], "l2": "flushed between timed steps (512 MiB write)"}
    if W["factor"] == "rs":
        out.update({"decomposition": "cbd", "subdomain_solver": f"recursive skeletonization, eps={W['eps']}",
                    "precision": "f64 throughout (FFT matvec, RS factors and apply, CG scalars)"})
    return out


def make_factor(iedd, prob, W, stream, fprec=None):
    """(partition, factor) of a workload: Schwarz boxes with dense Cholesky factors, or the CBD
    colours with recursive-skeletonization factors."""
    if W["factor"] == "rs":
        part = iedd.dd_partition(prob, W["m"], W["delta"], iedd.DD_CBD)
        return part, iedd.dd_factor_rs(prob, part, eps=W["eps"], stream=stream)
    if fprec is None:
        fprec = iedd.IE_FP64 if W["factor"] == "fp64" else iedd.IE_MIXED
    part = iedd.dd_partition(prob, W["m"], W["delta"], iedd.DD_SCHWARZ)
    return part, iedd.dd_factor(prob, part, fprec, stream=stream)


def inner_of(iedd, W) -> int:
    """pcg_opts.inner of a workload (0: the library's choice)."""
    return iedd.IE_FFT if W.get("inner") == "fft" else 0


# ------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def gpu_id_of(torch, dev):
    try:
        p = torch.cuda.get_device_properties(dev)
        dom = getattr(p, "pci_domain_id", 0)
        return f"{dom:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return None


# ------------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the workload, scaled
# ------------------------------------------------------------------------------------------
def cpu_model() -> str:
    """The host CPU's model name and architecture (for the CPU-baseline record)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return f"{line.split(':', 1)[1].strip()} ({platform.machine()})"
    except Exception:
        pass
    return platform.machine() or "unknown"


def oracle_fp64_count(name: str):
    """The oracle's own FP64 PCG iteration count at 1e-8 for a workload's first right-hand side
    (tests/golden/pcg_counts.json, written by a script that calls only the oracle), or None."""
    key = {"ie2d_n512_schwarz_m32_d2": "ie2d_n512_m32_d2_grf", "ie2d_n1024_schwarz_m64_d2": "ie2d_n1024_m64_d2_grf",
           "ie3d_n32_schwarz_m4_d1_rhs64": "ie3d_n32_m4_d1_uniform64"}.get(name)
    try:
        with open(os.path.join(ROOT, "tests", "golden", "pcg_counts.json")) as fh:
            return int(json.load(fh)[key]["it_fp64_at_1e-8"][0])
    except (OSError, KeyError, ValueError, TypeError, IndexError):
        return None


def workload_rhs(name: str, seed0: int = 0):
    """(N, nrhs) FP64 right-hand sides of a workload, seeds seed0..seed0+nrhs-1, on the host."""
    import numpy as np

    from paper_2108_12574_gb300 import inputs as I
    W = WORKLOADS[name]
    N = W["n"] ** W["dim"]
    seeds = [seed0 + k for k in range(W["seeds"])]
    if W["rhs"] == "grf":
        return np.stack([I.grf(W["dim"], W["n"], W["ell"], s_) for s_ in seeds], axis=1)
    return np.stack([I.uniform_rhs(N, s_) for s_ in seeds], axis=1)


def cpu_baseline(name: str, iterations: int, rows_sample: int = 2048, blocks_sample: int = 64,
                 iterations_from: str = "the oracle's FP64 count at 1e-8"):
    """The FP64 oracle on a bounded sample of a workload, scaled to the whole solve: the direct-sum
    matvec over ``rows_sample`` rows (C, OpenMP), the oracle's own Cholesky and triangular-solve
    apply on ``blocks_sample`` subdomains; total = factor + iterations x (matvec + apply).
    Extrapolated, and labelled so."""
    import numpy as np

    from oracle import ie_oracle as O
    W = WORKLOADS[name]
    dim, n = W["dim"], W["n"]
    N = n ** dim
    F = workload_rhs(name)
    nr = F.shape[1]
    rows = np.linspace(0, N - 1, min(rows_sample, N)).astype(np.int64)
    t0 = time.perf_counter()
    O.matvec_direct(dim, n, F, rows=rows)
    t_mv = (time.perf_counter() - t0) * N / rows.size
    blocks = O.partition(dim, n, W["m"], W["delta"], O.SCHWARZ)
    step = max(1, len(blocks) // blocks_sample)
    sb = [blocks[i] for i in range(0, len(blocks), step)][:blocks_sample]
    t0 = time.perf_counter()
    fac = O.factor(dim, n, sb)
    t_fac = (time.perf_counter() - t0) * len(blocks) / len(sb)
    t0 = time.perf_counter()
    O.apply(fac, sb, F if nr > 1 else F[:, 0])
    t_ap = (time.perf_counter() - t0) * len(blocks) / len(sb)
    total = t_fac + iterations * (t_mv + t_ap)
    return {"value": total, "unit": "s", "cores": oracle_cores(), "cpu": cpu_model(), "kind": "oracle",
            "workload": name, "extrapolated": True,
            "sample": (f"FP64 direct-sum matvec over {rows.size} of {N} rows x {nr} right-hand side(s) (C, "
                       f"OpenMP), own Cholesky and triangular-solve apply on {len(sb)} of {len(blocks)} "
                       f"subdomains, each scaled to the full workload; total = factor + {iterations} "
                       f"iterations ({iterations_from}) x (matvec + apply); extrapolated"),
            "parts_s": {"matvec": t_mv, "apply": t_ap, "factor": t_fac}}


def oracle_cores() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def oracle_full_solve(name: str, matvec: str):
    """The FP64 oracle's whole solve of a workload (discretize, partition, factor, PCG to 1e-8 on
    the recursive residual), timed end to end on the host cores: measured, not extrapolated."""
    from oracle import ie_oracle as O
    W = WORKLOADS[name]
    F = workload_rhs(name)
    t0 = time.perf_counter()
    P = O.Problem(W["dim"], W["n"], W["m"], W["delta"], O.SCHWARZ, matvec=matvec)
    t_fac = time.perf_counter() - t0
    _, its, rel = P.solve(F if F.shape[1] > 1 else F[:, 0], TOL)
    total = time.perf_counter() - t0
    its = [int(v) for v in (its if F.shape[1] > 1 else [its])]
    return {"value": total, "unit": "s", "workload": name, "extrapolated": False, "cores": oracle_cores(),
            "matvec": {"direct": "direct sum (C, OpenMP)", "fft": "FFT (numpy, the paper's matvec)"}[matvec],
            "factor_s": t_fac, "iterations_max": max(its), "iterations_min": min(its), "nrhs": F.shape[1]}


def oracle_measured_legs(per_step: bool):
    """End-to-end oracle solves that fit a bench run: the 64^2 FP64 workload (under a second)
    and, once per run, the 3D 32^3 workload with 64 right-hand sides (FFT matvec)."""
    out = {"ie2d_n64_schwarz_m4_d1": oracle_full_solve("ie2d_n64_schwarz_m4_d1", "direct")}
    if not per_step:
        out["ie3d_n32_schwarz_m4_d1_rhs64"] = oracle_full_solve("ie3d_n32_schwarz_m4_d1_rhs64", "fft")
    return out


def run_reference(args):
    """The oracle as the reference arm: each step is a bounded sample of the benchmarked workload
    (extrapolated to the whole solve, as cpu_baseline) plus the 64^2 workload solved in full;
    the 3D 64-column workload is solved in full once at the end."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    name = args.workload
    iters = oracle_fp64_count(name)
    src = "the oracle's FP64 count at 1e-8"
    if iters is None:
        iters, src = 80, "an assumed 80: no stored oracle count for this workload"
    for _ in range(args.warmup):
        cpu_baseline(name, iters, iterations_from=src)
    vals, small = [], []
    for _ in range(args.steps):
        vals.append(cpu_baseline(name, iters, iterations_from=src))
        small.append(oracle_measured_legs(per_step=True)["ie2d_n64_schwarz_m4_d1"]["value"])
    v = statistics.mean(x["value"] for x in vals)
    cb = dict(vals[-1])
    cb["value"] = v
    measured = oracle_measured_legs(per_step=False)
    measured["ie2d_n64_schwarz_m4_d1"]["value_mean_over_steps"] = statistics.mean(small)
    cb["measured_end_to_end"] = measured
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(name), "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------
def main():
    args = parse()
    if args.kernel:
        return kernel_case(args)
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_12574_gb300 import iedd
    from paper_2108_12574_gb300 import inputs as I

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def reduce_max(v: float) -> float:
        return max_over_ranks(v, dist, dev)

    W = WORKLOADS[args.workload]
    dim_w, n_w = W["dim"], W["n"]
    N = n_w ** dim_w
    nr = W["seeds"]
    prec = iedd.IE_FP64 if W["precision"] == "fp64" else iedd.IE_MIXED
    inner = inner_of(iedd, W)
    seeds = [rank * nr + k for k in range(nr)]
    if W["rhs"] == "grf":
        f_host = np.stack([I.grf(dim_w, n_w, W["ell"], s_) for s_ in seeds])
    else:
        f_host = np.stack([I.uniform_rhs(N, s_) for s_ in seeds])
    if nr == 1:
        f_host = f_host[0]
    f = torch.from_numpy(f_host).to(dev)
    u = torch.zeros_like(f)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    rs_stats = {}

    def step(fv, uv):
        prob = iedd.ie_discretize(dim_w, n_w, device=local)
        part, fac = make_factor(iedd, prob, W, stream)
        reps = iedd.pcg_solve(prob, fac, fv, uv, tol=TOL, precision=prec, replace_every=REPLACE_EVERY,
                              inner=inner, stream=stream)
        if W["factor"] == "rs":
            rs_stats.update(iedd.dd_rs_info(fac, stats=True)[2])
        fac.close(); part.close(); prob.close()
        return reps

    for _ in range(args.warmup):
        u.zero_()
        step(f, u)
    barrier()

    sampler = ClockSampler(gpu_id_of(torch, dev))
    sampler.start()
    iedd.ie_kernel_launches(reset=True)
    total_ms = 0.0
    reps = []
    for _ in range(args.steps):
        flush.fill_(1.0)  # L2 flush (outside the timed window)
        u.zero_()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps.append(step(f, u))
        e1.record(stream)
        torch.cuda.synchronize(dev)
        total_ms += e0.elapsed_time(e1)
    launches = iedd.ie_kernel_launches(reset=True)
    barrier()
    clocks = sampler.stop()
    total_ms = reduce_max(total_ms)
    ms_per_step = total_ms / args.steps
    value = ms_per_step / 1e3

    # correctness of what was timed: the true residual reported by the accurate matvec
    ok = all(r["status"] == 0 and 0 <= r["true_relres"] <= TOL for rs in reps for r in rs)
    last = reps[-1][0]
    its_all = [r["iterations"] for r in reps[-1]]

    # end to end through the public API with HOST buffers (copies inside the timed region)
    u_host = np.zeros_like(f_host)
    e2e_times = []
    for _ in range(max(1, args.steps)):
        flush.fill_(1.0)  # same L2 state as the device-timed steps (outside the timed window)
        barrier()
        t0 = time.perf_counter()
        step(f_host, u_host)
        e2e_times.append(time.perf_counter() - t0)
    e2e = {"value": reduce_max(statistics.mean(e2e_times)), "unit": "s",
           "h2d_bytes_per_step": int(f_host.nbytes), "d2h_bytes_per_step": int(u_host.nbytes)}

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roofline, kz_inner = roofline_of(iedd, args.workload, last, clocks, sms, rs_stats)
    cfg = config_dict(args.workload)
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None,
            "dtype": ("bf16 digit slices (Ozaki) + f32 windows + int64 sums + f64" if kz_inner else
                      "tf32x3 + f32 + f64" if prec == iedd.IE_MIXED and dim_w == 3 and nr >= 16 else
                      "f32 (double-float sums) + f64" if prec == iedd.IE_MIXED else "f64"),
            "data": "synthetic", "config": cfg, "iterations": last["iterations"],
            "iterations_max": max(its_all), "true_relres": max(r["true_relres"] for r in reps[-1]),
            "replacements": last["replacements"], "converged": ok,
            "t_solve_matvec_s": last["matvec_ms"] / 1e3, "t_solve_apply_s": last["apply_ms"] / 1e3,
            "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks}
    it_oracle = oracle_fp64_count(args.workload)
    if it_oracle is not None:
        line["iterations_oracle_fp64"] = it_oracle

    if not args.no_extras and rank == 0 and world == 1 and args.workload == WORKLOAD:
        line.update(extras(torch, iedd, I, dev, stream, clocks, sms, flush))
        line["warm_start"] = warm_start_leg()
        cb = (cpu_baseline(args.workload, it_oracle) if it_oracle is not None else
              cpu_baseline(args.workload, last["iterations"],
                           iterations_from="the GPU's count: no stored oracle count for this workload"))
        cb["measured_end_to_end"] = oracle_measured_legs(per_step=False)
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def tensor_peak(clocks: dict):
    """The bf16 dense denominator for a tensor-core kernel timed inside the step: the measured burst
    peak when the SM clock sampled in the timed region sat at its maximum with no power cap, else
    the measured sustained (power-capped) peak."""
    burst = measured_peak("bf16_tflops", 1900.0)
    sustained = measured_peak("bf16_tflops_sustained", 1700.0)
    sm, mx = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    at_max = sm is not None and mx is not None and sm >= 0.97 * mx
    capped = "sw_power_cap" in (clocks.get("reasons") or [])
    if at_max and not capped:
        return burst, "burst"
    return sustained, "sustained"


def roofline_of(iedd, name, rep, clocks, sms, rs_stats=None):
    """Roofline record of the inner matvec (the dominant kernel) from its CUDA-event time inside
    pcg_solve (the library times every inner matvec on the launching stream).  For the RS-CBD
    workload the dominant kernels are the factor's rs_id and rs_elim (the library times their
    launches with CUDA events on its stream and counts their algorithmic FP64 flops)."""
    W = WORKLOADS[name]
    if W["factor"] == "rs" and rs_stats:
        flops = rs_stats["id_flops"] + rs_stats["elim_flops"]
        t = (rs_stats["id_ms"] + rs_stats["elim_ms"]) / 1e3
        achieved = flops / t
        peak = FP64_NOMINAL_TFLOPS * 1e12
        ncu = NCU_RS.get(rs_source_hash(), {})
        fma = iedd.ie_fp64_fma_rate(0)
        return ({"bound": "alu", "achieved": achieved / 1e12, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                 "frac": achieved / peak, "fp64_fma_measured_tflops": fma, "frac_of_measured_fma": achieved / 1e12 / fma,
                 "traffic": ncu.get("traffic"), "kernel": "rs_id + rs_elim (RS factor)",
                 "launch_ms": t * 1e3, "fp64_flops": flops, "id_ms": rs_stats["id_ms"],
                 "elim_ms": rs_stats["elim_ms"], "fp64_pipe_ncu": ncu.get("fp64_pipe"),
                 "peak_basis": (f"GB300 FP64 {FP64_NOMINAL_TFLOPS} TFLOP/s nominal (no FP64 peak in the pool's "
                                "measured peaks; fp64_fma_measured_tflops: this device's FP64 FMA loop, "
                                "ie_fp64_fma_rate); work = the factor's algorithmic FP64 flops (ID: initial norms, 4 flops per row "
                                "and remaining column per Gram-Schmidt step, back substitution; elimination: M, B_rr, Cholesky, triangular "
                                "inverse, L^-T L^-1, X, B_ss) / the summed CUDA-event time of its rs_id and rs_elim "
                                "launches")}, False)
    dim_w, n_w, nr = W["dim"], W["n"], W["seeds"]
    N = n_w ** dim_w
    prec = iedd.IE_FP64 if W["precision"] == "fp64" else iedd.IE_MIXED
    pairs = float(N) * (N - 1)
    mv_launch_s = rep["matvec_ms"] / max(rep["matvecs"], 1) / 1e3
    f_mhz = clocks.get("sm_mhz") or 2070.0
    kz_inner = prec == iedd.IE_MIXED and dim_w == 2 and n_w % 128 == 0 and n_w <= 4096
    if kz_inner:
        # 2D: the exact tensor-core matvec (Ozaki scheme), 21 BF16 digit products (2 flops each) per pair
        bf16, kind = tensor_peak(clocks)
        peak = bf16 * 1e12
        achieved = pairs * nr * 2.0 * KZ_PRODUCTS_PER_PAIR / mv_launch_s
        fp32_pair_peak = sms * FP32_LANES_PER_SM / FP32_OPS_PER_PAIR_K2 * f_mhz * 1e6
        ncu = NCU_KZ.get((tc_exact_source_hash(), n_w), {})
        roofline = {"bound": "tensor", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": ncu.get("traffic"), "kernel": "kz_matvec_tc",
                    "launch_ms": mv_launch_s * 1e3, "launches": rep["matvecs"],
                    "tensor_pipe_ncu": ncu.get("tensor_pipe"),
                    "peak_kind": kind,
                    "pairs_per_s": pairs * nr / mv_launch_s,
                    "pairs_vs_fp32_pair_peak": pairs * nr / mv_launch_s / fp32_pair_peak,
                    "peak_basis": (f"bf16 dense {bf16:.1f} TFLOP/s {kind} (of measured; burst when the sampled "
                                   f"SM clock stayed at max with no power cap, else sustained); work = "
                                   f"{KZ_PRODUCTS_PER_PAIR} BF16 digit products (2 flops each) per pair x N(N-1) "
                                   f"pairs per launch; pairs_vs_fp32_pair_peak against "
                                   f"{fp32_pair_peak / 1e12:.2f} Tpairs/s, the FP32-pipe peak of the "
                                   "double-float kernel")}
    elif prec == iedd.IE_MIXED and dim_w == 2:
        per_clk = FP32_LANES_PER_SM / FP32_OPS_PER_PAIR_K2
        peak = sms * per_clk * f_mhz * 1e6
        achieved = pairs * nr / mv_launch_s
        roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpairs/s",
                    "frac": achieved / peak, "traffic": NCU_TRAFFIC.get(k2_source_hash()) if n_w == 512 else None,
                    "kernel": "k2_accurate_2d<true,1>",
                    "peak_basis": (f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes / {FP32_OPS_PER_PAIR_K2} FP32 ops per "
                                   f"pair x {f_mhz:.0f} MHz (median SM clock sampled in the timed region)")}
    elif prec == iedd.IE_MIXED and nr >= 16:
        # 3D batch: the tcgen05 kernel, 3 TF32 MMAs (3xTF32 split) per pair and right-hand side,
        # against the TF32 dense peak = measured bf16 peak x the nominal TF32/bf16 ratio
        bf16, kind = tensor_peak(clocks)
        peak = bf16 * TF32_PER_BF16 * 1e12
        achieved = pairs * nr * 6.0 / mv_launch_s
        ncu = NCU_K1W.get((tc_matvec_source_hash(), n_w), {})
        roofline = {"bound": "tensor", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": ncu.get("traffic"), "kernel": "k1w_matvec_tc<3>",
                    "tensor_pipe_ncu": ncu.get("tensor_pipe"), "peak_kind": kind,
                    "pair_rhs_per_s": pairs * nr / mv_launch_s,
                    "peak_basis": (f"TF32 dense = {bf16:.1f} TFLOP/s bf16 {kind} (of measured) x {TF32_PER_BF16:.3f} "
                                   "(nominal 1.1 / 2.25 PFLOP/s); work = 3 TF32 products (hi hi, hi lo, lo hi; 2 flops "
                                   "each) per pair per RHS")}
    elif prec == iedd.IE_MIXED:
        # batched FP32 kernel: one FFMA per pair and right-hand side dominates (entries amortised)
        peak = sms * FP32_LANES_PER_SM * f_mhz * 1e6
        achieved = pairs * nr / mv_launch_s
        roofline = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair-rhs/s",
                    "frac": achieved / peak, "traffic": None, "kernel": "k1m_matvec_f32<3,64>",
                    "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FFMA/clk x {f_mhz:.0f} MHz (one FFMA per pair per RHS)"}
    else:
        achieved = pairs * nr / mv_launch_s
        roofline = {"bound": "fp64", "achieved": achieved / 1e9, "peak": None, "unit": "Gpairs/s", "frac": None,
                    "traffic": None, "kernel": "kd_matvec_f64",
                    "peak_basis": "FP64 log per pair; no measured FP64 peak on this pool"}
    return roofline, kz_inner


def warm_start_leg(fields: int = 16):
    """The learned warm start on its own workload (2D 256^2, Schwarz 16 x 16 partitions, 2-cell
    overlap, held-out GRF fields with seeds 0..fields-1, 1e-8 true residual):
    - per field, one at a time: zero-start mixed PCG against the U-Net start (ws_predict + pcg_solve
      with the fallback start);
    - batched: all fields in one ws_predict and one pcg_solve call, zero start and U-Net start
      (mixed precision + batching + warm start, per field);
    - plain FP64 GPU PCG on field 0: FP64 factor, the FP64 regenerated matvec inside the iteration
      and for the residual.
    Solve times exclude the factor (shared by all fields); the factor times are listed beside."""
    import numpy as np
    import torch

    from paper_2108_12574_gb300 import iedd
    from paper_2108_12574_gb300 import warmstart as WS
    if not os.path.exists(WS.WEIGHTS):
        return {"unavailable": "trained weights not present"}
    prob, part, fac = WS.setup()
    model = WS.load_model()
    WS.evaluate(model, prob, fac, [fields])  # warm-up
    s = WS.summarize(WS.evaluate(model, prob, fac, list(range(fields))))
    s["workload"] = "ie2d_n256_schwarz_m16_d2"

    F = torch.from_numpy(WS.fields(list(range(fields)), prob.n)).cuda()
    batched = {}
    for start in ("zero", "warm", "zero", "warm"):  # the first pair warms up
        U = torch.zeros_like(F)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if start == "warm":
            model.predict(prob, F, U)
        reps = iedd.pcg_solve(prob, fac, F, U, tol=TOL, precision=iedd.IE_MIXED, use_x0=2 if start == "warm" else 0)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        batched[start] = {"per_field_s": t / fields, "total_s": t,
                          "iterations_mean": float(np.mean([r["iterations"] for r in reps])),
                          "max_true_relres": float(max(r["true_relres"] for r in reps))}
    s["batched"] = batched

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fac64 = iedd.dd_factor(prob, part, iedd.IE_FP64)
    torch.cuda.synchronize()
    t_fac64 = time.perf_counter() - t0
    f = F[0].contiguous()
    u = torch.zeros_like(f)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = iedd.pcg_solve(prob, fac64, f, u, tol=TOL, precision=iedd.IE_FP64, inner=16, residual=16)[0]
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    s["fp64_plain"] = {"value": t64, "unit": "s", "iterations": r["iterations"], "true_relres": r["true_relres"],
                       "factor_s": t_fac64, "basis": "field 0 (seed 0), FP64 factor, FP64 regenerated matvec inside "
                       "the iteration and for the residual, measured in full"}
    s["speedup_vs_fp64_plain"] = {"per_field_warm": t64 / s["time_warm_s"],
                                  "batched_warm": t64 / batched["warm"]["per_field_s"]}
    fac64.close()
    fac.close(); part.close(); prob.close()
    return s


def max_over_ranks(v: float, dist=None, device=None) -> float:
    """Largest value over the ranks of the default process group (v itself without one)."""
    if dist is None or not dist.is_initialized():
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def timed_solves(torch, iedd, dev, stream, name, steps, inner=0, factor=None, precision=None, flush=None):
    """Time ``steps`` whole steps (discretize + partition + factor + pcg_solve) of a workload with
    CUDA events on the library's stream, L2 flushed before each; returns (mean s, last reports)."""
    W = WORKLOADS[name]
    F = workload_rhs(name)
    f = torch.from_numpy(F.T.copy() if F.shape[1] > 1 else F[:, 0].copy()).to(dev)
    u = torch.zeros_like(f)
    fprec = factor if factor is not None else (iedd.IE_FP64 if W["factor"] == "fp64" else iedd.IE_MIXED)
    if W["factor"] == "rs":
        fprec = None
    prec = precision if precision is not None else (iedd.IE_FP64 if W["precision"] == "fp64" else iedd.IE_MIXED)
    if flush is None:
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    if not inner:
        inner = inner_of(iedd, W)

    def step():
        prob = iedd.ie_discretize(W["dim"], W["n"], device=dev.index)
        part, fac = make_factor(iedd, prob, W, stream, fprec)
        reps = iedd.pcg_solve(prob, fac, f, u, tol=TOL, precision=prec, inner=inner, replace_every=REPLACE_EVERY,
                              stream=stream)
        fac.close(); part.close(); prob.close()
        return reps
    u.zero_()
    step()
    ms = []
    for _ in range(steps):
        flush.fill_(1.0)
        u.zero_()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    return statistics.mean(ms) / 1e3, reps


def extras(torch, iedd, I, dev, stream, clocks, sms, flush):
    """Extra legs of the default run: the 512^2 workload's whole step; each matvec kernel alone;
    the step with the paper's FFT matvec (mixed and FP64) and with the previous double-float
    inner matvec; the plain FP64 GPU solve (timed per component, scaled: one regenerated FP64
    matvec of the 1024^2 workload takes over a minute); CBD against Schwarz; the stored-matrix
    fallback's bandwidth."""
    out = {}
    t512, reps512 = timed_solves(torch, iedd, dev, stream, "ie2d_n512_schwarz_m32_d2", 3, flush=flush)
    r512, _ = roofline_of(iedd, "ie2d_n512_schwarz_m32_d2", reps512[0], clocks, sms)
    out["ie2d_n512_schwarz_m32_d2"] = {"value": t512, "unit": "s", "iterations": reps512[0]["iterations"],
                                       "iterations_oracle_fp64": oracle_fp64_count("ie2d_n512_schwarz_m32_d2"),
                                       "true_relres": reps512[0]["true_relres"], "roofline": r512}

    def t_mv(prob, x, y, prec, reps):
        iedd.ie_matvec(prob, x, y, prec, stream=stream)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            iedd.ie_matvec(prob, x, y, prec, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps / 1e3

    bf16_burst = measured_peak("bf16_tflops", 1900.0)
    mats = {}
    for n in (512, 1024):
        N = n * n
        pairs = float(N) * (N - 1)
        x = torch.from_numpy(I.uniform_rhs(N, 0)).to(dev)
        y = torch.zeros_like(x)
        prob = iedd.ie_discretize(2, n, device=dev.index)
        t_kz = t_mv(prob, x, y, iedd.IE_TENSOR_EXACT, 10 if n == 512 else 4)
        t_fft = t_mv(prob, x, y, iedd.IE_FFT, 20)
        row = {"kz_ms": t_kz * 1e3, "kz_tflops_bf16": 42.0 * pairs / t_kz / 1e12,
               "kz_frac_of_burst": 42.0 * pairs / t_kz / 1e12 / bf16_burst, "kz_gpairs_s": pairs / t_kz / 1e9,
               "fft_ms": t_fft * 1e3}
        if n == 512:
            t_k1 = t_mv(prob, x, y, iedd.IE_MIXED, 5)
            t_k2 = t_mv(prob, x, y, iedd.IE_ACCURATE, 5)
            t_64 = t_mv(prob, x, y, iedd.IE_FP64, 1)
            row.update({"k2_double_float_gpairs_s": pairs / t_k2 / 1e9, "k1_fp32_sfu_gpairs_s": pairs / t_k1 / 1e9,
                        "kd_fp64_gpairs_s": pairs / t_64 / 1e9, "kd_fp64_ms": t_64 * 1e3})
        mats[f"n{n}"] = row
        prob.close()
    mats["basis"] = ("each matvec alone, CUDA events, 2D uniform[-1,1] x; KZ = the exact tensor-core matvec "
                     "(21 BF16 digit products per pair, 2 flops each) against the measured bf16 burst peak "
                     f"{bf16_burst:.1f} TFLOP/s (of measured); FFT = the paper's FP64 matvec on the 2n-periodic grid")
    out["matvecs"] = mats

    # the paper's FFT matvec as the inner matvec of the 1024^2 step, FP32 inverses and FP64 factors
    fft = {}
    for variant, fprec, prec in (("mixed", iedd.IE_MIXED, iedd.IE_MIXED), ("fp64", iedd.IE_FP64, iedd.IE_FP64)):
        t, reps = timed_solves(torch, iedd, dev, stream, WORKLOAD, 2, inner=iedd.IE_FFT, factor=fprec,
                               precision=prec, flush=flush)
        fft[variant] = {"value": t, "unit": "s", "iterations": reps[0]["iterations"],
                        "true_relres": reps[0]["true_relres"], "t_solve_matvec_s": reps[0]["matvec_ms"] / 1e3,
                        "t_solve_apply_s": reps[0]["apply_ms"] / 1e3}
    out["fft_solve"] = fft
    t, reps = timed_solves(torch, iedd, dev, stream, "ie2d_n512_schwarz_m32_d2", 2, inner=iedd.IE_ACCURATE,
                           flush=flush)
    out["k2_inner_solve_n512"] = {"value": t, "unit": "s", "iterations": reps[0]["iterations"],
                                  "note": "the 512^2 step with the double-float FP32-pipe matvec as inner matvec"}

    # plain FP64 GPU PCG on the 1024^2 workload: FP64 factor and apply measured at 1024^2, the
    # regenerated FP64 matvec measured at 512^2 and scaled by the pair count (compute-bound)
    W = WORKLOADS[WORKLOAD]
    n = W["n"]
    N = n * n
    x = torch.from_numpy(I.uniform_rhs(N, 0)).to(dev)
    z = torch.zeros_like(x)
    prob = iedd.ie_discretize(2, n, device=dev.index)
    part = iedd.dd_partition(prob, W["m"], W["delta"], iedd.DD_SCHWARZ)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    fac = iedd.dd_factor(prob, part, iedd.IE_FP64, stream=stream)
    torch.cuda.synchronize(dev)
    t_fac = time.perf_counter() - t0
    iedd.dd_apply(fac, x, z, stream=stream)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(5):
        iedd.dd_apply(fac, x, z, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_ap = e0.elapsed_time(e1) / 5 / 1e3
    fac.close(); part.close(); prob.close()
    scale = (float(N) * (N - 1)) / (512.0 ** 2 * (512.0 ** 2 - 1))
    t_64 = mats["n512"]["kd_fp64_ms"] / 1e3 * scale
    its = oracle_fp64_count(WORKLOAD) or fft["fp64"]["iterations"]
    out["fp64_plain"] = {"value": t_fac + (its + 1) * t_64 + its * t_ap, "unit": "s", "extrapolated": True,
                         "iterations": its,
                         "basis": (f"FP64 factor + {its} x (regenerated FP64 matvec + FP64 triangular-solve apply) + "
                                   "one FP64 true-residual matvec on this GPU; factor and apply measured at 1024^2, "
                                   f"the FP64 matvec measured at 512^2 and scaled by the pair count ({scale:.2f}x); "
                                   f"{its} = the FP64 iteration count at 1e-8"),
                         "parts_s": {"factor": t_fac, "matvec": t_64, "apply": t_ap}}
    out["cbd"] = cbd_leg(torch, iedd, I, dev, stream)
    out["cbd_rs"] = cbd_rs_leg(torch, iedd, dev, stream, flush)
    scale = {}
    for name in ("ie2d_n2048_cbd_rs_m256_d1", "ie3d_n64_cbd_rs_m8_d1"):
        t, reps = timed_solves(torch, iedd, dev, stream, name, 2, flush=flush)
        scale[name] = {"value": t, "unit": "s", "iterations": reps[0]["iterations"],
                       "true_relres": reps[0]["true_relres"], "t_solve_matvec_s": reps[0]["matvec_ms"] / 1e3,
                       "t_solve_apply_s": reps[0]["apply_ms"] / 1e3, "config": config_dict(name)}
    out["cbd_rs_scale"] = scale
    out["stored_matvec"] = stored_matvec_leg(torch, iedd, I, dev, stream)
    return out


def cbd_leg(torch, iedd, I, dev, stream, sizes=(128, 256), ell=0.1):
    """The paper's CBD preconditioner (Sec. 2.3: 2^d colour blocks, each the union of the extended
    boxes of one parity colour, factored densely) against Schwarz (one block per extended box) on
    the same 2D grids: boxes of 16 x 16 cells, 2-cell overlap, GRF l = 0.1, tol 1e-8, FFT matvec,
    FP32 factors and inverses on the tensor cores.  Times: dd_factor and pcg_solve (host clock
    around each, synchronized)."""
    out = {}
    for n in sizes:
        f = torch.from_numpy(I.grf(2, n, ell, 0)).to(dev)
        prob = iedd.ie_discretize(2, n, device=dev.index)
        row = {}
        for name, kind in (("schwarz", iedd.DD_SCHWARZ), ("cbd", iedd.DD_CBD)):
            part = iedd.dd_partition(prob, n // 16, 2, kind)
            nb, maxb = part.nblocks, part.max_block
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            fac = iedd.dd_factor(prob, part, iedd.IE_MIXED, stream=stream)
            torch.cuda.synchronize(dev)
            t_fac = time.perf_counter() - t0
            u = torch.zeros_like(f)
            iedd.pcg_solve(prob, fac, f, u, tol=TOL, inner=iedd.IE_FFT, stream=stream)  # warm-up
            u.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            rep = iedd.pcg_solve(prob, fac, f, u, tol=TOL, inner=iedd.IE_FFT, stream=stream)[0]
            torch.cuda.synchronize(dev)
            t_sol = time.perf_counter() - t0
            row[name] = {"blocks": nb, "max_block": maxb, "factor_s": t_fac, "solve_s": t_sol,
                         "iterations": rep["iterations"], "true_relres": rep["true_relres"],
                         "apply_ms_per_iteration": rep["apply_ms"] / max(rep["applies"], 1)}
            fac.close(); part.close()
        prob.close()
        out[f"n{n}"] = row
    return out


def cbd_rs_leg(torch, iedd, dev, stream, flush, name="ie2d_n1024_cbd_rs_m128_d1"):
    """The paper's CBD preconditioner with recursive-skeletonization subdomain factors (Sec. 4.3)
    on the same 1024^2 grid and right-hand side as the headline: whole steps (discretize +
    partition + RS factor + FP64 PCG with the FFT matvec), CUDA events, L2 flushed; the factor
    and the solve also timed apart (host clock, synchronized)."""
    t, reps = timed_solves(torch, iedd, dev, stream, name, 2, flush=flush)
    W = WORKLOADS[name]
    prob = iedd.ie_discretize(W["dim"], W["n"], device=dev.index)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    part, fac = make_factor(iedd, prob, W, stream)
    torch.cuda.synchronize(dev)
    t_fac = time.perf_counter() - t0
    levels, top = iedd.dd_rs_info(fac)
    fac.close(); part.close(); prob.close()
    rep = reps[0]
    return {"workload": name, "value": t, "unit": "s", "iterations": rep["iterations"],
            "iterations_oracle_fp64": rs_oracle_count(name), "true_relres": rep["true_relres"],
            "factor_s": t_fac, "t_solve_matvec_s": rep["matvec_ms"] / 1e3, "t_solve_apply_s": rep["apply_ms"] / 1e3,
            "apply_ms_per_iteration": rep["apply_ms"] / max(rep["applies"], 1), "levels": levels, "top_dofs": top,
            "config": config_dict(name), "cpu_baseline": rs_cpu_baseline(name, rep["iterations"])}


def rs_cpu_baseline(name: str, iterations: int, n_sample: int = 256):
    """The FP64 oracle's RS-CBD solve, timed on an n_sample^d grid with the workload's box size,
    overlap and eps (the RS factor and apply: the whole of that grid) and scaled to the workload by
    N, with the oracle's FFT matvec measured at the workload's size; total = factor + iterations x
    (matvec + apply).  Extrapolated, and labelled so."""
    from oracle import ie_oracle as O
    from oracle import rs_oracle as RS
    from paper_2108_12574_gb300 import inputs as I
    W = WORKLOADS[name]
    dim, n = W["dim"], W["n"]
    N, Ns = n ** dim, n_sample ** dim
    m_s = n_sample // (n // W["m"])
    t0 = time.perf_counter()
    F = RS.factor(dim, n_sample, m_s, W["delta"], W["eps"], 64 if dim == 2 else 256)
    t_fac = (time.perf_counter() - t0) * N / Ns
    t0 = time.perf_counter()
    RS.apply(F, I.uniform_rhs(Ns, 0))
    t_ap = (time.perf_counter() - t0) * N / Ns
    t0 = time.perf_counter()
    O.matvec_fft(dim, n, I.uniform_rhs(N, 0))
    t_mv = time.perf_counter() - t0
    return {"value": t_fac + iterations * (t_mv + t_ap), "unit": "s", "cores": oracle_cores(), "cpu": cpu_model(),
            "kind": "oracle", "workload": name, "extrapolated": True,
            "sample": (f"the oracle's RS factor and one apply on the whole {n_sample}^{dim} grid with the same box "
                       f"size ({m_s}^{dim} boxes), scaled by N to {n}^{dim}; its FFT matvec measured at {n}^{dim}; "
                       f"total = factor + {iterations} iterations x (matvec + apply); extrapolated"),
            "parts_s": {"factor": t_fac, "apply": t_ap, "matvec": t_mv}}


def rs_oracle_count(name: str):
    """The oracle's RS-CBD PCG count at 1e-8 (tests/golden/rs_counts.json, written by a script that
    calls only the oracle), or None."""
    key = {"ie2d_n1024_cbd_rs_m128_d1": "ie2d_n1024_cbd_m128"}.get(name)
    try:
        with open(os.path.join(ROOT, "tests", "golden", "rs_counts.json")) as fh:
            return int(json.load(fh)[key]["iterations"])
    except (OSError, KeyError, ValueError, TypeError):
        return None


def stored_matvec_leg(torch, iedd, I, dev, stream, n=256):
    """The stored-matrix fallback (dense FP32 A in HBM, 4 N^2 bytes streamed per product) against
    regenerating the entries, on the 2D 256^2 grid (N = 65536, 17.2 GB matrix)."""
    N = n * n
    prob = iedd.ie_discretize(2, n, device=dev.index)
    iedd.ie_store_matrix(prob, stream=stream)
    x = torch.from_numpy(I.uniform_rhs(N, 0)).to(dev)
    y = torch.zeros_like(x)

    def t(prec, reps=5):
        iedd.ie_matvec(prob, x, y, prec, stream=stream)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            iedd.ie_matvec(prob, x, y, prec, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps / 1e3

    ts, t2 = t(iedd.IE_STORED), t(iedd.IE_ACCURATE)
    iedd.ie_release_matrix(prob)
    gbs = 4.0 * N * N / ts / 1e9
    hbm = measured_peak("hbm_gbs", 6800.0)
    return {"workload": "2D n=256 (N=65536), dense FP32 A", "ms": ts * 1e3, "achieved_gbs": gbs,
            "hbm_peak_gbs": hbm, "frac": gbs / hbm, "regenerated_exact_ms": t2 * 1e3,
            "note": "peak = measured copy bandwidth (of measured)"}


if __name__ == "__main__":
    sys.exit(main())
