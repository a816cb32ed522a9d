"""Thin ctypes binding of libiedd (include/iedd.h): argument marshalling only.

Every compute step runs in the library's CUDA kernels.  The binding loads the in-tree
``_lib/libiedd.so`` and raises ``ImportError`` if it is missing -- there is no CPU fallback.

Vectors are torch tensors (CUDA or CPU) or numpy arrays, FP64, of shape (N,) or (nrhs, N)
with unit stride along N; a (nrhs, N) batch is the library's column-major N x nrhs layout
with ld = stride(0).  Host arrays are staged to the device by the library itself.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

IE_OK, IE_ERR_ARG, IE_ERR_CUDA, IE_ERR_OOM, IE_ERR_NOT_SPD = 0, -1, -2, -3, -4
IE_ERR_BREAKDOWN, IE_ERR_MAXIT, IE_ERR_STAGNATION, IE_ERR_TIMEOUT = -5, -6, -7, -8
IE_FP64, IE_MIXED, IE_ACCURATE, IE_STORED, IE_TENSOR, IE_FFT, IE_TENSOR_EXACT = 0, 1, 3, 5, 6, 9, 10
DD_JACOBI, DD_SCHWARZ, DD_CBD = 0, 1, 2
IE_GRID_TEXT, IE_GRID_TABLE = 0, 1

STATUS_NAMES = {0: "IE_OK", -1: "IE_ERR_ARG", -2: "IE_ERR_CUDA", -3: "IE_ERR_OOM", -4: "IE_ERR_NOT_SPD",
                -5: "IE_ERR_BREAKDOWN", -6: "IE_ERR_MAXIT", -7: "IE_ERR_STAGNATION", -8: "IE_ERR_TIMEOUT"}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libiedd.so")

# Every C-ABI symbol declared in include/iedd.h.
EXPORTS = ("ie_last_error", "ie_version", "ie_discretize", "ie_problem_info", "ie_destroy", "ie_matvec",
           "dd_partition", "dd_partition_info", "dd_partition_export", "dd_partition_destroy", "dd_factor",
           "dd_factor_destroy", "dd_apply", "ie_kernel_launches", "pcg_default_opts", "pcg_solve",
           "ie_matvec_noalloc", "ws_create", "ws_destroy", "ws_num_params", "ws_get_params", "ws_set_params",
           "ws_forward_raw", "ws_backward_raw", "ws_train_step", "ws_predict", "ie_store_matrix",
           "ie_release_matrix", "ie_autotune", "ie_autotune_report", "dd_factor_rs", "dd_rs_info", "dd_rs_export", "ie_fp64_fma_rate")
IE_NOALLOC_MAX_N = 4194304 - 1024


class IEError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class PcgOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_it", ctypes.c_int), ("precision", ctypes.c_int),
                ("replace_every", ctypes.c_int), ("use_x0", ctypes.c_int), ("timeout_s", ctypes.c_double),
                ("check_every", ctypes.c_int), ("verify", ctypes.c_int), ("inner", ctypes.c_int),
                ("residual", ctypes.c_int)]


class RsOpts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("nproxy", ctypes.c_int), ("rho", ctypes.c_double)]


class PcgReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("replacements", ctypes.c_int), ("status", ctypes.c_int),
                ("x0_used", ctypes.c_int), ("recursive_relres", ctypes.c_double), ("true_relres", ctypes.c_double),
                ("matvecs", ctypes.c_int), ("applies", ctypes.c_int), ("matvec_ms", ctypes.c_double),
                ("apply_ms", ctypes.c_double), ("accurate_matvecs", ctypes.c_int), ("accurate_mode", ctypes.c_int),
                ("accurate_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("pad")}


_LIB = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libiedd.so; raises ImportError if it was not built (build with __graft_entry__.build())."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise ImportError(f"libiedd.so not found at {path}: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i, ll, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "ie_last_error": (ctypes.c_char_p, []),
        "ie_version": (ctypes.c_char_p, []),
        "ie_discretize": (i, [i, i, d, i, i, P(vp)]),
        "ie_problem_info": (i, [vp, P(i), P(i), P(ll), P(d), P(d)]),
        "ie_destroy": (None, [vp]),
        "ie_matvec": (i, [vp, vp, vp, i, ll, i, vp]),
        "dd_partition": (i, [vp, i, i, i, P(vp)]),
        "dd_partition_info": (i, [vp, P(i), P(ll), P(i)]),
        "dd_partition_export": (i, [vp, vp, vp]),
        "dd_partition_destroy": (None, [vp]),
        "dd_factor": (i, [vp, vp, i, P(vp), P(i), vp]),
        "dd_factor_destroy": (None, [vp]),
        "dd_factor_rs": (i, [vp, vp, P(RsOpts), P(vp), vp]),
        "dd_rs_info": (i, [vp, P(i), vp, vp, vp]),
        "dd_rs_export": (i, [vp, i, i, P(i), P(ll), vp, vp, vp]),
        "ie_fp64_fma_rate": (i, [i, P(d)]),
        "dd_apply": (i, [vp, vp, vp, i, ll, vp]),
        "ie_kernel_launches": (ll, [i]),
        "ie_autotune": (i, [i]),
        "ie_autotune_report": (ctypes.c_char_p, []),
        "ie_store_matrix": (i, [vp, vp]),
        "ie_release_matrix": (i, [vp]),
        "ie_matvec_noalloc": (i, [i, i, d, i, vp, vp, vp]),
        "ws_create": (i, [i, ctypes.c_ulonglong, P(vp)]),
        "ws_destroy": (None, [vp]),
        "ws_num_params": (ll, [vp]),
        "ws_get_params": (i, [vp, vp]),
        "ws_set_params": (i, [vp, vp]),
        "ws_forward_raw": (i, [vp, vp, vp, i, i, vp]),
        "ws_backward_raw": (i, [vp, vp, vp, vp, i, i, vp]),
        "ws_train_step": (i, [vp, vp, vp, vp, i, ll, ctypes.c_float, P(d), vp]),
        "ws_predict": (i, [vp, vp, vp, vp, i, ll, vp]),
        "pcg_default_opts": (None, [P(PcgOpts)]),
        "pcg_solve": (i, [vp, vp, vp, vp, i, ll, P(PcgOpts), P(PcgReport), vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(st: int):
    if st != IE_OK:
        raise IEError(st, load_library().ie_last_error().decode())


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _vec(x, N: int, writable: bool = False):
    """(pointer, nrhs, ld, keepalive) of an FP64 vector / batch."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64:
            raise TypeError("vectors must be float64")
        if writable and not x.flags.writeable:
            raise ValueError("output array is read-only")
        if x.ndim == 1:
            if x.shape[0] != N or x.strides[0] != 8:
                raise ValueError("expected a contiguous vector of length N")
            return ctypes.c_void_p(x.ctypes.data), 1, N, x
        if x.ndim == 2 and x.shape[1] == N and x.strides[1] == 8 and x.strides[0] % 8 == 0:
            return ctypes.c_void_p(x.ctypes.data), x.shape[0], x.strides[0] // 8, x
        raise ValueError("expected shape (N,) or (nrhs, N) with unit stride along N")
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError("vectors must be torch tensors or numpy arrays")
    if x.dtype != torch.float64:
        raise TypeError("vectors must be float64")
    if x.dim() == 1:
        if x.shape[0] != N or x.stride(0) != 1:
            raise ValueError("expected a contiguous vector of length N")
        return ctypes.c_void_p(x.data_ptr()), 1, N, x
    if x.dim() == 2 and x.shape[1] == N and x.stride(1) == 1:
        return ctypes.c_void_p(x.data_ptr()), x.shape[0], x.stride(0), x
    raise ValueError("expected shape (N,) or (nrhs, N) with unit stride along N")


class _Handle:
    _destroy = None

    def __init__(self, ptr):
        self._ptr = ptr

    @property
    def ptr(self):
        if self._ptr is None:
            raise ValueError("handle already destroyed")
        return self._ptr

    def close(self):
        if getattr(self, "_ptr", None) is not None and _LIB is not None:
            getattr(_LIB, self._destroy)(self._ptr)
        self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Problem(_Handle):
    _destroy = "ie_destroy"

    def __init__(self, ptr):
        super().__init__(ptr)
        dim, n, N, h, diag = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
        _check(load_library().ie_problem_info(ptr, ctypes.byref(dim), ctypes.byref(n), ctypes.byref(N),
                                              ctypes.byref(h), ctypes.byref(diag)))
        self.dim, self.n, self.N, self.h, self.diag = dim.value, n.value, N.value, h.value, diag.value


class Partition(_Handle):
    _destroy = "dd_partition_destroy"

    def __init__(self, ptr, problem):
        super().__init__(ptr)
        self.problem = problem  # keep the problem alive
        nb, tot, mx = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_int()
        _check(load_library().dd_partition_info(ptr, ctypes.byref(nb), ctypes.byref(tot), ctypes.byref(mx)))
        self.nblocks, self.total, self.max_block = nb.value, tot.value, mx.value

    def export(self):
        """List of index arrays (ascending global indices), one per subdomain."""
        offs = np.zeros(self.nblocks + 1, dtype=np.int64)
        idx = np.zeros(max(self.total, 1), dtype=np.int32)
        _check(load_library().dd_partition_export(self.ptr, offs.ctypes.data, idx.ctypes.data))
        return [idx[offs[i]:offs[i + 1]].astype(np.int64) for i in range(self.nblocks)]


class Factor(_Handle):
    _destroy = "dd_factor_destroy"

    def __init__(self, ptr, problem, partition, precision):
        super().__init__(ptr)
        self.problem, self.partition, self.precision = problem, partition, precision

    def close(self):  # the factor must go before its problem and partition
        super().close()


def ie_version() -> str:
    return load_library().ie_version().decode()


def ie_discretize(dim: int, n: int, a_shift: float = 0.0, grid: int = IE_GRID_TEXT, device: int = 0) -> Problem:
    out = ctypes.c_void_p()
    _check(load_library().ie_discretize(dim, n, a_shift, grid, device, ctypes.byref(out)))
    return Problem(out)


def ie_matvec(prob: Problem, x, y, precision: int = IE_MIXED, stream=None):
    px, k, ld, _kx = _vec(x, prob.N)
    py, k2, ld2, _ky = _vec(y, prob.N, writable=True)
    if k != k2 or ld != ld2:
        raise ValueError("x and y must have the same shape and stride")
    _check(load_library().ie_matvec(prob.ptr, px, py, k, ld, precision, _stream(stream)))
    return y


def ie_store_matrix(prob: Problem, stream=None):
    _check(load_library().ie_store_matrix(prob.ptr, _stream(stream)))


def ie_release_matrix(prob: Problem):
    _check(load_library().ie_release_matrix(prob.ptr))


def dd_partition(prob: Problem, m: int, delta: int, kind: int = DD_SCHWARZ) -> Partition:
    out = ctypes.c_void_p()
    _check(load_library().dd_partition(prob.ptr, m, delta, kind, ctypes.byref(out)))
    return Partition(out, prob)


def dd_factor(prob: Problem, part: Partition, precision: int = IE_MIXED, stream=None) -> Factor:
    out = ctypes.c_void_p()
    info = ctypes.c_int(-1)
    st = load_library().dd_factor(prob.ptr, part.ptr, precision, ctypes.byref(out), ctypes.byref(info),
                                  _stream(stream))
    fac = Factor(out, prob, part, precision) if out.value else None
    if st != IE_OK:
        err = IEError(st, load_library().ie_last_error().decode())
        err.info = info.value
        if fac is not None:
            fac.close()
        raise err
    return fac


def dd_factor_rs(prob: Problem, part: Partition, eps: float = 0.0, nproxy: int = 0, rho: float = 0.0,
                 stream=None) -> Factor:
    """RS factors of the CBD subdomains (0 selects the library's default for eps, nproxy, rho)."""
    out = ctypes.c_void_p()
    opts = RsOpts(eps, nproxy, rho)
    _check(load_library().dd_factor_rs(prob.ptr, part.ptr, ctypes.byref(opts), ctypes.byref(out), _stream(stream)))
    return Factor(out, prob, part, IE_FP64)


def dd_rs_info(fac: Factor, stats: bool = False):
    """(levels per colour, last-level DOFs per colour) of an RS factor; with ``stats`` also a dict
    of the factor's FP64 flops and kernel times (id_flops, elim_flops, id_ms, elim_ms)."""
    nc = ctypes.c_int()
    lv = np.zeros(8, dtype=np.int32)
    tp = np.zeros(8, dtype=np.int32)
    st = np.zeros(4, dtype=np.float64)
    _check(load_library().dd_rs_info(fac.ptr, ctypes.byref(nc), lv.ctypes.data, tp.ctypes.data, st.ctypes.data))
    out = (lv[:nc.value].tolist(), tp[:nc.value].tolist())
    if stats:
        return out + (dict(zip(("id_flops", "elim_flops", "id_ms", "elim_ms"), st.tolist())),)
    return out


def dd_rs_export(fac: Factor, colour: int, level: int):
    """Regions of one colour at one level (1-based; the last level is levels[colour] + 1): a list of
    (points: int64 global indices with the skeletons first in pivot order, rank)."""
    lib = load_library()
    nreg, tot = ctypes.c_int(), ctypes.c_longlong()
    _check(lib.dd_rs_export(fac.ptr, colour, level, ctypes.byref(nreg), ctypes.byref(tot), None, None, None))
    offs = np.zeros(nreg.value + 1, dtype=np.int64)
    pts = np.zeros(max(tot.value, 1), dtype=np.int32)
    rk = np.zeros(max(nreg.value, 1), dtype=np.int32)
    _check(lib.dd_rs_export(fac.ptr, colour, level, ctypes.byref(nreg), ctypes.byref(tot), offs.ctypes.data,
                            pts.ctypes.data, rk.ctypes.data))
    return [(pts[offs[b]:offs[b + 1]].astype(np.int64), int(rk[b])) for b in range(nreg.value)]


def ie_fp64_fma_rate(device: int = 0) -> float:
    """The device's measured FP64 FMA throughput in TFLOP/s (instrumentation)."""
    out = ctypes.c_double()
    _check(load_library().ie_fp64_fma_rate(device, ctypes.byref(out)))
    return out.value


def dd_apply(fac: Factor, r, z, stream=None):
    pr, k, ld, _kr = _vec(r, fac.problem.N)
    pz, k2, ld2, _kz = _vec(z, fac.problem.N, writable=True)
    if k != k2 or ld != ld2:
        raise ValueError("r and z must have the same shape and stride")
    _check(load_library().dd_apply(fac.ptr, pr, pz, k, ld, _stream(stream)))
    return z


def ie_matvec_noalloc(dim: int, n: int, x, y, a_shift: float = 0.0, grid: int = IE_GRID_TEXT, stream=None):
    """y = A x (FP32 SFU kernel) with no device allocation; x, y: CUDA FP64 vectors of length n^dim."""
    N = n ** dim
    px, k, _, _kx = _vec(x, N)
    py, k2, _, _ky = _vec(y, N, writable=True)
    if k != 1 or k2 != 1:
        raise ValueError("ie_matvec_noalloc takes one right-hand side")
    _check(load_library().ie_matvec_noalloc(dim, n, a_shift, grid, px, py, _stream(stream)))
    return y


class WarmStartModel(_Handle):
    """The warm-start U-Net (ws_* calls)."""
    _destroy = "ws_destroy"

    @property
    def nparams(self) -> int:
        return int(load_library().ws_num_params(self.ptr))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.nparams, dtype=np.float32)
        _check(load_library().ws_get_params(self.ptr, out.ctypes.data))
        return out

    def set_params(self, theta) -> None:
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        if theta.size != self.nparams:
            raise ValueError("wrong parameter count")
        _check(load_library().ws_set_params(self.ptr, theta.ctypes.data))

    def forward_raw(self, x: np.ndarray, stream=None) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32)
        B, n = x.shape[0], x.shape[1]
        out = np.zeros((B, n, n), dtype=np.float32)
        _check(load_library().ws_forward_raw(self.ptr, x.ctypes.data, out.ctypes.data, B, n, _stream(stream)))
        return out

    def backward_raw(self, x: np.ndarray, dout: np.ndarray, stream=None) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32)
        dout = np.ascontiguousarray(dout, dtype=np.float32)
        B, n = x.shape[0], x.shape[1]
        g = np.zeros(self.nparams, dtype=np.float32)
        _check(load_library().ws_backward_raw(self.ptr, x.ctypes.data, dout.ctypes.data, g.ctypes.data, B, n,
                                              _stream(stream)))
        return g

    def train_step(self, prob: Problem, f, u, lr: float, stream=None) -> float:
        pf, k, ld, _kf = _vec(f, prob.N)
        pu, k2, ld2, _ku = _vec(u, prob.N)
        if k != k2 or ld != ld2:
            raise ValueError("f and u must have the same shape and stride")
        loss = ctypes.c_double(0.0)
        _check(load_library().ws_train_step(self.ptr, prob.ptr, pf, pu, k, ld, lr, ctypes.byref(loss),
                                            _stream(stream)))
        return loss.value

    def predict(self, prob: Problem, f, u0, stream=None):
        pf, k, ld, _kf = _vec(f, prob.N)
        pu, k2, ld2, _ku = _vec(u0, prob.N, writable=True)
        if k != k2 or ld != ld2:
            raise ValueError("f and u0 must have the same shape and stride")
        _check(load_library().ws_predict(self.ptr, prob.ptr, pf, pu, k, ld, _stream(stream)))
        return u0


def ws_create(device: int = 0, seed: int = 0) -> WarmStartModel:
    out = ctypes.c_void_p()
    _check(load_library().ws_create(device, seed, ctypes.byref(out)))
    return WarmStartModel(out)


def ie_kernel_launches(reset: bool = False) -> int:
    return load_library().ie_kernel_launches(1 if reset else 0)


def ie_autotune(mode: int = -1) -> bool:
    """Autotuner switch: -1 query, 0 off, 1 on, 2 forget cached choices; returns the previous state."""
    return bool(load_library().ie_autotune(mode))


def ie_autotune_report() -> str:
    return load_library().ie_autotune_report().decode()


def pcg_default_opts() -> PcgOpts:
    o = PcgOpts()
    load_library().pcg_default_opts(ctypes.byref(o))
    return o


def pcg_solve(prob: Problem, fac: Factor, f, u, opts: PcgOpts | None = None, stream=None, check=True, **kw):
    """Solve A u = f; returns the list of per-column reports.  ``kw`` overrides option fields."""
    o = opts if opts is not None else pcg_default_opts()
    for key, val in kw.items():
        setattr(o, key, val)
    pf, k, ld, _kf = _vec(f, prob.N)
    pu, k2, ld2, _ku = _vec(u, prob.N, writable=True)
    if k != k2 or ld != ld2:
        raise ValueError("f and u must have the same shape and stride")
    reps = (PcgReport * k)()
    st = load_library().pcg_solve(prob.ptr, fac.ptr, pf, pu, k, ld, ctypes.byref(o), reps, _stream(stream))
    out = [r.as_dict() for r in reps]
    if check and st != IE_OK:
        err = IEError(st, load_library().ie_last_error().decode())
        err.reports = out
        raise err
    return out
