"""ie_matvec_noalloc: the allocation-free matvec entry point, through the C ABI (needs a GPU).

Some callers cannot allocate device memory (code running inside an allocator, a memory-capped
host framework, or a process that reserved all its memory up front).  ie_matvec_noalloc gives
them y = A x with the FP32 SFU kernel, using only a static device array as scratch.  These tests
check it against the allocating entry point ie_matvec(IE_MIXED) and against the FP64 oracle's
direct sum, within the FP32 matvec tolerance of the other parity tests (4e-6 ||A||_inf
||x||_inf), on two calls in a row with different inputs (the shared scratch keeps the previous
call's contents), for both grid conventions and a second-kind shift, and check that oversized
problems, host memory and (with two GPUs) another device's memory are rejected.  The file is
named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ie_oracle as O  # noqa: E402
from paper_2108_12574_gb300 import iedd  # noqa: E402
from paper_2108_12574_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    torch.cuda.init()
    return iedd.load_library()


def _scale(dim, n, x, grid=O.GRID_TEXT, a_shift=0.0):
    rows = O.matvec_direct(dim, n, np.ones(n ** dim), rows=np.array([0, (n ** dim) // 2]), convention=grid,
                           a_shift=abs(a_shift))
    return 2.0 * float(np.max(np.abs(rows))) * float(np.max(np.abs(x)))


def _noalloc(lib, dim, n, a_shift, grid, x, y):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.ie_matvec_noalloc(dim, n, a_shift, grid, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                               stream)
    assert st == iedd.IE_OK, lib.ie_last_error()
    torch.cuda.synchronize()


@pytest.mark.parametrize("dim,n,grid,a_shift", [(2, 64, O.GRID_TEXT, 0.0), (2, 512, O.GRID_TEXT, 0.0),
                                                (3, 24, O.GRID_TEXT, 0.0), (2, 37, O.GRID_TEXT, 0.0),
                                                (2, 64, O.GRID_TEXT, 0.5), (3, 24, O.GRID_TABLE, 0.0),
                                                (2, 40, O.GRID_TABLE, -0.25)])
def test_noalloc_matches_ie_matvec_and_oracle_two_calls_in_a_row(lib, dim, n, grid, a_shift):
    N = n ** dim
    prob = iedd.ie_discretize(dim, n, a_shift=a_shift, grid=grid)
    rows = None if N <= 20000 else np.unique(np.concatenate([[0, N - 1, N // 2 + n // 2],
                                                            np.random.default_rng(n).integers(0, N, 29)]))
    scale_of = lambda xh: _scale(dim, n, xh, grid, a_shift)  # noqa: E731
    for seed in (11, 12):  # two calls in a row, different inputs
        xh = I.uniform_rhs(N, seed)
        x = torch.from_numpy(xh).cuda()
        y_ref = torch.zeros_like(x)
        iedd.ie_matvec(prob, x, y_ref, iedd.IE_MIXED)
        y = torch.full_like(x, float("nan"))
        _noalloc(lib, dim, n, a_shift, grid, x, y)
        tol = 4e-6 * scale_of(xh)
        err = float((y - y_ref).abs().max())
        assert err <= tol, (seed, err)
        # the FP64 oracle's direct sum (all rows, or sampled rows of the 512^2 grid)
        ref = O.matvec_direct(dim, n, xh, rows=rows, convention=grid, a_shift=a_shift)
        got = y.cpu().numpy() if rows is None else y.cpu().numpy()[rows]
        err_o = float(np.max(np.abs(got - ref)))
        assert err_o <= tol, (seed, err_o)


def test_noalloc_rejects_oversized_problems(lib):
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    st = lib.ie_matvec_noalloc(2, 2048, 0.0, iedd.IE_GRID_TEXT, ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(y.data_ptr()), None)
    assert st == iedd.IE_ERR_ARG
    assert b"exceeds" in lib.ie_last_error()
    assert 2048 * 2048 > iedd.IE_NOALLOC_MAX_N >= 2047 * 2047


def test_noalloc_rejects_host_pointers(lib):
    xh = np.zeros(16 * 16)
    yh = np.zeros(16 * 16)
    st = lib.ie_matvec_noalloc(2, 16, 0.0, iedd.IE_GRID_TEXT, ctypes.c_void_p(xh.ctypes.data),
                               ctypes.c_void_p(yh.ctypes.data), None)
    assert st == iedd.IE_ERR_ARG


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2, reason="needs two GPUs")
def test_noalloc_rejects_another_devices_memory(lib):
    # x and y on cuda:1 while cuda:0 is current: rejected before any launch
    x = torch.zeros(16 * 16, dtype=torch.float64, device="cuda:1")
    y = torch.zeros_like(x)
    with torch.cuda.device(0):
        st = lib.ie_matvec_noalloc(2, 16, 0.0, iedd.IE_GRID_TEXT, ctypes.c_void_p(x.data_ptr()),
                                   ctypes.c_void_p(y.data_ptr()), None)
    assert st == iedd.IE_ERR_ARG
    assert b"current device" in lib.ie_last_error()
