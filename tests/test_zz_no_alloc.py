"""ie_matvec_noalloc: the allocation-free matvec entry point, through the C ABI (needs a GPU).

Some callers cannot allocate device memory (code running inside an allocator, a memory-capped
host framework, or a process that reserved all its memory up front).  ie_matvec_noalloc gives
them y = A x with the FP32 SFU kernel, using only a static device array as scratch.  This test
checks it against the allocating entry point ie_matvec(IE_MIXED), within the FP32 matvec
tolerance of the other parity tests (4e-6 ||A||_inf ||x||_inf), on two calls in a row with
different inputs (the shared scratch keeps the previous call's contents), and checks that an
oversized problem is rejected.  The file is named so that pytest collects it last.
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


def _scale(dim, n, x):
    rows = O.matvec_direct(dim, n, np.ones(n ** dim), rows=np.array([0, (n ** dim) // 2]))
    return 2.0 * float(np.max(np.abs(rows))) * float(np.max(np.abs(x)))


@pytest.mark.parametrize("dim,n", [(2, 64), (2, 512), (3, 24), (2, 37)])
def test_noalloc_matches_ie_matvec_two_calls_in_a_row(lib, dim, n):
    N = n ** dim
    prob = iedd.ie_discretize(dim, n)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (11, 12):  # two calls in a row, different inputs
        xh = I.uniform_rhs(N, seed)
        x = torch.from_numpy(xh).cuda()
        y_ref = torch.zeros_like(x)
        iedd.ie_matvec(prob, x, y_ref, iedd.IE_MIXED)
        y = torch.full_like(x, float("nan"))
        st = lib.ie_matvec_noalloc(dim, n, 0.0, iedd.IE_GRID_TEXT, ctypes.c_void_p(x.data_ptr()),
                                   ctypes.c_void_p(y.data_ptr()), stream)
        assert st == iedd.IE_OK, lib.ie_last_error()
        torch.cuda.synchronize()
        err = float((y - y_ref).abs().max())
        assert err <= 4e-6 * _scale(dim, n, xh), (seed, err)


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
