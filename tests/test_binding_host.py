"""Host logic of the Python binding (no GPU): how arrays map onto the C ABI's vector layout.

The C ABI takes an N x nrhs batch column-major with a leading dimension ld >= N (entry (i, k) at
x[k * ld + i]).  The binding accepts (N,) vectors and (nrhs, N) batches whose rows are unit-stride;
row k of the batch is column k of the ABI's layout and the row stride is ld.
"""
import numpy as np
import pytest
import torch

from paper_2108_12574_gb300 import iedd


def test_vector_maps_to_one_column():
    x = np.zeros(37)
    ptr, nrhs, ld, keep = iedd._vec(x, 37)
    assert (ptr.value, nrhs, ld) == (x.ctypes.data, 1, 37)
    assert keep is x


def test_batch_rows_are_columns_with_leading_dimension():
    big = np.zeros((5, 48))
    x = big[1:4, :40]  # 3 right-hand sides of length 40 inside rows of 48
    ptr, nrhs, ld, _ = iedd._vec(x, 40)
    assert (nrhs, ld) == (3, 48)
    assert ptr.value == big.ctypes.data + 1 * 48 * 8
    # entry (i, k) of the ABI's layout is row k, element i
    big[2, 7] = 1.5
    flat = np.ctypeslib.as_array((np.ctypeslib.ctypes.c_double * (nrhs * ld)).from_address(ptr.value))
    assert flat[1 * ld + 7] == 1.5


def test_torch_batch_stride_is_leading_dimension():
    t = torch.zeros((4, 64), dtype=torch.float64)
    ptr, nrhs, ld, _ = iedd._vec(t[:, :50], 50)
    assert (nrhs, ld) == (4, 64)
    assert ptr.value == t.data_ptr()


@pytest.mark.parametrize("bad", [
    np.zeros(36),                       # wrong length
    np.zeros(74)[::2],                  # not unit stride
    np.zeros((3, 37)).T.copy(),         # (N, nrhs) instead of (nrhs, N)
    np.zeros((2, 74))[:, ::2],          # rows not unit stride
])
def test_bad_shapes_and_strides_are_rejected(bad):
    with pytest.raises(ValueError):
        iedd._vec(bad, 37)


def test_wrong_dtype_and_read_only_output_are_rejected():
    with pytest.raises(TypeError):
        iedd._vec(np.zeros(8, dtype=np.float32), 8)
    with pytest.raises(TypeError):
        iedd._vec(torch.zeros(8, dtype=torch.float32), 8)
    with pytest.raises(TypeError):
        iedd._vec([0.0] * 8, 8)
    ro = np.zeros(8)
    ro.flags.writeable = False
    iedd._vec(ro, 8)  # fine as an input
    with pytest.raises(ValueError):
        iedd._vec(ro, 8, writable=True)


def test_stream_argument_forms():
    assert iedd._stream(0).value in (None, 0)
    assert iedd._stream(1234).value == 1234

    class FakeStream:
        cuda_stream = 4321
    assert iedd._stream(FakeStream()).value == 4321
    if not torch.cuda.is_available():
        assert iedd._stream(None).value in (None, 0)
