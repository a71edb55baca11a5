"""Host-side argument checks of the Python binding (no GPU, no library call).

tucker_gram_noalloc writes I_n x I_n FP64 values through the caller's S and
reads prod(dims) elements of y; the binding must reject a mismatched S or y
before anything is launched.
"""
import pytest

torch = pytest.importorskip("torch")

from paper_1901_06043_gb300 import tucker


def _ok(dims=(6, 5, 4), mode=1):
    y = torch.zeros(6 * 5 * 4, dtype=torch.float32)
    I = dims[mode]
    return y, dims, mode, torch.zeros((I, I), dtype=torch.float64)


def test_gram_out_accepts_a_matching_output():
    tucker._check_gram_out(*_ok())


@pytest.mark.parametrize("bad", ["fp32", "shape", "numel", "mode", "transposed_rect"])
def test_gram_out_rejects_mismatches(bad):
    y, dims, mode, S = _ok()
    if bad == "fp32":
        S = S.float()
    elif bad == "shape":
        S = torch.zeros((6, 6), dtype=torch.float64)
    elif bad == "numel":
        y = y[:-1]
    elif bad == "mode":
        mode = 3
    elif bad == "transposed_rect":
        S = torch.zeros((5, 4), dtype=torch.float64)
    with pytest.raises(ValueError):
        tucker._check_gram_out(y, dims, mode, S)


def test_gram_noalloc_rejects_a_wrong_output_before_any_call():
    # a wrongly shaped S is refused by the binding's checks, which run before
    # the device checks and before the library is touched
    y, dims, mode, _ = _ok()
    with pytest.raises(ValueError, match="shape"):
        tucker.gram_noalloc(y, dims, mode, torch.zeros((2, 2), dtype=torch.float64))


def test_host_buffer_of_numpy_and_cpu_tensors():
    import numpy as np
    a = np.zeros(12, dtype=np.float32)
    ptr, code, n = tucker._host_buffer(a)
    assert (ptr, code, n) == (a.ctypes.data, tucker.F32, 12)
    t = torch.zeros(7, dtype=torch.float64)
    ptr, code, n = tucker._host_buffer(t)
    assert (ptr, code, n) == (t.data_ptr(), tucker.F64, 7)


@pytest.mark.parametrize("bad", ["strided_numpy", "int_numpy", "strided_tensor", "int_tensor"])
def test_host_buffer_rejects_what_the_library_cannot_read(bad):
    import numpy as np
    x = {"strided_numpy": np.zeros((4, 4), dtype=np.float32)[:, ::2],
         "int_numpy": np.zeros(4, dtype=np.int32),
         "strided_tensor": torch.zeros((4, 4))[:, ::2],
         "int_tensor": torch.zeros(4, dtype=torch.int32)}[bad]
    with pytest.raises((ValueError, TypeError)):
        tucker._host_buffer(x)
