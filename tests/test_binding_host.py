"""Host-side argument checks of the Python binding (no GPU): a caller-provided
output tensor is checked before the device would write into it, since the
library cannot see its size."""
import pytest

torch = pytest.importorskip("torch")
from paper_2305_14306_gb300 import hav  # noqa: E402


def test_new_output_tensors_take_the_shape_asked_for():
    like = torch.zeros(4, 3)
    t = hav._out(None, 6, torch.int32, like, "out")
    assert t.shape == (6,) and t.dtype == torch.int32
    t = hav._out(None, 12, torch.float32, like, "xyz", shape=(4, 3))
    assert t.shape == (4, 3) and t.dtype == torch.float32


def test_caller_outputs_are_checked():
    like = torch.zeros(4, 3)
    good = torch.empty(8, dtype=torch.int32)
    assert hav._out(good, 8, torch.int32, like, "out") is good
    assert hav._out(good, 5, torch.int32, like, "out") is good  # larger is fine
    for bad in (torch.empty(7, dtype=torch.int32),            # too small
                torch.empty(8, dtype=torch.int64),            # wrong type
                torch.empty(16, dtype=torch.int32)[::2],      # not contiguous
                [0] * 8):                                     # not a tensor
        with pytest.raises(ValueError):
            hav._out(bad, 8, torch.int32, like, "out")


def test_points_must_be_a_contiguous_cuda_float_array():
    for bad in (torch.zeros(4, 3), torch.zeros(4, 2), torch.zeros(4, 3, dtype=torch.float64)):
        with pytest.raises(ValueError):
            hav._points(bad)


def test_a_missing_library_fails_loudly():
    # no CPU fallback: without libhav.so the binding raises (fresh process, so
    # that no earlier load is cached)
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("from paper_2305_14306_gb300 import hav\n"
            "try:\n    hav.load('/nonexistent/libhav.so')\nexcept RuntimeError as e:\n"
            "    print('raised', e)\nelse:\n    print('loaded')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("raised"), r.stdout + r.stderr
