"""The Python binding refuses mis-sized buffers before any call into the
library: the C entry points take raw device pointers and cannot check their
sizes, so a short x or a small `out` would be read or written out of bounds
on the GPU.  Runs on the CPU: the checks come before any device access."""
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1304_4235_gb300 import urchin as U  # noqa: E402

DIRS = np.tile([[0.0, 0.0, 1.0]], (12, 1))


def _bvh(n=100):
    # a stand-in with no handle: reaching the library would raise AttributeError
    return types.SimpleNamespace(n=n)


@pytest.mark.parametrize("fn", [U.urchin_trace_columns, U.urchin_trace_columns_noalloc])
def test_wrong_out_shape_is_refused(fn):
    x = torch.ones(100, dtype=torch.float64)
    with pytest.raises(ValueError, match="out has shape"):
        fn(_bvh(), x, DIRS, 1.0, out=torch.empty((99, 12), dtype=torch.float32))
    with pytest.raises(ValueError, match="out has shape"):
        fn(_bvh(), x, DIRS, 1.0, origins=torch.zeros(7, dtype=torch.int32),
           out=torch.empty((100, 12), dtype=torch.float32))


@pytest.mark.parametrize("fn", [U.urchin_trace_columns, U.urchin_trace_columns_noalloc,
                                U.urchin_trace_columns_nearfar])
def test_wrong_x_size_is_refused(fn):
    with pytest.raises(ValueError, match="the BVH has 100 particles"):
        fn(_bvh(), torch.ones(99, dtype=torch.float64), DIRS, 1.0)


def test_wrong_out_dtype_and_origins_dtype_are_refused():
    x = torch.ones(100, dtype=torch.float64)
    with pytest.raises(TypeError, match="expected torch.float64"):
        U.urchin_trace_columns(_bvh(), x, DIRS, 1.0, precision=U.F64, out=torch.empty((100, 12)))
    with pytest.raises(TypeError, match="origins must be int32"):
        U.urchin_trace_columns(_bvh(), x, DIRS, 1.0, origins=torch.zeros(3, dtype=torch.int64))


def test_non_contiguous_out_is_refused():
    x = torch.ones(100, dtype=torch.float64)
    out = torch.empty((12, 100), dtype=torch.float32).t()
    with pytest.raises(ValueError, match="contiguous"):
        U.urchin_trace_columns(_bvh(), x, DIRS, 1.0, out=out)


def test_vjp_wrong_xbar_size_is_refused():
    with pytest.raises(ValueError, match="x_bar has 5 values"):
        U.urchin_trace_columns_vjp(_bvh(), DIRS, 1.0, torch.zeros((100, 12), dtype=torch.float32),
                                   x_bar=torch.zeros(5, dtype=torch.float64))
