"""The library's host-side Newell tensor (Eq. 2's kernel, computed once per
mesh when a context is created) against the oracle's binary128 tensor,
entry by entry: within 1e-13 of max|N| on meshes up to 64 x 64 x 4, cubic
and non-cubic cells.  No GPU is involved: the tensor is host code."""
import ctypes

import numpy as np
import pytest

import oracle as O


class _Args(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("Ms", ctypes.c_double)]


@pytest.fixture(scope="module")
def lib():
    from paper_2107_06729_gb300 import build
    L = ctypes.CDLL(build.build())
    L.mmx_host_tensor.argtypes = [ctypes.POINTER(_Args), ctypes.POINTER(ctypes.c_double)]
    L.mmx_host_tensor.restype = ctypes.c_int
    return L


@pytest.mark.parametrize("n,d", [
    ((4, 3, 2), (1e-9, 2e-9, 3e-9)),
    ((16, 16, 4), (4e-9, 4e-9, 4e-9)),
    ((32, 8, 1), (2.5e-9, 2.5e-9, 1e-9)),
    ((64, 64, 4), (2e-9, 2e-9, 2e-9)),
])
def test_library_tensor_matches_oracle(lib, n, d):
    nx, ny, nz = n
    a = _Args(nx, ny, nz, *d, 8e5)
    got = np.zeros((6, nz, ny, nx))
    assert lib.mmx_host_tensor(ctypes.byref(a), got.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == 0
    want = O.newell_octant(nx, ny, nz, *d)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-13 * scale, np.abs(got - want).max() / scale
