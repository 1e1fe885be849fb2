"""Argument marshalling of the Python binding (no library call, no GPU): blocks are checked for
shape, dtype and contiguity before any pointer reaches the C ABI."""
import numpy as np
import pytest
import torch

from paper_2503_22652_gb300 import _check_arr


def test_numpy_blocks_converted_and_checked():
    a = np.arange(12, dtype=np.float32).reshape(3, 4)
    b = _check_arr(a, (3, 4), "X")
    assert b.dtype == np.float64 and b.flags.c_contiguous and np.array_equal(b, a)
    f = np.asfortranarray(np.ones((3, 4)))
    assert _check_arr(f, (3, 4), "X").flags.c_contiguous
    with pytest.raises(ValueError):
        _check_arr(np.ones((3, 5)), (3, 4), "X")
    c = _check_arr(np.ones((2, 2)), (2, 2), "X", np.complex128)
    assert c.dtype == np.complex128
    assert _check_arr(None, (3, 4), "X") is None


def test_torch_blocks_checked_not_copied():
    t = torch.ones(3, 4, dtype=torch.float64)
    assert _check_arr(t, (3, 4), "X") is t
    with pytest.raises(ValueError):
        _check_arr(t.t(), (4, 3), "X")                      # not contiguous
    with pytest.raises(ValueError):
        _check_arr(t.float(), (3, 4), "X")                  # wrong element type
    with pytest.raises(ValueError):
        _check_arr(t, (3, 5), "X")                          # wrong size
    with pytest.raises(ValueError):
        _check_arr(t, (3, 4), "X", np.complex128)           # real tensor for a complex block
    z = torch.ones(3, 4, dtype=torch.complex128)
    assert _check_arr(z, (3, 4), "X", np.complex128) is z


def test_inplace_solve_refuses_arrays_it_would_copy():
    """solve(inplace=True) writes the Ritz vectors into the caller's array, so an array the binding
    would have to convert or copy (wrong dtype, not C-contiguous, read-only) is refused before any
    library call."""
    from paper_2503_22652_gb300 import Solver
    s = object.__new__(Solver)  # no handle: the check comes before the library is touched
    s.dt, s.m, s.N = np.float64, 3, 4
    ro = np.ones((3, 4))
    ro.flags.writeable = False
    for bad in (np.ones((3, 4), dtype=np.float32), np.asfortranarray(np.ones((3, 4))), ro):
        with pytest.raises(ValueError):
            s.solve(bad, inplace=True)
