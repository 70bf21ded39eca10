"""Nonzero Dirichlet data through the C ABI (hif_rhs_from_bc, host code of
the library) against the oracle's oracle.stencil.rhs_from_bc, on the CPU.

Both add, at every interior node next to the boundary, (1/h^2) a g for
each boundary neighbour, axis by axis and the lower neighbour first, so the
two agree to the last bit up to a fused multiply-add (tolerance: 2 ulp of
the sum of magnitudes).  Covered: 2D and 3D, a high-contrast field, several
columns with a row stride larger than their count, the smallest grid (n = 4,
where every interior node touches the boundary), zero data and argument
errors.
"""
import ctypes

import numpy as np
import pytest

from oracle import stencil
from paper_1307_2895_gb300 import hif, inputs


def _case(dim, n, nrhs, seed):
    a, _ = inputs.high_contrast_coefficients(dim, n, seed=seed, low=1e-2, high=1e2)
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(((n + 1) ** dim, nrhs))
    f = rng.standard_normal(((n - 1) ** dim, nrhs))
    return a, g, f


def _bound(dim, n, a, g, f):
    """2 ulp of |f| + (1/h^2) sum |a g| per entry."""
    mag = stencil.rhs_from_bc(dim, n, np.abs(a), np.abs(g), np.abs(f))
    return 2 * np.finfo(np.float64).eps * mag


@pytest.mark.parametrize("dim,n,nrhs", [(2, 4, 1), (2, 37, 3), (2, 64, 1), (3, 4, 2), (3, 13, 2), (3, 24, 1)])
def test_rhs_from_bc_matches_oracle(dim, n, nrhs):
    hif.load(build_if_missing=True)
    a, g, f = _case(dim, n, nrhs, seed=dim * 100 + n)
    got = hif.rhs_from_bc(dim, n, a, g, f)
    want = stencil.rhs_from_bc(dim, n, a, g, f)
    assert got.shape == f.shape
    assert (np.abs(got - want) <= _bound(dim, n, a, g, f)).all()
    # nodes away from the boundary keep f exactly
    X = stencil.coords(dim, n)
    inner = ((X > 1) & (X < n - 1)).all(axis=1)
    assert np.array_equal(got[inner], f[inner])


def test_row_stride_and_zero_data():
    lib = hif.load(build_if_missing=True)
    dim, n, nrhs, ld = 3, 9, 2, 5
    a, g, f = _case(dim, n, nrhs, seed=5)
    G = np.zeros(((n + 1) ** dim, ld))
    G[:, :nrhs] = g
    G[:, nrhs:] = np.nan                      # never read
    R = np.full(((n - 1) ** dim, ld), 7.0)
    R[:, :nrhs] = f
    grid = hif._Grid(dim, n, 8, 1)
    rc = lib.hif_rhs_from_bc(ctypes.byref(grid), a.ctypes.data, G.ctypes.data, R.ctypes.data, nrhs, ld)
    assert rc == hif.HIF_OK
    want = stencil.rhs_from_bc(dim, n, a, g, f)
    assert (np.abs(R[:, :nrhs] - want) <= _bound(dim, n, a, g, f)).all()
    assert (R[:, nrhs:] == 7.0).all()
    assert np.array_equal(hif.rhs_from_bc(dim, n, a, np.zeros_like(g), f), f)


def test_rhs_from_bc_argument_errors():
    lib = hif.load(build_if_missing=True)
    a, g, f = _case(2, 8, 1, seed=1)
    ok = hif._Grid(2, 8, 8, 1)
    call = lambda grid, nrhs=1, ld=1, gp=g.ctypes.data: lib.hif_rhs_from_bc(
        ctypes.byref(grid), a.ctypes.data, gp, f.ctypes.data, nrhs, ld)
    assert call(hif._Grid(4, 8, 8, 1)) == hif.HIF_ERR_ARG
    assert call(hif._Grid(2, 3, 8, 1)) == hif.HIF_ERR_ARG
    assert call(ok, nrhs=0) == hif.HIF_ERR_ARG
    assert call(ok, nrhs=2, ld=1) == hif.HIF_ERR_ARG
    assert call(ok, gp=None) == hif.HIF_ERR_ARG
    with pytest.raises(ValueError):
        hif.rhs_from_bc(2, 8, a[:-1], g, f)
