"""Edge cases of the CUDA path against the FP64 oracle.

* The smallest trees: n = 4 (cells and fronts of one DOF) and n = 5 (a
  ragged grid) in 2D and 3D: front sets, skeletons and |s_L| equal to the
  oracle's, F^-1 x within 1e-10.
* Right-hand sides through the C ABI with a row stride above their count:
  one and 32 columns (the largest the vector kernels take in one chunk is
  16, so 32 is two chunks), hif_apply against the oracle's F^-1 and
  hif_solve to 1e-12 checked in extended precision; the padding columns are
  neither read nor written.
"""
import ctypes

import numpy as np
import pytest

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs

pytestmark = pytest.mark.gpu


def _contrast(dim, n):
    return inputs.high_contrast_coefficients(dim, n, seed=11, low=1e-2, high=1e2)


@pytest.mark.parametrize("dim,n", [(2, 4), (2, 5), (3, 4), (3, 5)])
def test_smallest_grids_match_oracle(hiflib, dim, n):
    from paper_1307_2895_gb300 import hif
    eps = 1e-6
    a, b = _contrast(dim, n)
    A = stencil.assemble(dim, n, a, b)
    F = hifde.factor(A, dim, n, eps)
    x = inputs.rhs(dim, n, 2, seed=5)
    G = hif.factor(dim, n, a, b, eps, precision="fp64")
    try:
        fronts, root = G.structure()
        y = G.apply(x, inverse=True)
    finally:
        G.free()
    ostruct, oroot = F.skeleton_structure()
    assert root == oroot
    got = {}
    for lev, c, sk in fronts:
        got.setdefault(lev, {})[tuple(c)] = sk
    for lev, d in enumerate(ostruct):
        assert len(got.get(lev, {})) == len(d)
        for c, sk, _ in d.values():
            assert got[lev][tuple(c)] == sk
    yo = F.apply_inverse(x)
    assert np.linalg.norm(y - yo) <= 1e-10 * np.linalg.norm(yo)


@pytest.mark.parametrize("nrhs", [1, 32])
def test_strided_right_hand_sides_through_the_abi(hiflib, nrhs):
    from paper_1307_2895_gb300 import hif
    dim, n, eps = 2, 32, 1e-6
    ld = nrhs + 3
    a, b = _contrast(dim, n)
    A = stencil.assemble(dim, n, a, b)
    F = hifde.factor(A, dim, n, eps)
    N = (n - 1) ** dim
    f = inputs.rhs(dim, n, nrhs, seed=7)
    X = np.full((N, ld), 7.0)
    X[:, :nrhs] = f
    Y = np.full((N, ld), -3.0)
    G = hif.factor(dim, n, a, b, eps, precision="fp64")
    lib = hif.load()
    try:
        rc = lib.hif_apply(G._live(), hif.APPLY_FINV, X.ctypes.data, Y.ctypes.data, nrhs, ld)
        assert rc == hif.HIF_OK, lib.hif_last_error()
        Xh = np.full((N, ld), 5.0)
        Xl = np.full((N, ld), 5.0)
        info = hif._SolveInfo()
        rc = lib.hif_solve(G._live(), X.ctypes.data, Xh.ctypes.data, Xl.ctypes.data, nrhs, ld, 1e-12, 100,
                           ctypes.byref(info))
        assert rc == hif.HIF_OK, lib.hif_last_error()
    finally:
        G.free()
    yo = F.apply_inverse(f)
    assert np.linalg.norm(Y[:, :nrhs] - yo) <= 1e-10 * np.linalg.norm(yo)
    assert (Y[:, nrhs:] == -3.0).all() and (X[:, nrhs:] == 7.0).all()
    assert (Xh[:, nrhs:] == 5.0).all() and (Xl[:, nrhs:] == 5.0).all()
    assert info.converged and info.relres_max <= 1e-12
    assert stencil.residual_ext(dim, n, a, b, f, Xh[:, :nrhs], Xl[:, :nrhs]).max() <= 2e-12
