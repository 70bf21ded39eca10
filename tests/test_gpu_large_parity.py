"""Parity near full size: the upper levels and the multi-block paths taken
by the workloads themselves rather than forced.

* 2D 255^2 (L = 5) with the bench field's recipe (contrast 1e6, b = 1e-3,
  eps 1e-6) in plain FP64: fronts, skeletons in pivot order, ranks and |s_L|
  identical to the oracle's; F^-1 x and F x within 1e-10 relative, in the
  2-norm and element-wise (largest error over the largest entry).  For
  F^-1 x the bound is raised to 10 u kappa(A) where that is larger: two
  backward-stable FP64 evaluations of it differ by up to about u kappa in
  the forward sense (kappa(A) ~ 1e10 on this field).
* 3D 47^3 (L = 3) Laplacian at eps 1e-3, whose level-1 and level-2 faces
  hold 128+ DOFs and go through the multi-block ID and elimination at the
  default thresholds: the same checks.
The oracle takes seconds (2D) to about a minute (3D) here.
"""
import numpy as np
import pytest

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _kappa(A):
    """2-norm condition number of A (extreme eigenvalues by scipy's eigsh)."""
    import scipy.sparse.linalg as spla
    lmax = spla.eigsh(A, k=1, which="LA", return_eigenvectors=False)[0]
    lmin = spla.eigsh(A.tocsc(), k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
    return lmax / lmin


def _fields(dim, n, field):
    if field == "lap":
        return inputs.constant_coefficients(dim, n)
    a, _ = inputs.high_contrast_coefficients(dim, n, seed=2, low=1e-3, high=1e3)
    return a, np.full((n - 1) ** dim, 1e-3)


@pytest.mark.parametrize("dim,n,field,eps", [(2, 256, "contrast6", 1e-6), (3, 48, "lap", 1e-3)])
def test_large_grid_matches_oracle(hiflib, dim, n, field, eps):
    from paper_1307_2895_gb300 import hif
    a, b = _fields(dim, n, field)
    A = stencil.assemble(dim, n, a, b)
    F = hifde.factor(A, dim, n, eps)
    x = inputs.rhs(dim, n, 2, seed=5)
    G = hif.factor(dim, n, a, b, eps, precision="fp64")
    try:
        fronts, root = G.structure()
        st = G.stats()
        yi = G.apply(x, inverse=True)
        yf = G.apply(x, inverse=False)
    finally:
        G.free()
    ostruct, oroot = F.skeleton_structure()
    assert root == oroot
    assert st["near_threshold_fronts"] == 0
    got = {(lev, tuple(c)): sk for lev, c, sk in fronts}
    nfront, nbig = 0, 0
    for lev, dd in enumerate(ostruct):
        for key, (c, sk, k) in dd.items():
            nfront += 1
            nbig += len(c) >= 128
            assert got.get((lev, tuple(c))) == sk, f"level {lev} front {c[:4]}...: skeletons differ"
    assert len(fronts) == nfront
    if dim == 3:
        assert nbig > 0
    oi, of = F.apply_inverse(x), F.apply(x)
    tol_i = max(1e-10, 10 * 2.2e-16 * _kappa(A))
    for y, o, tol in ((yi, oi, tol_i), (yf, of, 1e-10)):
        print(f"{dim}D n={n}: 2-norm {np.linalg.norm(y - o) / np.linalg.norm(o):.2e}, "
              f"element-wise {np.abs(y - o).max() / np.abs(o).max():.2e}, bound {tol:.1e}")
        assert np.linalg.norm(y - o) <= tol * np.linalg.norm(o)
        assert np.abs(y - o).max() <= tol * np.abs(o).max()
