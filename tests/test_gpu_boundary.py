"""Nonzero Dirichlet data end to end on the GPU: hif_rhs_from_bc, then
hif_factor + hif_solve (PCG with F^-1 to a relative residual of 1e-12).

The stencil's second differences are exact on quadratics, so for the
Laplacian (a = 1, b = 0) and a harmonic quadratic u with boundary values
g = u, the discrete solution at the interior nodes is u itself.  The solve
must return it within kappa(A) times its residual tolerance (kappa below
2e3 on these grids): 1e-8 of max |u|.
"""
import numpy as np
import pytest

from paper_1307_2895_gb300 import hif, inputs

pytestmark = pytest.mark.gpu


def _nodes(dim, n, fn):
    c = np.meshgrid(*[np.arange(n + 1)] * dim, indexing="ij")
    return fn(*[ci.transpose(*reversed(range(dim))).ravel() / n for ci in c])


@pytest.mark.parametrize("dim,n", [(2, 64), (3, 16)])
def test_harmonic_quadratic_through_solve(hiflib, dim, n):
    if dim == 2:
        u = lambda x, y: x * x - y * y + 0.3 * x * y + 0.5 * x - 0.2
    else:
        u = lambda x, y, z: x * x + y * y - 2 * z * z + 0.7 * x * z - 0.4 * y + 0.1
    a, b = inputs.constant_coefficients(dim, n)
    g = _nodes(dim, n, u)
    f = hif.rhs_from_bc(dim, n, a, g[:, None], np.zeros(((n - 1) ** dim, 1)))
    G = hif.factor(dim, n, a, b, 1e-6)
    try:
        x, info = G.solve(f, tol=1e-12, maxit=100)
    finally:
        G.free()
    c = np.meshgrid(*[np.arange(1, n)] * dim, indexing="ij")
    ui = u(*[ci.transpose(*reversed(range(dim))).ravel() / n for ci in c])
    assert info["converged"]
    assert np.abs(np.asarray(x)[:, 0] - ui).max() <= 1e-8 * np.abs(ui).max()
