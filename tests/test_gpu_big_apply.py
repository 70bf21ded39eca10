"""F^-1 with the large blocks of a level applied by many thread blocks each
(hif_opts.big_apply) against the one-block kernels and the oracle.

The many-block kernels compute the same products in another order, so in
FP64 the two F^-1 x agree to rounding (1e-12 relative, element-wise
against the largest entry) and both match the oracle's to 1e-10.  The cases
force the path onto most blocks with a small threshold (2D and 3D, hifde3
and hifde3x, cells and fronts, 12 right-hand sides: a chunk of 8 and one of
4) and use the default threshold at 63^3, where the upper levels' cells
and faces are the blocks it is meant for.
"""
import numpy as np
import pytest

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs

pytestmark = pytest.mark.gpu


def _apply(dim, n, a, b, eps, variant, big_apply, x, precision="fp64"):
    from paper_1307_2895_gb300 import hif
    G = hif.factor(dim, n, a, b, eps, precision=precision, variant=variant, big_apply=big_apply)
    try:
        return G.apply(x, inverse=True)
    finally:
        G.free()


@pytest.mark.parametrize("dim,n,variant,big_apply", [(2, 128, "hifde", 512), (3, 24, "hifde", 2048),
                                                     (3, 32, "hifde3x", 4096)])
def test_big_apply_matches_oracle(hiflib, dim, n, variant, big_apply):
    a, b = inputs.high_contrast_coefficients(dim, n, seed=3, low=1e-2, high=1e2)
    eps = 1e-6
    A = stencil.assemble(dim, n, a, b)
    F = hifde.factor3x(A, n, eps) if variant == "hifde3x" else hifde.factor(A, dim, n, eps)
    x = inputs.rhs(dim, n, 12, seed=8)
    y_big = _apply(dim, n, a, b, eps, variant, big_apply, x)
    y_one = _apply(dim, n, a, b, eps, variant, -1, x)
    o = F.apply_inverse(x)
    e_pair = np.abs(y_big - y_one).max() / np.abs(y_one).max()
    e_orc = np.abs(y_big - o).max() / np.abs(o).max()
    print(f"{variant} {dim}D n={n}: many-block vs one-block {e_pair:.2e}, vs oracle {e_orc:.2e}")
    assert e_pair <= 1e-12
    assert e_orc <= 1e-10


def test_big_apply_default_threshold_laplace3d_63(hiflib):
    a, b = inputs.constant_coefficients(3, 64)
    x = inputs.rhs(3, 64, 4, seed=2)
    for precision, tol in (("fp64", 1e-12), ("fp32_apply", 1e-4)):
        y_big = _apply(3, 64, a, b, 1e-6, "hifde", 0, x, precision)
        y_one = _apply(3, 64, a, b, 1e-6, "hifde", -1, x, precision)
        err = np.abs(y_big - y_one).max() / np.abs(y_one).max()
        print(f"63^3 {precision}: many-block vs one-block {err:.2e}")
        assert err <= tol
