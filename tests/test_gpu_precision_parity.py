"""The timed configuration (FP64 factorization, factor stored and applied in
FP32: precision "fp32_apply") against the FP64 oracle.

The factorization itself runs in FP64, so its skeletons, ranks and |s_L| are
the oracle's bit for bit (checked).  Rounding the stored blocks to FP32 and
applying them in FP32 perturbs each of the d = 2(2L + 1) + 1 factors of
F^-1 = V_0 V_1/2 ... D^-1 ... V_1/2^T V_0^T (Eq. 4.2) by a relative
O(u) with u = 2^-24, so F^-1 x moves by at most about d u kappa(F) relative,
kappa(F) ~ kappa(A) for eps kappa << 1 (Section 4.3):

    ||y_fp32 - y_oracle||_2 <= d u kappa(A) ||y_oracle||_2.

The element-wise largest relative error, max_i |y_fp32 - y_oracle|_i / max_i
|y_oracle|_i, is held to the same bound.  Cases: 2D Laplacian and contrast
1e4 at 63^2, contrast 1e6 with b = 1e-3 at 127^2 (the bench field's recipe),
3D Laplacian at 15^3 and contrast 1e4 at 19^3.
"""
import numpy as np
import pytest

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _fields(dim, n, field):
    if field == "lap":
        return inputs.constant_coefficients(dim, n)
    if field == "contrast6":
        a, _ = inputs.high_contrast_coefficients(dim, n, seed=2, low=1e-3, high=1e3)
        return a, np.full((n - 1) ** dim, 1e-3)
    return inputs.high_contrast_coefficients(dim, n, seed=11, low=1e-2, high=1e2)


def _kappa(A):
    import scipy.sparse.linalg as spla
    lmax = spla.eigsh(A, k=1, which="LA", return_eigenvectors=False)[0]
    lmin = spla.eigsh(A.tocsc(), k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
    return lmax / lmin


@pytest.mark.parametrize("dim,n,field,eps", [
    (2, 64, "lap", 1e-6),
    (2, 64, "contrast", 1e-6),
    (2, 128, "contrast6", 1e-6),
    (3, 16, "lap", 1e-6),
    (3, 20, "contrast", 1e-4),
])
def test_fp32_apply_matches_oracle(hiflib, dim, n, field, eps):
    from paper_1307_2895_gb300 import hif
    a, b = _fields(dim, n, field)
    A = stencil.assemble(dim, n, a, b)
    F = hifde.factor(A, dim, n, eps)
    x = inputs.rhs(dim, n, 4, seed=5)
    G = hif.factor(dim, n, a, b, eps, precision="fp32_apply")
    try:
        fronts, root = G.structure()
        y = G.apply(x, inverse=True)
    finally:
        G.free()
    ostruct, oroot = F.skeleton_structure()
    assert root == oroot
    got = {(lev, tuple(c)): sk for lev, c, sk in fronts}
    for lev, dd in enumerate(ostruct):
        for key, (c, sk, k) in dd.items():
            assert got.get((lev, tuple(c))) == sk
    yo = F.apply_inverse(x)
    d = 2 * (2 * F.L + 1) + 1
    bound = d * U32 * _kappa(A)
    fwd = np.linalg.norm(y - yo) / np.linalg.norm(yo)
    elem = np.abs(y - yo).max() / np.abs(yo).max()
    print(f"{dim}D n={n} {field}: 2-norm {fwd:.2e}, element-wise {elem:.2e}, bound d u kappa = {bound:.2e}")
    assert fwd <= bound, (fwd, bound)
    assert elem <= bound, (elem, bound)
    # the FP32 rounding is visible (the stored factor is not FP64) but small
    assert fwd > 0.0
