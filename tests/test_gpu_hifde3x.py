"""hifde3x on the GPU (Section 4.5, Algorithm 4.2) against the oracle's
factor3x, plain FP64.

Levels 0 and 1 (cells and faces) are hifde3's; from level 1's edges on the
CUDA path takes its cells, faces, edges and their neighbour sets from the
host symbolic stage, which follows the factorization's own skeletons, and
holds A_l as one dense matrix of the active DOFs.  Required: every face and
edge group (keyed by its fractional level and DOF set), its skeletons in
pivot order and its rank, and |s_L| identical to the oracle's; no pivot ratio
near eps; F^-1 x and F x within 1e-10 relative (F^-1: raised to 10 u kappa(A)
where larger), in the 2-norm and element-wise.

Cases: 15^3 (one level: hifde3 itself, no edges), 23^3 and 31^3 (two levels:
level 1's edges, the first assembled step; 31^3 also with every group of 128+
DOFs through the multi-block ID), 31^3 high contrast, the indefinite
Helmholtz operator at 23^3 and 31^3 (LDL^T blocks), and 47^3 (three
levels: the algebraic cells of level 2, its faces and edges, with cells of
192+ interior DOFs through the tiled elimination).
"""
import numpy as np
import pytest

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs

pytestmark = pytest.mark.gpu


def _fields(n, field):
    if field == "lap":
        return inputs.constant_coefficients(3, n)
    if field == "helm":   # Example 6 at 8 DOFs per wavelength, a = 1 +- 10% (no symmetric pivot ties)
        return inputs.helmholtz_coefficients(3, n, 8, perturb=0.1, seed=7)
    return inputs.high_contrast_coefficients(3, n, seed=5, low=1e-2, high=1e2)


def _kappa(A):
    import scipy.sparse.linalg as spla
    lmax = spla.eigsh(A, k=1, which="LM", return_eigenvectors=False)[0]
    lmin = spla.eigsh(A.tocsc(), k=1, sigma=0, which="LM", return_eigenvectors=False)[0]
    return abs(lmax) / abs(lmin)


CASES = [
    (16, "lap", 1e-3, 0),
    (24, "lap", 1e-3, 0),
    (32, "lap", 1e-3, 0),
    (32, "lap", 1e-6, 128),
    (32, "contrast", 1e-6, 0),
    (24, "helm", 1e-6, 0),
    (32, "helm", 1e-6, 0),
    pytest.param(48, "lap", 1e-3, 0, marks=pytest.mark.slow),
]


@pytest.mark.parametrize("n,field,eps,big_cell", CASES)
def test_hifde3x_matches_oracle(hiflib, n, field, eps, big_cell):
    from paper_1307_2895_gb300 import hif
    a, b = _fields(n, field)
    A = stencil.assemble(3, n, a, b)
    F = hifde.factor3x(A, n, eps)
    x = inputs.rhs(3, n, 2, seed=5)
    G = hif.factor(3, n, a, b, eps, variant="hifde3x", precision="fp64", big_cell=big_cell)
    try:
        fronts, root = G.structure()
        st = G.stats()
        yi = G.apply(x, inverse=True)
        yf = G.apply(x, inverse=False)
    finally:
        G.free()
    ostruct, oroot = F.skeleton_structure()
    got = {(lev, tuple(c)): sk for lev, c, sk in fronts}
    assert len(got) == len(fronts)
    nexp = 0
    for lev, dd in enumerate(ostruct):
        for key, (c, sk, k) in dd.items():
            nexp += 1
            assert got.get((lev, tuple(c))) == sk, f"fractional level {lev} group {c[:4]}...: skeletons differ"
    assert len(fronts) == nexp
    assert root == oroot
    assert st["root_size"] == oroot
    assert st["near_threshold_fronts"] == 0
    if n >= 24:
        assert any(len(d) for d in ostruct[3::2])          # edges were skeletonized
    tol_i = max(1e-10, 10 * 2.2e-16 * _kappa(A))
    for y, o, tol in ((yi, F.apply_inverse(x), tol_i), (yf, F.apply(x), 1e-10)):
        print(f"n={n} {field} eps={eps:g}: 2-norm {np.linalg.norm(y - o) / np.linalg.norm(o):.2e}, "
              f"element-wise {np.abs(y - o).max() / np.abs(o).max():.2e}, |s_L| {root}")
        assert np.linalg.norm(y - o) <= tol * np.linalg.norm(o)
        assert np.abs(y - o).max() <= tol * np.abs(o).max()


@pytest.mark.parametrize("n,edge_start", [(16, 0), (32, 0), (32, 2), pytest.param(48, 2, marks=pytest.mark.slow)])
def test_hifde3x_edge_start_matches_oracle(hiflib, n, edge_start):
    """The rule of thumb's option (Section 4.5): edges from level 0 (the
    assembled stage starts after level 0's faces) or from level 2 (31^3: none
    at all, the result is hifde3's; 47^3: levels 0-2 are hifde3's)."""
    from paper_1307_2895_gb300 import hif
    eps = 1e-3
    a, b = _fields(n, "lap")
    A = stencil.assemble(3, n, a, b)
    F = hifde.factor3x(A, n, eps, edge_start=edge_start)
    x = inputs.rhs(3, n, 2, seed=5)
    G = hif.factor(3, n, a, b, eps, variant="hifde3x", precision="fp64", edge_start=edge_start)
    try:
        fronts, root = G.structure()
        yi = G.apply(x, inverse=True)
    finally:
        G.free()
    ostruct, oroot = F.skeleton_structure()
    got = {(lev, tuple(c)): sk for lev, c, sk in fronts}
    nexp = 0
    for lev, dd in enumerate(ostruct):
        for key, (c, sk, k) in dd.items():
            nexp += 1
            assert got.get((lev, tuple(c))) == sk, f"fractional level {lev} group {c[:4]}...: skeletons differ"
    assert len(fronts) == nexp and root == oroot
    oi = F.apply_inverse(x)
    assert np.linalg.norm(yi - oi) <= 1e-10 * np.linalg.norm(oi)


def test_hifde3x_pcg_reaches_1e12(hiflib):
    """FP32-stored factor of hifde3x as the preconditioner: PCG to 1e-12,
    re-checked on the host in extended precision."""
    from paper_1307_2895_gb300 import hif
    n, eps = 32, 1e-6
    a, b = _fields(n, "contrast")
    f = inputs.rhs(3, n, 2)
    G = hif.factor(3, n, a, b, eps, variant="hifde3x", precision="fp32_apply")
    try:
        xh, xl, info = G.solve(f, tol=1e-12, maxit=200, want_lo=True)
    finally:
        G.free()
    assert info["converged"] and info["relres_max"] <= 1e-12
    assert stencil.residual_ext(3, n, a, b, f, xh, xl).max() <= 2e-12


def test_hifde3x_argument_errors(hiflib):
    from paper_1307_2895_gb300 import hif
    a, b = inputs.constant_coefficients(2, 32)
    with pytest.raises(hif.HifError) as e:
        hif.factor(2, 32, a, b, 1e-6, variant="hifde3x")
    assert e.value.code == hif.HIF_ERR_ARG
    a, b = inputs.constant_coefficients(3, 30)
    with pytest.raises(hif.HifError) as e:
        hif.factor(3, 30, a, b, 1e-6, variant="hifde3x")     # 30 is not divisible by 2^L = 4
    assert e.value.code == hif.HIF_ERR_ARG
