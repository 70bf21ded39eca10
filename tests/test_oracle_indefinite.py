"""The oracle on indefinite operators (Section 5: diagonal blocks factored by
Cholesky if A is SPD, by an LDL^T decomposition otherwise; Examples 3 and 6,
the Helmholtz equation with b = -k^2).

Pins: the signed LDL^T decomposition against the matrix it factors and
against the Cholesky decomposition on SPD input; MF (eps = 0) on 2D and 3D
Helmholtz operators with several negative eigenvalues against a dense
solve; HIF-DE's e_a = O(eps) and GMRES with F^-1 to 1e-12 in a few steps.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs


def test_ldl_signed_reconstructs_indefinite_matrices():
    """Diagonally dominant indefinite matrices (the 1 x 1 pivots in order
    then stay away from zero, as on the stencil's diagonal blocks, whose
    diagonal 2 d n^2 - k^2 dominates their 2 d off-diagonal n^2 entries)."""
    rng = np.random.default_rng(1)
    for n in (1, 5, 40):
        dsgn = np.where(rng.random(n) < 0.4, -1.0, 1.0)
        E = rng.standard_normal((n, n))
        A = np.diag(dsgn * rng.uniform(2.0, 3.0, n)) + 0.5 * (E + E.T) / max(n, 1)
        lam = np.linalg.eigvalsh(A)
        L, s = hifde.ldl_signed(A)
        assert np.allclose(np.tril(L), L)
        assert np.linalg.norm(A - (L * s) @ L.T) <= 1e-13 * np.linalg.norm(A)
        b = rng.standard_normal(n)
        x = sla.solve_triangular(L, s * sla.solve_triangular(L, b, lower=True), lower=True, trans="T")
        assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-12 * np.linalg.norm(x)
        # the number of negative signs is the inertia's (Sylvester)
        assert int((s < 0).sum()) == int((lam < 0).sum())


def test_ldl_signed_is_cholesky_on_spd_input():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((30, 40))
    A = X @ X.T + np.eye(30)
    L, s = hifde.ldl_signed(A)
    assert np.all(s == 1.0)
    assert np.allclose(L, np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)
    with pytest.raises(np.linalg.LinAlgError):
        hifde.ldl_signed(np.array([[0.0, 1.0], [1.0, 0.0]]))


@pytest.mark.parametrize("dim,n,ppw", [(2, 32, 32), (2, 64, 32), (2, 64, 16), (3, 12, 8)])
def test_mf_on_helmholtz_matches_dense_solve(dim, n, ppw):
    a, b = inputs.helmholtz_coefficients(dim, n, ppw)
    A = stencil.assemble(dim, n, a, b)
    ev = np.linalg.eigvalsh(A.toarray())
    assert (ev < 0).sum() >= 1                      # indefinite
    F = hifde.factor(A, dim, n, 0.0)
    f = inputs.rhs(dim, n, 2, seed=3)
    x = F.apply_inverse(f)
    xd = np.linalg.solve(A.toarray(), f)
    kappa = np.abs(ev).max() / np.abs(ev).min()
    assert np.linalg.norm(x - xd) <= max(1e-12, 10 * 2.2e-16 * kappa) * np.linalg.norm(xd)
    # F itself reproduces A on the vectors (MF is exact)
    assert np.linalg.norm(F.apply(xd) - f) <= 1e-10 * np.linalg.norm(f)
    # the root carries negative signs
    assert F.Dsgn is not None and (F.Dsgn < 0).any()


def test_hifde_on_helmholtz_is_an_accurate_preconditioner():
    dim, n, eps = 2, 64, 1e-6
    a, b = inputs.helmholtz_coefficients(dim, n, 16)
    A = stencil.assemble(dim, n, a, b)
    F = hifde.factor(A, dim, n, eps)
    nneg = sum(int((r.sgn < 0).sum()) for lev in F.levels for r in lev.cells if r.sgn is not None)
    nneg += sum(int((fr.sgn < 0).sum()) for lev in F.levels for fr in lev.fronts if fr.sgn is not None)
    assert nneg > 0                                  # indefinite blocks below the root
    ea, es = hifde.power_estimates(A, F, inputs.power_start(dim, n))
    assert ea <= 100 * eps
    f = inputs.rhs(dim, n, 1, seed=4)
    x, it, rel = hifde.fgmres(A, F.apply_inverse, f, tol=1e-12, maxit=60)
    assert rel[0] <= 1e-12 and it[0] <= 20
