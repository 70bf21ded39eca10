"""Pins of the oracle's two-sided (unsymmetric) variant, the generalization
Section 6 sketches: two-sided elimination operators from A_pp = L U and the
ID of the stacked [A_{N,c}; A_{c,N}^T].  Checked against what the
mathematics fixes: the convection stencil on linear functions, the LU, MF
against a dense solve, exactness with nothing truncated, the symmetric
factorization recovered for a symmetric A, ||A - F|| of order eps with F as
unsymmetric as A, and GMRES with F^-1 as the preconditioner."""
import numpy as np
import pytest

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs

BETA = {2: (100.0, -60.0), 3: (40.0, 25.0, -30.0)}


def _problem(dim, n, beta=None, seed=3):
    a, b = inputs.high_contrast_coefficients(dim, n, seed=seed, low=0.5, high=2.0)
    A = stencil.assemble(dim, n, a, b)
    if beta is None:
        beta = BETA[dim]
    return (A + stencil.convection(dim, n, beta)).tocsr()


@pytest.mark.parametrize("dim", [2, 3])
def test_convection_skew_and_exact_on_linear_functions(dim):
    n = 9
    beta = BETA[dim]
    C = stencil.convection(dim, n, beta)
    assert abs(C + C.T).max() == 0.0
    X = stencil.coords(dim, n).astype(np.float64)       # integer node coordinates, x first
    h = 1.0 / n
    inner = np.all((X > 1) & (X < n - 1), axis=1)       # every neighbour interior
    for axis in range(dim):
        u = X[:, axis] * h
        assert np.allclose((C @ u)[inner], beta[axis], rtol=0, atol=1e-9 * abs(beta[axis]))


def test_lu_nopivot():
    rng = np.random.default_rng(2)
    M = rng.standard_normal((12, 12)) + 12 * np.eye(12)
    L, U = hifde.lu_nopivot(M)
    assert np.allclose(np.diag(L), 1.0) and np.allclose(L, np.tril(L)) and np.allclose(U, np.triu(U))
    assert np.abs(L @ U - M).max() <= 1e-13 * np.abs(M).max()


@pytest.mark.parametrize("dim,n", [(2, 16), (2, 27), (3, 8)])
def test_two_sided_mf_is_exact(dim, n):
    A = _problem(dim, n)
    f = inputs.rhs(dim, n, 2)
    F = hifde.factor(A, dim, n, 0.0, two_sided=True)
    xd = np.linalg.solve(A.toarray(), f)
    assert np.linalg.norm(F.apply_inverse(f) - xd) <= 1e-12 * np.linalg.norm(xd)
    v = inputs.standard_normal(3, A.shape[0])
    assert np.linalg.norm(F.apply(v) - A @ v) <= 1e-13 * np.linalg.norm(A @ v)


@pytest.mark.parametrize("dim,n", [(2, 32), (3, 12)])
def test_two_sided_exact_without_truncation(dim, n):
    A = _problem(dim, n)
    F = hifde.factor(A, dim, n, 1e-300, two_sided=True)
    v = inputs.standard_normal(4, A.shape[0])
    assert np.linalg.norm(F.apply(v) - A @ v) <= 1e-13 * np.linalg.norm(A @ v)


@pytest.mark.parametrize("dim,n,eps", [(2, 32, 1e-6), (3, 12, 1e-3)])
def test_two_sided_recovers_the_symmetric_factorization(dim, n, eps):
    A = _problem(dim, n, beta=(0.0,) * dim)
    F2 = hifde.factor(A, dim, n, eps, two_sided=True)
    F1 = hifde.factor(A, dim, n, eps)
    assert F2.skeleton_structure() == F1.skeleton_structure()
    f = inputs.rhs(dim, n, 2, seed=4)
    y1 = F1.apply_inverse(f)
    assert np.linalg.norm(F2.apply_inverse(f) - y1) <= 1e-11 * np.linalg.norm(y1)


@pytest.mark.parametrize("dim,n,eps", [(2, 32, 1e-6), (2, 32, 1e-3), (3, 12, 1e-3)])
def test_two_sided_error_of_order_eps(dim, n, eps):
    A = _problem(dim, n)
    Ad = A.toarray()
    N = Ad.shape[0]
    F = hifde.factor(A, dim, n, eps, two_sided=True)
    Fd = F.apply(np.eye(N))
    ea = np.linalg.norm(Ad - Fd, 2) / np.linalg.norm(Ad, 2)
    assert 0.0 < ea <= eps
    skew = np.linalg.norm(Ad - Ad.T, 2)
    assert np.linalg.norm(Fd - Fd.T, 2) >= 0.5 * skew        # F is as unsymmetric as A
    assert np.abs(F.apply_inverse(Fd) - np.eye(N)).max() <= 1e-10


def test_two_sided_preconditioned_gmres():
    dim, n = 2, 64
    A = _problem(dim, n)
    F = hifde.factor(A, dim, n, 1e-6, two_sided=True)
    b = inputs.rhs(dim, n, 1, seed=8)[:, 0]
    x, iters, rel = hifde.fgmres(A, F.apply_inverse, b, tol=1e-12, maxit=50)
    print(f"two-sided 63^2: GMRES {iters[0]} iterations, relres {rel[0]:.1e}")
    assert rel[0] <= 1e-12 and iters[0] <= 6
    assert np.linalg.norm(A @ x.ravel() - b) <= 1e-11 * np.linalg.norm(b)


@pytest.mark.parametrize("dim,n,eps", [(2, 32, 1e-6), (3, 12, 1e-3)])
def test_two_sided_commutes_with_transposition(dim, n, eps):
    """Factoring A^T (beta -> -beta) stacks the same two blocks in the other
    order, so the pivoted QR picks the same skeletons and T, and the
    factorization is the transpose: F(A^T) = F(A)^T.  A mix-up of the row
    and column operators (A_qp against A_pq^T, L against U^T) breaks it."""
    A = _problem(dim, n)
    At = _problem(dim, n, beta=tuple(-b for b in BETA[dim]))
    assert abs(At - A.T).max() <= 1e-12 * abs(A).max()
    F = hifde.factor(A, dim, n, eps, two_sided=True)
    Ft = hifde.factor(At, dim, n, eps, two_sided=True)
    assert F.skeleton_structure() == Ft.skeleton_structure()
    N = A.shape[0]
    Fd = F.apply(np.eye(N))
    assert np.abs(Ft.apply(np.eye(N)) - Fd.T).max() <= 1e-12 * np.abs(Fd).max()
    Fi = F.apply_inverse(np.eye(N))
    assert np.abs(Ft.apply_inverse(np.eye(N)) - Fi.T).max() <= 1e-10 * np.abs(Fi).max()
