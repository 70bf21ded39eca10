"""Pins of the oracle's flexible GMRES (oracle.hifde.fgmres) against facts
that do not come from it: finite termination of a Krylov method, the exact
preconditioner, the dense solve and scipy's independent GMRES, the monotone
residual of a minimal-residual cycle, and PCG on an SPD system preconditioned
by the oracle's own HIF-DE factor."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs


def _nonsym(n, seed):
    rng = np.random.default_rng(seed)
    return np.eye(n) * 4 + rng.standard_normal((n, n)) / np.sqrt(n)


def test_finite_termination_unpreconditioned():
    """Without restarts GMRES solves an n x n system in at most n steps."""
    n = 24
    A = _nonsym(n, 1)
    b = np.random.default_rng(2).standard_normal(n)
    x, it, rel = hifde.fgmres(A, lambda v: v, b, tol=1e-12, maxit=200, restart=n)
    assert it[0] <= n and rel[0] <= 1e-12
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-10 * np.linalg.norm(x))


def test_exact_preconditioner_one_step():
    n = 30
    A = _nonsym(n, 3)
    b = np.random.default_rng(4).standard_normal(n)
    x, it, rel = hifde.fgmres(A, lambda v: np.linalg.solve(A, v), b, tol=1e-12)
    assert it[0] == 1 and rel[0] <= 1e-12


def test_matches_scipy_gmres_and_dense_solve():
    n = 60
    A = _nonsym(n, 5)
    b = np.random.default_rng(6).standard_normal((n, 2))
    D = np.diag(1.0 / np.diag(A))
    x, it, rel = hifde.fgmres(A, lambda v: D @ v, b, tol=1e-11, restart=10, maxit=400)
    xd = np.linalg.solve(A, b)
    assert np.abs(x - xd).max() <= 1e-9 * np.abs(xd).max()
    for c in range(2):
        xs, info = spla.gmres(A, b[:, c], rtol=1e-11, restart=10, maxiter=400)
        assert info == 0
        assert np.abs(x[:, c] - xs).max() <= 1e-8 * np.abs(xs).max()


def test_residual_monotone_within_a_cycle():
    """The cycle's least-squares residual is ||b - A x_j||: it never grows."""
    n = 40
    A = _nonsym(n, 7)
    b = np.random.default_rng(8).standard_normal(n)
    res = []
    for k in range(1, 25):
        x, it, rel = hifde.fgmres(A, lambda v: v, b, tol=1e-14, maxit=k, restart=40)
        res.append(rel[0])
    assert all(res[i + 1] <= res[i] * (1 + 1e-12) for i in range(len(res) - 1))


@pytest.mark.parametrize("dim,n", [(2, 16), (3, 8)])
def test_hif_preconditioned_spd_matches_pcg(dim, n):
    """SPD A with the SPD preconditioner F^-1 of the oracle's HIF-DE: GMRES and
    PCG both reach 1e-10, with similar iteration counts (right-preconditioned
    GMRES minimizes the residual over the same Krylov space)."""
    a, b = inputs.high_contrast_coefficients(dim, n, seed=11, low=1e-2, high=1e2)
    A = stencil.assemble(dim, n, a, b)
    F = hifde.factor(A, dim, n, 1e-3)
    f = inputs.rhs(dim, n, 1, seed=0)
    xg, itg, relg = hifde.fgmres(A, F.apply_inverse, f, tol=1e-10)
    xc, itc, relc = hifde.pcg(A, F, f, tol=1e-10)
    assert relg[0] <= 1e-10 and relc[0] <= 1e-10
    assert itg[0] <= itc[0] + 2
    assert np.linalg.norm(xg - xc) <= 1e-6 * np.linalg.norm(xc)
