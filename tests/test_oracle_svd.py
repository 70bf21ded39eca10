"""Pins of the oracle's SVD skeletonization (Section 4.4) against what the
mathematics fixes: the rank rule and an orthogonal V on blocks of known rank,
one skeletonization of a block with exactly low-rank interactions (F = A to
rounding, with a real rotation), the whole factorization exact when nothing
is truncated, and ||A - F|| / ||A|| of order eps with F symmetric."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs


def test_svd_skel_rank_and_basis():
    rng = np.random.default_rng(4)
    U = rng.standard_normal((20, 3))
    W = rng.standard_normal((3, 12))
    M = U @ np.diag([5.0, 1.0, 1e-3]) @ W
    sv = hifde.svd_skel(M, 1e-6)
    assert sv.k == 3 and not sv.near_threshold
    assert np.allclose(sv.V.T @ sv.V, np.eye(12), atol=1e-14)
    assert np.all(np.diff(sv.sigma) <= 0)
    # the dropped directions carry no interaction, the kept ones all of it
    assert np.linalg.norm(M @ sv.V[:, 3:]) <= 1e-13 * np.linalg.norm(M)
    assert np.isclose(np.linalg.norm(M @ sv.V[:, :3]), np.linalg.norm(M), rtol=1e-14)
    # the rank rule: sigma_i > eps sigma_1
    assert hifde.svd_skel(M, 1e-3 / 5.0 * 1.001).k == 2
    assert hifde.svd_skel(np.zeros((4, 5)), 1e-6).k == 0
    assert hifde.svd_skel(np.zeros((0, 5)), 1e-6).k == 0


def _low_rank_problem(seed=5, np_=6, nq=8, rank=2):
    rng = np.random.default_rng(seed)
    n = np_ + nq
    A = np.zeros((n, n))
    B = rng.standard_normal((np_, np_))
    A[:np_, :np_] = B @ B.T + np_ * np.eye(np_)
    C = rng.standard_normal((nq, nq))
    A[np_:, np_:] = C @ C.T + 50.0 * np.eye(nq)
    Aqp = rng.standard_normal((nq, rank)) @ rng.standard_normal((rank, np_))
    A[np_:, :np_] = Aqp
    A[:np_, np_:] = Aqp.T
    return A


def test_skeletonize_svd_exact_on_low_rank_interactions():
    """Lemma of Section 4.4 with A_qp of exact rank 2: after Q_c and the
    elimination of the four dropped directions, F = A to rounding; the
    rotation is a real one (0 < k < |c|)."""
    A = _low_rank_problem()
    Am = hifde.ActiveMatrix(sp.csr_matrix(A))
    c = list(range(6))
    sv = hifde.svd_skel(Am.block(Am.neighbors(c), c), 1e-10)
    assert sv.k == 2
    fr = hifde.skeletonize_svd(Am, c, sv)
    assert fr.V is not None and len(fr.sk) == 2 and len(fr.rd) == 4
    act = Am.active()
    assert act == [0, 1] + list(range(6, 14))
    D = Am.block(act, act)
    b = inputs.standard_normal(11, 14)
    # F^-1 b = U_c^-T ... : apply_U_T, D^-1 on the active set, apply_U
    x = b.copy()
    hifde.apply_U_T(fr, x)
    x[act] = np.linalg.solve(D, x[act])
    hifde.apply_U(fr, x)
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)
    # F b through the inverse operators
    y = b.copy()
    hifde.apply_U_inv(fr, y)
    y[act] = D @ y[act]
    hifde.apply_U_inv_T(fr, y)
    assert np.linalg.norm(y - A @ b) <= 1e-12 * np.linalg.norm(A @ b)


@pytest.mark.parametrize("dim,n", [(2, 16), (3, 8)])
def test_svd_factor_exact_without_truncation(dim, n):
    a, b = inputs.high_contrast_coefficients(dim, n, seed=3, low=1e-2, high=1e2)
    A = stencil.assemble(dim, n, a, b)
    F = hifde.factor(A, dim, n, 1e-300, skel="svd")
    v = inputs.standard_normal(3, A.shape[0])
    assert np.linalg.norm(F.apply(v) - A @ v) <= 1e-13 * np.linalg.norm(A @ v)


@pytest.mark.parametrize("dim,n,eps", [(2, 16, 1e-6), (2, 32, 1e-3), (3, 12, 1e-3)])
def test_svd_factor_error_of_order_eps(dim, n, eps):
    """||A - F||_2 <= eps ||A||_2, F symmetric, F^-1 F = I: with rotations
    taken (a wrong transpose of V or a dropped Schur term gives O(1))."""
    a, b = inputs.high_contrast_coefficients(dim, n, seed=3, low=1e-2, high=1e2)
    A = stencil.assemble(dim, n, a, b)
    Ad = A.toarray()
    N = Ad.shape[0]
    F = hifde.factor(A, dim, n, eps, skel="svd")
    assert sum(1 for lev in F.levels for fr in lev.fronts if fr.V is not None) > 0
    Fd = F.apply(np.eye(N))
    ea = np.linalg.norm(Ad - Fd, 2) / np.linalg.norm(Ad, 2)
    assert 0.0 < ea <= eps
    assert np.abs(Fd - Fd.T).max() <= 1e-14 * np.abs(Fd).max()
    assert np.abs(F.apply_inverse(Fd) - np.eye(N)).max() <= 1e-10
