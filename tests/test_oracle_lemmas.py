"""Pins of the oracle's building blocks against dense algebra and LAPACK:
Lemma 2.1 (sparse elimination), Lemma 2.2 / Cor. 2.3 (ID), Lemma 2.4
(skeletonization)."""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import hifde


def _spd_with_structure(rng, npp, nq, nr):
    """Random SPD matrix over (p, q, r) with A_pr = 0 (Eq. 2.1 structure)."""
    n = npp + nq + nr
    X = rng.standard_normal((n, n))
    A = X @ X.T / n + np.eye(n)
    A[:npp, npp + nq:] = 0.0
    A[npp + nq:, :npp] = 0.0
    A += n * np.eye(n)          # keep it SPD after zeroing
    return A


def _dense_op(apply, n):
    M = np.eye(n)
    for j in range(n):
        apply(M[:, j:j + 1])  # in place on a column view
    return M


def test_lemma21_schur_and_decoupling():
    rng = np.random.default_rng(0)
    npp, nq, nr = 6, 5, 7
    A = _spd_with_structure(rng, npp, nq, nr)
    act = hifde.ActiveMatrix(sp.csr_matrix(A))
    p = list(range(npp))
    rec = hifde.eliminate(act, p)
    q = list(range(npp, npp + nq))
    assert rec.q.tolist() == q                      # c^N from the sparsity pattern
    # Schur complement through an explicit inverse (independent of Cholesky)
    Bqq = A[npp:npp + nq, npp:npp + nq] - A[npp:npp + nq, :npp] @ np.linalg.inv(A[:npp, :npp]) @ A[:npp, npp:npp + nq]
    rest = list(range(npp, npp + nq + nr))
    got = act.block(rest, rest)
    expect = A[npp:, npp:].copy()
    expect[:nq, :nq] = Bqq
    assert np.allclose(got, expect, rtol=0, atol=1e-12 * np.abs(A).max())
    # S_p^T A S_p = diag(I, B): build S from the oracle's operator
    n = A.shape[0]
    S = np.eye(n)
    for j in range(n):
        col = S[:, j].copy()
        hifde.apply_S(rec, col)
        S[:, j] = col
    M = S.T @ A @ S
    assert np.allclose(M[:npp, :npp], np.eye(npp), atol=1e-12)
    assert np.abs(M[:npp, npp:]).max() <= 1e-12 * np.abs(A).max()
    assert np.allclose(M[npp:, npp:], expect, atol=1e-11 * np.abs(A).max())
    # S^-1 and S^T / S^-T consistency
    x = rng.standard_normal(n)
    y = x.copy(); hifde.apply_S(rec, y); hifde.apply_S_inv(rec, y)
    assert np.allclose(y, x, atol=1e-13)
    y = x.copy(); hifde.apply_S_T(rec, y); hifde.apply_S_inv_T(rec, y)
    assert np.allclose(y, x, atol=1e-13)
    y = x.copy(); hifde.apply_S_T(rec, y)
    assert np.allclose(y, S.T @ x, atol=1e-13)


def test_id_exact_low_rank():
    rng = np.random.default_rng(1)
    for (m, n, k) in [(40, 12, 5), (30, 30, 9), (8, 20, 4)]:
        M = rng.standard_normal((m, k)) @ rng.standard_normal((k, n))
        r = hifde.interp_decomp(M, 1e-10)
        assert len(r.sk) == k
        assert sorted(r.sk.tolist() + r.rd.tolist()) == list(range(n))
        assert np.all(np.diff(r.rd) > 0)
        E = M[:, r.rd] - M[:, r.sk] @ r.T
        assert np.linalg.norm(E) <= 1e-12 * np.linalg.norm(M)


def test_id_pivots_match_lapack():
    """Without ties the pivot order equals LAPACK's column-pivoted QR (dgeqp3)."""
    rng = np.random.default_rng(2)
    for _ in range(5):
        M = rng.standard_normal((25, 10)) * rng.uniform(0.1, 10, size=10)
        r = hifde.interp_decomp(M, 1e-15)
        _, R, piv = sla.qr(M, pivoting=True, mode="economic")
        assert r.sk.tolist() == piv[:len(r.sk)].tolist()
        assert np.allclose(np.abs(r.pivots[:len(r.sk)]), np.abs(np.diag(R))[:len(r.sk)], rtol=1e-12)


def test_id_rank_rule_orthogonal_columns():
    """Orthogonal columns with norms d: |R_ii| are the sorted d, so the rank is
    #{d_j > eps max d} and the skeletons are the columns by decreasing norm."""
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 12)))
    d = np.array([1.0, 3e-1, 1e-1, 5e-2, 2e-3, 9e-4, 1.1e-4, 9e-5, 1e-6, 1e-7, 1e-9, 5e-2 * 0.9])
    M = Q * d
    for eps, k in [(2e-1, 2), (1e-3, 6), (1e-4, 8), (1e-5, 9), (1e-8, 11)]:
        r = hifde.interp_decomp(M, eps)
        assert len(r.sk) == k
        assert r.sk.tolist() == np.argsort(-d, kind="stable")[:k].tolist()


def test_id_tie_rule_lowest_index():
    """Equal residual norms: the lowest original column position is the pivot."""
    M = np.zeros((4, 4))
    M[0, 2] = 1.0
    M[1, 0] = 1.0
    M[2, 3] = 0.5
    M[3, 1] = 1.0
    r = hifde.interp_decomp(M, 1e-12)
    assert r.sk.tolist()[:3] == [0, 1, 2]


def test_id_error_bounds_statistically():
    """||T|| <= sqrt(4k(n-k)) and ||E|| <= sqrt(1+4k(n-k)) sigma_{k+1} (Section 2.2)
    hold for the large majority of random matrices with decaying spectra."""
    rng = np.random.default_rng(4)
    ok_T = ok_E = total = 0
    for _ in range(40):
        m, n = 40, 20
        U, _ = np.linalg.qr(rng.standard_normal((m, n)))
        V, _ = np.linalg.qr(rng.standard_normal((n, n)))
        s = 10.0 ** (-np.arange(n) * rng.uniform(0.3, 1.0))
        M = (U * s) @ V.T
        r = hifde.interp_decomp(M, 1e-6)
        k = len(r.sk)
        if k in (0, n):
            continue
        total += 1
        E = M[:, r.rd] - M[:, r.sk] @ r.T
        sv = np.linalg.svd(M, compute_uv=False)
        ok_T += np.linalg.norm(r.T, 2) <= np.sqrt(4 * k * (n - k))
        ok_E += np.linalg.norm(E, 2) <= np.sqrt(1 + 4 * k * (n - k)) * sv[k]
    assert total >= 30 and ok_T >= 0.9 * total and ok_E >= 0.9 * total


def test_lemma24_skeletonization_exact_low_rank():
    """A_qp of exact rank k: Z_p(A) equals U^T A U with U = Q_p S_r exactly
    (Lemma 2.4): r decoupled, A_qs unchanged, A_qr = 0, B_ss the Schur form."""
    rng = np.random.default_rng(5)
    npp, nq, k = 9, 12, 3
    n = npp + nq
    X = rng.standard_normal((n, n))
    A = X @ X.T / n + n * np.eye(n)
    A[npp:, :npp] = rng.standard_normal((nq, k)) @ rng.standard_normal((k, npp))
    A[:npp, npp:] = A[npp:, :npp].T
    A += 2 * n * np.eye(n)
    assert np.all(np.linalg.eigvalsh(A) > 0)
    act = hifde.ActiveMatrix(sp.csr_matrix(A))
    p = list(range(npp))
    idr = hifde.interp_decomp(act.block(act.neighbors(p), p), 1e-12)
    assert len(idr.sk) == k
    fr = hifde.skeletonize(act, p, idr)
    U = np.eye(n)
    for j in range(n):
        col = U[:, j].copy()
        hifde.apply_U(fr, col)
        U[:, j] = col
    M = U.T @ A @ U
    rd, sk = fr.rd.tolist(), fr.sk.tolist()
    q = list(range(npp, n))
    scale = np.abs(A).max()
    assert np.allclose(M[np.ix_(rd, rd)], np.eye(len(rd)), atol=1e-10)
    others = sk + q
    assert np.abs(M[np.ix_(rd, others)]).max() <= 1e-10 * scale
    assert np.allclose(M[np.ix_(q, sk)], A[np.ix_(q, sk)], atol=1e-10 * scale)
    assert np.allclose(M[np.ix_(sk, sk)], act.block(sk, sk), atol=1e-10 * scale)
    # remaining active set is exactly s and q
    assert sorted(act.active()) == sorted(sk + q)
    # B_ss against the explicit formula with inverses (independent route)
    T = idr.T
    Ass, Asr, Arr = A[np.ix_(sk, sk)], A[np.ix_(sk, rd)], A[np.ix_(rd, rd)]
    Brr = Arr - T.T @ Asr - Asr.T @ T + T.T @ Ass @ T
    Bsr = Asr - Ass @ T
    Bss = Ass - Bsr @ np.linalg.inv(Brr) @ Bsr.T
    assert np.allclose(act.block(sk, sk), Bss, atol=1e-10 * scale)
