"""Pins of the oracle's randomized ID and rank-prediction MLP (CPU)."""
import numpy as np

from oracle import learned
from paper_1307_2895_gb300 import inputs


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    nin, H, n = 10, 64, 37
    flat = rng.standard_normal(H * nin + H + H * H + H + H + 1) * 0.2
    X = rng.standard_normal((n, nin))
    t = rng.standard_normal(n) * 2
    net = learned.MLP.unpack(flat, nin, H)
    loss, g = net.loss_and_grad(X, t)
    idx = rng.choice(len(flat), 60, replace=False)
    for i in idx:
        h = 1e-6
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = learned.MLP.unpack(fp, nin, H).loss_and_grad(X, t)
        lm, _ = learned.MLP.unpack(fm, nin, H).loss_and_grad(X, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_mlp_huber_regions():
    """Residuals beyond delta contribute a clipped gradient (Huber loss)."""
    nin, H = 3, 64
    net = learned.MLP.unpack(np.zeros(H * nin + H + H * H + H + H + 1), nin, H)
    X = np.zeros((2, nin))
    loss, g = net.loss_and_grad(X, np.array([0.5, 5.0]))
    assert np.isclose(loss, (0.5 * 0.25 + (5.0 - 0.5)) / 2)
    assert np.isclose(g[-1], (-0.5 - 1.0) / 2)          # d/db3


def test_randomized_id_exact_low_rank():
    rng = np.random.default_rng(1)
    m, n, k = 60, 25, 6
    M = rng.standard_normal((m, k)) @ rng.standard_normal((k, n))
    ell = k + 10
    Phi = inputs.standard_normal(3, ell * m).reshape(ell, m)
    idr, ok = learned.randomized_id(M, 1e-10, Phi)
    assert ok and len(idr.sk) == k
    E = M[:, idr.rd] - M[:, idr.sk] @ idr.T
    assert np.linalg.norm(E) <= 1e-10 * np.linalg.norm(M)


def test_randomized_id_check_is_the_qr_stopping_rule():
    """The acceptance check is the pivoted QR's own stopping rule: on a
    matrix whose pivoted QR stops at rank k (|R_kk| > eps |R_11| >=
    |R_{k+1,k+1}|), the QR's ID passes the column check while the Frobenius
    test ||E||_F <= eps ||M||_F, stricter by up to sqrt(#columns), rejects
    it; and a sketched ID of a matrix with a clear gap (tail below
    SKETCH_RANK_TOL * eps) keeps at least the numerical rank and passes."""
    from oracle import hifde
    rng = np.random.default_rng(7)
    m, n, k, eps = 400, 200, 10, 1e-6
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.concatenate([np.logspace(0, -3, k), np.full(n - k, 0.1 * eps)])
    M = (U * s) @ V.T
    idq = hifde.interp_decomp(M, eps)
    E = M[:, idq.rd] - M[:, idq.sk] @ idq.T
    assert len(idq.sk) == k
    assert np.linalg.norm(E, axis=0).max() <= eps * np.linalg.norm(M, axis=0).max()
    assert np.linalg.norm(E) > eps * np.linalg.norm(M)

    m, n = 200, 60
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.concatenate([np.logspace(0, -3, k), np.full(n - k, 0.02 * eps)])
    M = (U * s) @ V.T
    Phi = inputs.standard_normal(8, (k + 30) * m).reshape(k + 30, m)
    idr, ok = learned.randomized_id(M, eps, Phi)
    E = M[:, idr.rd] - M[:, idr.sk] @ idr.T
    assert ok and k <= len(idr.sk) < k + 30
    assert np.linalg.norm(E, axis=0).max() <= eps * np.linalg.norm(M, axis=0).max()


def test_randomized_id_undersized_sketch_is_rejected():
    rng = np.random.default_rng(2)
    m, n = 50, 20
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    M = U * (10.0 ** -np.arange(n) * 0.5)     # numerical rank ~ 12 at eps 1e-6
    Phi = inputs.standard_normal(4, 4 * m).reshape(4, m)
    idr, ok = learned.randomized_id(M, 1e-6, Phi)
    assert not ok


def test_factor_with_identity_sketch_is_the_plain_factorization():
    """Phi = I makes the sketch the block itself: every front's randomized ID
    is its pivoted-QR ID at SKETCH_RANK_TOL * eps (least squares on the
    QR's skeletons gives the QR's own T) and passes the check at eps, so the
    factorization is the plain one at SKETCH_RANK_TOL * eps (same skeletons
    in pivot order, same root)."""
    from oracle.learned import SKETCH_RANK_TOL
    from oracle import hifde, stencil
    from paper_1307_2895_gb300 import inputs
    dim, n, eps = 2, 32, 1e-6
    a, b = inputs.high_contrast_coefficients(dim, n, seed=11, low=1e-2, high=1e2)
    A = stencil.assemble(dim, n, a, b)
    F0 = hifde.factor(A, dim, n, SKETCH_RANK_TOL * eps)
    F1 = hifde.factor(A, dim, n, eps, sketch=lambda l, c, rows: np.eye(len(rows)) if len(rows) > len(c) else None)
    s0, r0 = F0.skeleton_structure()
    s1, r1 = F1.skeleton_structure()
    assert s0 == s1 and r0 == r1
    assert F1.sketched > 0 and F1.fallback == 0


def test_factor_with_undersized_sketch_falls_back_everywhere():
    """A one-row sketch saturates (k = ell) on every front of rank > 1 or
    fails the check: each such front falls back to the pivoted-QR ID, so the
    skeletons are the plain ones and the rejections are counted."""
    from oracle import hifde, stencil
    from paper_1307_2895_gb300 import inputs
    dim, n, eps = 2, 32, 1e-6
    a, b = inputs.high_contrast_coefficients(dim, n, seed=11, low=1e-2, high=1e2)
    A = stencil.assemble(dim, n, a, b)
    F0 = hifde.factor(A, dim, n, eps)
    rng = np.random.default_rng(0)
    F1 = hifde.factor(A, dim, n, eps, sketch=lambda l, c, rows: rng.standard_normal((1, len(rows))))
    assert F1.skeleton_structure() == F0.skeleton_structure()
    nfronts = sum(len(lev.fronts) for lev in F1.levels)
    assert F1.sketched == 0 and F1.fallback == nfronts


def test_power_sketch_recovers_a_slowly_decaying_spectrum():
    """Power iterations (Section 4.5's remedy for inaccurate sketches): with
    one power iteration the rank rule is applied at (eps/10)^3 to Y, whose
    singular values are M's cubed, and recovers the numerical rank k of a
    matrix with a gap at k; with two, (eps/10)^5 = 1e-20 lies below FP64
    resolution, the sketch saturates and the ID falls back (the option is
    meaningful only while that threshold stays well above 1e-16)."""
    rng = np.random.default_rng(3)
    m, n, k, eps = 300, 120, 20, 1e-3
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.concatenate([np.logspace(0, -2, k), 1e-5 * np.logspace(0, -1, n - k)])
    M = (U * s) @ V.T
    Phi = inputs.standard_normal(9, (k + 4) * m).reshape(k + 4, m)
    idp, okp = learned.randomized_id(M, eps, Phi, power=1)
    assert okp and len(idp.sk) == k
    E = M[:, idp.rd] - M[:, idp.sk] @ idp.T
    assert np.linalg.norm(E, axis=0).max() <= eps * np.linalg.norm(M, axis=0).max()
    id2, ok2 = learned.randomized_id(M, eps, Phi, power=2)
    assert not ok2 and len(id2.sk) == k + 4
