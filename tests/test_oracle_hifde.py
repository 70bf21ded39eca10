"""Pins of the oracle's MF / HIF-DE (Algorithms 3.1, 4.1), the apply of F and
F^-1 (Eq. 4.2), PCG and the error estimates against what the paper and the
mathematics fix: dense LU solves, exactness of MF, e_a = O(eps), structure
invariants, and the paper's Table 7 at 31^3."""
import os

import numpy as np
import pytest

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _problem(dim, n, contrast=False, seed=7):
    if contrast:
        a, b = inputs.high_contrast_coefficients(dim, n, seed=seed, low=1e-2, high=1e2)
    else:
        a, b = inputs.constant_coefficients(dim, n)
    return stencil.assemble(dim, n, a, b)


@pytest.mark.parametrize("dim,n,contrast", [(2, 8, False), (2, 16, True), (2, 32, False), (2, 27, True),
                                            (3, 8, False), (3, 12, True)])
def test_mf_is_exact(dim, n, contrast):
    """eps -> 0 (skeletonization off): F^-1 b equals the dense LU solve."""
    A = _problem(dim, n, contrast)
    f = inputs.rhs(dim, n, 2)
    F = hifde.factor(A, dim, n, 0.0)
    x = F.apply_inverse(f)
    xd = np.linalg.solve(A.toarray(), f)
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd) * (100 if contrast else 1)
    # F itself reproduces A
    v = inputs.standard_normal(3, A.shape[0])
    assert np.linalg.norm(F.apply(v) - A @ v) <= 1e-12 * np.linalg.norm(A @ v) * (100 if contrast else 1)


@pytest.mark.parametrize("dim,n", [(2, 16), (2, 32), (3, 8)])
def test_hif_tiny_eps_matches_dense(dim, n):
    A = _problem(dim, n)
    f = inputs.rhs(dim, n, 1)[:, 0]
    F = hifde.factor(A, dim, n, 1e-14)
    assert sum(len(l.fronts) for l in F.levels) > 0
    xd = np.linalg.solve(A.toarray(), f)
    assert np.linalg.norm(F.apply_inverse(f) - xd) <= 1e-10 * np.linalg.norm(xd)


def test_inverse_and_symmetry():
    dim, n = 2, 32
    A = _problem(dim, n, contrast=True)
    F = hifde.factor(A, dim, n, 1e-4)
    x = inputs.standard_normal(1, A.shape[0])
    y = inputs.standard_normal(2, A.shape[0])
    assert np.linalg.norm(F.apply(F.apply_inverse(x)) - x) <= 1e-12 * np.linalg.norm(x) * 1e2
    assert abs(x @ F.apply(y) - y @ F.apply(x)) <= 1e-12 * abs(x @ F.apply(y)) * 1e2
    assert abs(x @ F.apply_inverse(y) - y @ F.apply_inverse(x)) <= 1e-10 * abs(x @ F.apply_inverse(y))


def test_structure_partition():
    """Every DOF is eliminated exactly once (cells, redundant front DOFs, root);
    s and r split each front; fronts hold only strict edge interiors."""
    dim, n = 2, 64
    A = _problem(dim, n)
    F = hifde.factor(A, dim, n, 1e-6)
    seen = []
    X = stencil.coords(dim, n)
    for lev in F.levels:
        seps = hifde.level_separators(n, F.L, lev.ell)
        for c in lev.cells:
            seen += c.p.tolist()
        for fr in lev.fronts:
            assert sorted(fr.sk.tolist() + fr.rd.tolist()) == fr.c.tolist()
            on = np.isin(X[fr.c], seps).sum(axis=1)
            assert np.all(on == 1)
            seen += fr.rd.tolist()
    seen += F.root.tolist()
    assert sorted(seen) == list(range(A.shape[0]))


def test_error_estimates_scale_with_eps():
    """e_a = O(eps) (Section 5, Tables 2, 8): decreases with eps and stays
    within a modest factor of eps; e_s >= e_a."""
    dim, n = 2, 64
    A = _problem(dim, n)
    x0 = inputs.power_start(dim, n)
    prev = None
    for eps in (1e-3, 1e-6, 1e-9):
        F = hifde.factor(A, dim, n, eps)
        ea, es = hifde.power_estimates(A, F, x0)
        assert ea <= 20 * eps
        assert es >= ea
        if prev is not None:
            assert ea < prev
        prev = ea


def test_pcg_converges_fast():
    """F^-1 is an effective preconditioner (Section 5, Tables 2, 4): few
    iterations.  The Laplacian reaches 1e-12; the contrast-1e4 field stops at
    1e-10 because its FP64 residual floor (sparse LU + refinement) is ~2e-12."""
    dim, n = 2, 64
    A = _problem(dim, n)
    F = hifde.factor(A, dim, n, 1e-6)
    f = inputs.rhs(dim, n, 2)
    x, iters, rel = hifde.pcg(A, F, f, tol=1e-12)
    assert max(rel) <= 1e-12 and max(iters) <= 8
    A = _problem(dim, n, contrast=True)
    F = hifde.factor(A, dim, n, 1e-6)
    x, iters, rel = hifde.pcg(A, F, f, tol=1e-10)
    assert max(rel) <= 1e-10 and max(iters) <= 12


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return rows


@pytest.mark.parametrize("row", [0, 1])
def test_paper_table7_soft_pin(row):
    """Example 4 at 31^3 (Table 7 / 8): |s_L| within 10% of the paper's, e_a
    within a factor 10 and e_s within a factor 5 (the paper's tree details
    differ slightly; e_s also carries kappa(A))."""
    eps, sL, ea_paper, _, es_paper = _read_golden("paper_table7_example4.txt")[row]
    dim, n = 3, 32
    A = _problem(dim, n)
    F = hifde.factor(A, dim, n, eps)
    assert abs(len(F.root) - sL) <= 0.1 * sL
    ea, es = hifde.power_estimates(A, F, inputs.power_start(dim, n))
    assert ea_paper / 10 <= ea <= ea_paper * 10
    assert es_paper / 5 <= es <= es_paper * 5


# ---- planted mistakes: the pins above must catch them ---------------------

def test_planted_sign_error_in_T_is_caught(monkeypatch):
    real = hifde.interp_decomp

    def bad(M, eps):
        r = real(M, eps)
        r.T = -r.T
        return r

    dim, n, eps = 2, 32, 1e-6
    A = _problem(dim, n)
    v = inputs.standard_normal(4, A.shape[0])
    good = hifde.factor(A, dim, n, eps)
    assert np.linalg.norm(good.apply(v) - A @ v) <= 20 * eps * np.linalg.norm(A @ v)
    monkeypatch.setattr(hifde, "interp_decomp", bad)
    F = hifde.factor(A, dim, n, eps)
    assert np.linalg.norm(F.apply(v) - A @ v) > 1e3 * eps * np.linalg.norm(A @ v)


def test_planted_dropped_stencil_term_is_caught():
    dim, n = 2, 16
    a, b = inputs.constant_coefficients(dim, n)
    A = stencil.assemble(dim, n, a, b).tolil()
    A[5, 5] -= n * n          # one bond missing from a diagonal entry
    h = 1.0 / n
    X = stencil.coords(dim, n) / n
    v = np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])
    lam = (8.0 / h ** 2) * np.sin(np.pi * h / 2) ** 2
    assert np.linalg.norm(A.tocsr() @ v - lam * v) > 1e-6 * lam * np.linalg.norm(v)


@pytest.mark.parametrize("dim,n,eps,field", [(2, 16, 1e-3, "lap"), (2, 32, 1e-4, "contrast"),
                                             (3, 8, 1e-2, "lap"), (3, 12, 1e-3, "contrast")])
def test_power_estimates_against_exact_norms(dim, n, eps, field):
    """e_a and e_s of Section 5 against the exact 2-norms of A - F, A and
    I - A F^-1 (dense F and F^-1 from applying them to the identity): each
    power iteration stops at 1e-2 relative change, so each estimated norm is
    at most the true one and, on these problems, within 15% of it; e_a, a
    quotient of two such estimates, within 15% either way."""
    if field == "lap":
        a, b = inputs.constant_coefficients(dim, n)
    else:
        a, b = inputs.high_contrast_coefficients(dim, n, seed=3, low=1e-2, high=1e2)
    A = stencil.assemble(dim, n, a, b)
    F = hifde.factor(A, dim, n, eps)
    I = np.eye(A.shape[0])
    Ad = A.toarray()
    nA = np.linalg.norm(Ad, 2)
    nE = np.linalg.norm(Ad - F.apply(I), 2)
    es_x = np.linalg.norm(I - Ad @ F.apply_inverse(I), 2)
    x0 = inputs.power_start(dim, n)
    est_A = hifde.power_norm(lambda v: A @ v, x0)
    est_E = hifde.power_norm(lambda v: A @ v - F.apply(v), x0)
    assert 0.85 * nA <= est_A <= nA * (1 + 1e-12)
    assert 0.85 * nE <= est_E <= nE * (1 + 1e-9)
    ea, es = hifde.power_estimates(A, F, x0)
    assert ea == pytest.approx(est_E / est_A, rel=1e-12)
    assert 0.85 <= ea / (nE / nA) <= 1.15
    assert 0.85 * es_x <= es <= es_x * (1 + 1e-9)


@pytest.mark.parametrize("dim,n,eps", [(2, 32, 1e-2), (3, 12, 1e-1)])
def test_pcg_iterates_match_scipy_cg(dim, n, eps):
    """The oracle's PCG (Section 5) and scipy's preconditioned CG, the same
    textbook recurrences with M^-1 = F^-1, produce the same iterate after
    every step k (a loose eps keeps several steps before convergence)."""
    import scipy.sparse.linalg as spla
    a, b = inputs.high_contrast_coefficients(dim, n, seed=8, low=1e-1, high=1e1)
    A = stencil.assemble(dim, n, a, b)
    F = hifde.factor(A, dim, n, eps)
    f = inputs.rhs(dim, n, 1, seed=2)[:, 0]
    M = spla.LinearOperator(A.shape, matvec=lambda v: F.apply_inverse(np.asarray(v).ravel()))
    seen = []
    spla.cg(A, f, rtol=1e-15, atol=0.0, maxiter=6, M=M, callback=lambda xk: seen.append(xk.copy()))
    assert len(seen) == 6
    for k, xs in enumerate(seen, start=1):
        x, it, _ = hifde.pcg(A, F, f, tol=1e-15, maxit=k)
        assert it[0] == k
        assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs), k


@pytest.mark.parametrize("dim,n,eps", [(2, 32, 1e-6), (2, 64, 1e-6), (2, 32, 1e-9), (3, 16, 1e-3), (3, 16, 1e-6)])
def test_factor_on_closed_form_eigenmodes(dim, n, eps):
    """a = 1, b = 0: on the discrete sine modes v (A v = lambda v with the
    closed-form lambda of Section 5's Laplacian), F v = lambda v up to
    O(eps) relative to lambda, the lowest modes included (where A's own
    scale would allow eps kappa): at most 20 eps on these grids."""
    a, b = inputs.constant_coefficients(dim, n)
    A = stencil.assemble(dim, n, a, b)
    F = hifde.factor(A, dim, n, eps)
    h = 1.0 / n
    X = stencil.coords(dim, n) / n
    for idx in [(1,) * dim, (2,) + (1,) * (dim - 1), (3,) + (1,) * (dim - 1), (n // 2,) * dim, (n - 1,) * dim]:
        v = np.ones(X.shape[0])
        for ax, i in enumerate(idx):
            v *= np.sin(i * np.pi * X[:, ax])
        lam = (4.0 / h ** 2) * np.sum(np.sin(np.array(idx) * np.pi * h / 2) ** 2)
        assert np.linalg.norm(F.apply(v) - lam * v) <= 20 * eps * lam * np.linalg.norm(v), idx


@pytest.mark.parametrize("dim,n", [(2, 4), (2, 5), (3, 4), (3, 5)])
@pytest.mark.parametrize("eps", [0.0, 1e-6])
def test_smallest_grids_match_dense_solve(dim, n, eps):
    """The smallest trees (one level; at n = 4 every cell holds one DOF and
    every front one DOF): F^-1 b equals the dense solve to rounding, and
    every DOF is eliminated once."""
    a, b = inputs.high_contrast_coefficients(dim, n, seed=1, low=1e-2, high=1e2)
    A = stencil.assemble(dim, n, a, b)
    f = inputs.rhs(dim, n, 2)
    F = hifde.factor(A, dim, n, eps)
    xd = np.linalg.solve(A.toarray(), f)
    assert np.linalg.norm(F.apply_inverse(f) - xd) <= 1e-12 * np.linalg.norm(xd)
    done = [g for lev in F.levels for rec in lev.cells for g in rec.p.tolist()]
    done += [g for lev in F.levels for fr in lev.fronts for g in fr.rd.tolist()]
    assert sorted(done + F.root.tolist()) == list(range((n - 1) ** dim))
