"""The two-sided (unsymmetric) factorization on the GPU (hif_opts.two_sided,
the generalization of Section 6) against the oracle's two-sided variant
(``hifde.factor(..., two_sided=True)``) on the stencil plus a convection
term beta . grad u (central differences; A unsymmetric, its symmetric part
SPD): the same fronts, skeletons in pivot order and ranks as the oracle's
(both take the pivoted-QR ID of the stacked [A_{N,c}; A_{c,N}^T]), the same
|s_L|, and F^-1 x, F x element-wise within 1e-10 of the largest entry in
FP64; MF against a dense solve; with beta = 0 the two-sided factorization
gives the symmetric one's F^-1 x; the FP32-stored factor within the FP32
apply bound d u32 kappa(A).  Cases: 2D 31^2 (eps 1e-6) and 63^2 (1e-3), 3D
11^3 (1e-3, faces).
"""
import numpy as np
import pytest

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs

pytestmark = pytest.mark.gpu

BETA = {2: (100.0, -60.0), 3: (40.0, 25.0, -30.0)}
CASES = [(2, 32, 1e-6), (2, 64, 1e-3), (3, 12, 1e-3)]


def _problem(dim, n, beta):
    a, b = inputs.high_contrast_coefficients(dim, n, seed=3, low=0.5, high=2.0)
    A = (stencil.assemble(dim, n, a, b) + stencil.convection(dim, n, beta)).tocsr()
    return a, b, A


@pytest.mark.parametrize("dim,n,eps", CASES)
def test_two_sided_matches_oracle(hiflib, dim, n, eps):
    from paper_1307_2895_gb300 import hif
    beta = BETA[dim]
    a, b, A = _problem(dim, n, beta)
    F = hifde.factor(A, dim, n, eps, two_sided=True)
    x = inputs.rhs(dim, n, 5, seed=7)
    G = hif.factor(dim, n, a, b, eps, precision="fp64", two_sided=True, beta=beta)
    try:
        fronts, root = G.structure()
        st = G.stats()
        yi = G.apply(x, inverse=True)
        yf = G.apply(x, inverse=False)
    finally:
        G.free()
    ostruct, oroot = F.skeleton_structure()
    got = {(lev, tuple(c)): sk for lev, c, sk in fronts}
    nfr = 0
    for lev, d in enumerate(ostruct):
        for key, (c, sk, k) in d.items():
            assert got.get((lev, tuple(c))) == sk, f"level {lev} front {c[:4]}...: skeletons differ"
            nfr += 1
    assert nfr == len(fronts) and nfr > 0
    assert root == oroot and st["root_size"] == oroot
    assert st["near_threshold_fronts"] == 0
    oi, of = F.apply_inverse(x), F.apply(x)
    ei = np.abs(yi - oi).max() / np.abs(oi).max()
    ef = np.abs(yf - of).max() / np.abs(of).max()
    ax = A @ x
    print(f"two-sided {dim}D n={n} eps={eps:g}: |s_L| {root}, F^-1 x {ei:.2e}, F x {ef:.2e}, "
          f"||Fx - Ax|| / ||Ax|| {np.linalg.norm(yf - ax) / np.linalg.norm(ax):.1e}")
    assert ei <= 1e-10
    assert ef <= 1e-10


def test_two_sided_mf_is_exact(hiflib):
    from paper_1307_2895_gb300 import hif
    dim, n = 2, 32
    beta = BETA[dim]
    a, b, A = _problem(dim, n, beta)
    f = inputs.rhs(dim, n, 3, seed=1)
    G = hif.factor(dim, n, a, b, 0.0, variant="mf", precision="fp64", two_sided=True, beta=beta)
    try:
        y = G.apply(f, inverse=True)
    finally:
        G.free()
    xd = np.linalg.solve(A.toarray(), f)
    assert np.abs(y - xd).max() <= 1e-10 * np.abs(xd).max()


def test_two_sided_without_convection_is_the_symmetric_factorization(hiflib):
    from paper_1307_2895_gb300 import hif
    dim, n, eps = 2, 64, 1e-6
    a, b = inputs.high_contrast_coefficients(dim, n, seed=3, low=0.5, high=2.0)
    x = inputs.rhs(dim, n, 2, seed=3)
    ys = []
    for two in (False, True):
        G = hif.factor(dim, n, a, b, eps, precision="fp64", two_sided=two)
        try:
            ys.append((G.structure(), G.apply(x, inverse=True)))
        finally:
            G.free()
    assert ys[0][0] == ys[1][0]
    assert np.abs(ys[1][1] - ys[0][1]).max() <= 1e-11 * np.abs(ys[0][1]).max()


def test_two_sided_fp32_apply(hiflib):
    from paper_1307_2895_gb300 import hif
    dim, n, eps = 2, 64, 1e-6
    beta = BETA[dim]
    a, b, A = _problem(dim, n, beta)
    F = hifde.factor(A, dim, n, eps, two_sided=True)
    x = inputs.rhs(dim, n, 3, seed=4)
    G = hif.factor(dim, n, a, b, eps, precision="fp32_apply", two_sided=True, beta=beta)
    try:
        yi = G.apply(x, inverse=True)
        with pytest.raises(Exception):   # the solver's stencil products have no convection term
            G.solve(x)
    finally:
        G.free()
    oi = F.apply_inverse(x)
    kappa = np.linalg.cond(A.toarray())
    bound = (2 * (2 * F.L + 1) + 1) * 2.0 ** -24 * kappa
    elem = np.abs(yi - oi).max() / np.abs(oi).max()
    print(f"two-sided fp32_apply 2D n={n}: element-wise {elem:.2e}, bound d u32 kappa = {bound:.2e}")
    assert elem <= bound


def test_two_sided_option_errors(hiflib):
    from paper_1307_2895_gb300 import hif
    a, b = inputs.constant_coefficients(2, 16)
    with pytest.raises(Exception):
        hif.factor(2, 16, a, b, 1e-3, beta=(1.0, 0.0))                    # beta needs two_sided
    with pytest.raises(Exception):
        hif.factor(2, 16, a, b, 1e-3, precision="mixed", two_sided=True)
    with pytest.raises(Exception):
        hif.factor(2, 16, a, b, 1e-3, skel="svd", two_sided=True)
