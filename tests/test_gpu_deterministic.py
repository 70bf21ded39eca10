"""Bit-reproducible applications and solves (hif_opts.deterministic).

Without the option the cells of a level add their updates of shared
boundary DOFs with floating-point atomics, so F^-1 x depends on the order
the blocks run in.  With it: two independent factorizations of the same
problem give bit-identical F^-1 x and F x, and bit-identical solves, on the
2D bench workload (FP32-stored factor, 8 right-hand sides) and on 3D hifde3
at 31^3, whose root of more than 256 DOFs goes through the multi-block root
apply; the FP64 F^-1 x agrees with the oracle's to 1e-10 element-wise and
with the atomic form to 1e-13 (the FP32-stored one to 1e-3: a reordered FP32
addition is amplified by the later sweeps like any FP32 rounding, 3.5e-5 on
this workload).
"""
import numpy as np
import pytest

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(dim, n, a, b, eps, precision, det, x, solve=True):
    from paper_1307_2895_gb300 import hif
    G = hif.factor(dim, n, a, b, eps, precision=precision, deterministic=det)
    try:
        yi = G.apply(x, inverse=True)
        yf = G.apply(x, inverse=False)
        sol = G.solve(x, tol=1e-12, maxit=500) if solve else None
        root = G.stats()["root_size"]
    finally:
        G.free()
    return yi, yf, sol, root


@pytest.mark.parametrize("dim,n,precision", [(2, 512, "fp32_apply"), (3, 32, "fp64")])
def test_deterministic_applications_are_bit_identical(hiflib, dim, n, precision):
    if dim == 2:
        w = inputs.workload("contrast2d_n512")
        a, b, eps = w["a_stag"], w["b"], w["eps"]
    else:
        a, b = inputs.constant_coefficients(dim, n)
        eps = 1e-6
    x = inputs.rhs(dim, n, 8, seed=6)
    r1 = _run(dim, n, a, b, eps, precision, True, x)
    r2 = _run(dim, n, a, b, eps, precision, True, x)
    if dim == 3:
        assert r1[3] >= 256                      # the multi-block root apply
    assert np.array_equal(r1[0], r2[0])
    assert np.array_equal(r1[1], r2[1])
    (x1, i1), (x2, i2) = r1[2], r2[2]
    assert i1["converged"] and i1["iters"] == i2["iters"]
    assert np.array_equal(x1, x2)
    r0 = _run(dim, n, a, b, eps, precision, False, x, solve=False)
    err = np.abs(r1[0] - r0[0]).max() / np.abs(r0[0]).max()
    print(f"{dim}D n={n} {precision}: deterministic vs atomic F^-1 x {err:.2e}")
    assert err <= (1e-13 if precision == "fp64" else 1e-3)


def test_deterministic_matches_oracle(hiflib):
    from paper_1307_2895_gb300 import hif
    dim, n, eps = 2, 64, 1e-6
    a, b = inputs.high_contrast_coefficients(dim, n, seed=3, low=1e-3, high=1e3)
    A = stencil.assemble(dim, n, a, b)
    F = hifde.factor(A, dim, n, eps)
    x = inputs.rhs(dim, n, 3, seed=4)
    G = hif.factor(dim, n, a, b, eps, precision="fp64", deterministic=True)
    try:
        yi = G.apply(x, inverse=True)
        yf = G.apply(x, inverse=False)
    finally:
        G.free()
    for y, o in ((yi, F.apply_inverse(x)), (yf, F.apply(x))):
        assert np.abs(y - o).max() <= 1e-10 * np.abs(o).max()
