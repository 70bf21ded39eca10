"""Flexible GMRES (hif_set_solver) through the C ABI.

* GMRES alone reaches 1e-12 (double-double refinement as for CG) on 2D and
  3D workloads, with restart lengths 50 and 5 (the restart path: D += Z y
  and a new cycle from the true residual), re-checked in extended precision.
* Parity with the oracle's fgmres: in the FP64 mode (F^-1 equal to the
  oracle's to 1e-10) the number of Arnoldi steps to a relative residual of
  1e-9 is the oracle's, within one step.
* AUTO: CG on an SPD preconditioner never hands over; where CG breaks down
  (the FP32 factorization of the contrast-1e6 workload, whose clamped pivots
  make F^-1 a poor preconditioner: CG stalls) the step is handed to GMRES.
  GMRES does not converge there either: the hand-over is what is tested.
"""
import numpy as np
import pytest

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs

pytestmark = pytest.mark.gpu


def _contrast(dim, n):
    return inputs.high_contrast_coefficients(dim, n, seed=11, low=1e-2, high=1e2)


@pytest.mark.parametrize("dim,n,restart,precision", [(2, 64, 50, "fp64"), (2, 64, 5, "fp32_apply"),
                                                     (3, 16, 50, "fp32_apply"), (2, 128, 20, "mixed")])
def test_gmres_reaches_1e12(hiflib, dim, n, restart, precision):
    from paper_1307_2895_gb300 import hif
    a, b = _contrast(dim, n)
    f = inputs.rhs(dim, n, 3, seed=1)
    G = hif.factor(dim, n, a, b, 1e-6, precision=precision)
    try:
        G.set_solver("gmres", restart)
        xh, xl, info = G.solve(f, tol=1e-12, maxit=400, want_lo=True)
        G.set_solver("cg")
        _, info_cg = G.solve(f, tol=1e-12, maxit=400)
    finally:
        G.free()
    assert info["converged"] and info["relres_max"] <= 1e-12
    assert info["gmres_iters"] == info["iters"] > 0
    assert info_cg["gmres_iters"] == 0 and info_cg["converged"]
    assert stencil.residual_ext(dim, n, a, b, f, xh, xl).max() <= 2e-12
    if restart >= 50:
        # minimal residual over the same Krylov space: not more steps than CG
        assert info["iters"] <= info_cg["iters"] + 2


@pytest.mark.parametrize("dim,n,eps", [(2, 32, 1e-6), (2, 64, 1e-4), (3, 12, 1e-6)])
def test_gmres_steps_match_oracle(hiflib, dim, n, eps):
    from paper_1307_2895_gb300 import hif
    a, b = _contrast(dim, n)
    A = stencil.assemble(dim, n, a, b)
    F = hifde.factor(A, dim, n, eps)
    f = inputs.rhs(dim, n, 2, seed=3)
    _, it_o, rel_o = hifde.fgmres(A, F.apply_inverse, f, tol=1e-9, restart=50)
    G = hif.factor(dim, n, a, b, eps, precision="fp64")
    try:
        G.set_solver("gmres", 50)
        for c in range(2):
            _, info = G.solve(np.ascontiguousarray(f[:, c]), tol=1e-9, maxit=200)
            assert info["converged"]
            assert abs(info["iters"] - it_o[c]) <= 1, (info["iters"], it_o[c])
    finally:
        G.free()


def test_auto_keeps_cg_on_spd_preconditioner(hiflib):
    from paper_1307_2895_gb300 import hif
    a, b = _contrast(2, 64)
    f = inputs.rhs(2, 64, 2, seed=1)
    G = hif.factor(2, 64, a, b, 1e-6, precision="fp32_apply")
    try:
        _, info = G.solve(f, tol=1e-12)
    finally:
        G.free()
    assert info["converged"] and info["gmres_iters"] == 0


def test_auto_hands_over_on_breakdown(hiflib):
    from paper_1307_2895_gb300 import hif
    w = inputs.workload("contrast2d_n512")
    f = inputs.rhs(2, 512, 2, seed=0)
    G = hif.factor(2, 512, w["a_stag"], w["b"], w["eps"], precision="mixed")
    try:
        assert G.stats()["clamped_pivots"] > 0
        G.set_solver("cg")
        _, cg = G.solve(f, tol=1e-12, maxit=120)
        G.set_solver("auto")
        _, auto = G.solve(f, tol=1e-12, maxit=120)
    finally:
        G.free()
    assert not cg["converged"] and cg["gmres_iters"] == 0 and cg["iters"] == 120
    assert 0 < auto["gmres_iters"] < auto["iters"] == 120


def test_set_solver_arguments(hiflib):
    from paper_1307_2895_gb300 import hif
    a, b = _contrast(2, 16)
    G = hif.factor(2, 16, a, b, 1e-6)
    try:
        with pytest.raises(hif.HifError):
            G.set_solver("gmres", 1)
        with pytest.raises(hif.HifError):
            G.set_solver("gmres", 501)
        G.set_solver("auto", 0)
    finally:
        G.free()
