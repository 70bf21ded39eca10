"""Full-size workloads on the GPU: properties that hold at any size.

* 3D 63^3 Laplacian (Example 4 shape), eps 1e-3 and 1e-6, 4 right-hand
  sides: |s_L| within 10% of the paper's hifde3 value (Table 7) and the
  F^-1-preconditioned CG reaches 1e-12 in about the paper's n_i (Table 8);
  the residual is re-checked on the host in extended precision with the
  stencil in bond form (``oracle.stencil.residual_ext``).
* 2D 511^2 contrast-1e6 workload in the launch configuration bench.py times
  (FP32 apply, 8 right-hand sides): 1e-12 reached and re-checked likewise.
* 3D 127^3 contrast-1e4 workload with the learned rank predictor sizing the
  randomized ID (trained on 31^3 rank logs of other fields): |s_L| within 15%
  of the paper's Example 5 value (Table 9, hifde3 at 127^3: 6679), 1e-12
  reached with 4 right-hand sides and re-checked likewise.
* The batched workload: 64 independent 2D problems (interior edges
  log-uniform in 127..1023, contrast 1e2 / 1e4 / 1e6, 32 right-hand sides
  each) factored and solved concurrently through hif_factor_batch /
  hif_solve_batch: every column reaches 1e-12; the three smallest problems
  are re-checked in extended precision.
"""
import os

import numpy as np
import pytest

from oracle import stencil
from paper_1307_2895_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                e, s, ea, ni = line.split()
                rows.append((float(e), int(s), float(ea), int(ni)))
    return rows


@pytest.mark.parametrize("row", [0, 1])
def test_laplace3d_63_matches_paper_table7(hiflib, row):
    from paper_1307_2895_gb300 import hif
    eps, sL, _, ni = _golden("paper_table7_example4_63.txt")[row]
    dim, n = 3, 64
    a, b = inputs.constant_coefficients(dim, n)
    f = inputs.rhs(dim, n, 4, seed=0)
    F = hif.factor(dim, n, a, b, eps, precision="fp64")
    try:
        st = F.stats()
        xh, xl, info = F.solve(f, tol=1e-12, maxit=100, want_lo=True)
    finally:
        F.free()
    assert abs(st["root_size"] - sL) <= 0.1 * sL, (st["root_size"], sL)
    assert st["near_threshold_fronts"] == 0
    assert info["converged"] and info["relres_max"] <= 1e-12
    assert info["iters"] <= ni + 4
    assert stencil.residual_ext(dim, n, a, b, f, xh, xl).max() <= 2e-12


def test_contrast2d_511_bench_configuration(hiflib):
    from paper_1307_2895_gb300 import hif
    w = inputs.workload("contrast2d_n512")
    f = inputs.rhs(2, 512, w["nrhs"], seed=0)
    F = hif.factor(2, 512, w["a_stag"], w["b"], w["eps"], precision="fp32_apply")
    try:
        xh, xl, info = F.solve(f, tol=1e-12, maxit=1000, want_lo=True)
        st = F.stats()
    finally:
        F.free()
    assert info["converged"] and info["relres_max"] <= 1e-12
    assert stencil.residual_ext(2, 512, w["a_stag"], w["b"], f, xh, xl).max() <= 2e-12
    assert st["clamped_pivots"] == 0


def test_contrast3d_127_learned(hiflib):
    import torch
    from paper_1307_2895_gb300 import hif
    H, NF = 64, 10
    rng = np.random.default_rng(7)
    p = np.zeros(hif.MLP_PARAMS, np.float32)
    p[:H * NF] = rng.standard_normal(H * NF) * np.sqrt(2 / NF)
    o = H * NF + H
    p[o:o + H * H] = rng.standard_normal(H * H) * np.sqrt(2 / H)
    o += H * H + H
    p[o:o + H] = rng.standard_normal(H) * np.sqrt(1 / H)
    Xs, ts = [], []
    for seed in (11, 12):
        a, b = inputs.high_contrast_coefficients(3, 32, seed=seed, low=1e-2, high=1e2)
        G = hif.factor(3, 32, a, b, 1e-6)
        try:
            f_, r_, _ = G.front_log()
        finally:
            G.free()
        Xs.append(f_)
        ts.append(np.log1p(r_.astype(np.float32)))
    params = torch.tensor(p, device="cuda")
    hif.mlp_train(torch.tensor(np.concatenate(Xs), device="cuda"), torch.tensor(np.concatenate(ts), device="cuda"),
                  params, steps=2000, batch=512, lr=2e-3, seed=1)
    w = inputs.workload("contrast3d_n128")
    f = inputs.rhs(3, 128, w["nrhs"], seed=0)
    F = hif.factor(3, 128, w["a_stag"], w["b"], w["eps"], precision="fp32_apply", id_mode="learned",
                   rank_model=params, seed=5)
    try:
        st = F.stats()
        xh, xl, info = F.solve(f, tol=1e-12, maxit=200, want_lo=True)
    finally:
        F.free()
    assert abs(st["root_size"] - 6679) <= 0.15 * 6679, st["root_size"]
    assert info["converged"] and info["relres_max"] <= 1e-12
    assert stencil.residual_ext(3, 128, w["a_stag"], w["b"], f, xh, xl).max() <= 2e-12


def test_batched_problems(hiflib):
    from paper_1307_2895_gb300 import hif
    probs = inputs.batched_problems(64, seed=0)
    facts = hif.factor_batch([(p["dim"], p["n"], p["a_stag"], p["b"]) for p in probs], 1e-6,
                             precision="fp32_apply", nthreads=8)
    try:
        rhs = [inputs.rhs(2, p["n"], p["nrhs"], seed=p["seed"]) for p in probs]
        res = hif.solve_batch(facts, rhs, tol=1e-12, maxit=2000, nthreads=8)
    finally:
        for F in facts:
            F.free()
    for p, (x, info) in zip(probs, res):
        assert info["converged"] and info["relres_max"] <= 1e-12, (p["n"], p["contrast"], info)
    order = sorted(range(len(probs)), key=lambda i: probs[i]["n"])[:3]
    for i in order:
        p = probs[i]
        r = stencil.residual_ext(2, p["n"], p["a_stag"], p["b"], rhs[i], res[i][0])
        # x_hi alone: within the FP64 floor of the problem (contrast up to 1e6)
        assert r.max() <= 1e-9
