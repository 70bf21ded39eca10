"""Rank-prediction MLP and randomized ID on the GPU, through the C ABI.

* ``hif_mlp_grad`` (FP32) against the oracle's FP64 forward/backward
  (``oracle.learned.MLP``), whose gradient is pinned by finite differences.
* ``hif_mlp_predict`` (BF16 weights, FP32 accumulation) against the oracle's
  forward on the same weights rounded to BF16.
* ``hif_mlp_train`` lowers the Huber loss on rank data logged from a
  pivoted-QR factorization.
* Factorizations with the randomized ID (model-free or learned sketch size)
  keep the solver's 1e-12 target; the learned sketch size takes fewer
  fallbacks than the model-free guess and less front time than pivoted QR.
"""
import numpy as np
import pytest

from oracle import learned
from paper_1307_2895_gb300 import inputs

pytestmark = pytest.mark.gpu

H, NF = 64, 10


def _init_params(seed):
    rng = np.random.default_rng(seed)
    p = np.zeros(H * NF + H + H * H + H + H + 1, np.float32)
    p[:H * NF] = rng.standard_normal(H * NF) * np.sqrt(2 / NF)
    o = H * NF + H
    p[o:o + H * H] = rng.standard_normal(H * H) * np.sqrt(2 / H)
    o += H * H + H
    p[o:o + H] = rng.standard_normal(H) * np.sqrt(1 / H)
    p[H * NF:H * NF + H] = rng.standard_normal(H) * 0.1
    return p


def _bf16_round(x):
    """Round-to-nearest-even FP32 -> BF16 (kept in FP32), from the bit layout."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def test_mlp_gradient_matches_oracle(hiflib):
    import torch
    from paper_1307_2895_gb300 import hif
    rng = np.random.default_rng(3)
    n = 333                      # several 64-sample blocks and a ragged tail
    p = _init_params(1)
    X = rng.standard_normal((n, NF)).astype(np.float32)
    t = (rng.standard_normal(n) * 2).astype(np.float32)
    loss, g = hif.mlp_grad(torch.tensor(X, device="cuda"), torch.tensor(t, device="cuda"),
                           torch.tensor(p, device="cuda"))
    oloss, og = learned.MLP.unpack(p.astype(np.float64), NF, H).loss_and_grad(X.astype(np.float64),
                                                                              t.astype(np.float64))
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss - oloss) <= 1e-5 * abs(oloss)
    # FP32 sums of ~n products: relative to the gradient's scale
    assert np.max(np.abs(g - og)) <= 1e-4 * np.max(np.abs(og))
    assert np.linalg.norm(g - og) <= 1e-5 * np.linalg.norm(og)


def test_mlp_predict_bf16_matches_oracle(hiflib):
    import torch
    from paper_1307_2895_gb300 import hif
    rng = np.random.default_rng(4)
    n = 257
    p = _init_params(2)
    X = rng.standard_normal((n, NF)).astype(np.float32)
    y = hif.mlp_predict(torch.tensor(X, device="cuda"), torch.tensor(p, device="cuda")).cpu().numpy()
    yo, _ = learned.MLP.unpack(_bf16_round(p).astype(np.float64), NF, H).forward(X.astype(np.float64))
    assert np.max(np.abs(y - yo)) <= 1e-4 * max(1.0, np.max(np.abs(yo)))


def test_mlp_train_reduces_loss(hiflib):
    import torch
    from paper_1307_2895_gb300 import hif
    rng = np.random.default_rng(5)
    n = 2000
    X = rng.standard_normal((n, NF)).astype(np.float32)
    t = np.log1p(np.abs(X[:, 0] * 3 + X[:, 1] ** 2)).astype(np.float32)
    params = torch.tensor(_init_params(3), device="cuda")
    Xd, td = torch.tensor(X, device="cuda"), torch.tensor(t, device="cuda")
    l0, _ = hif.mlp_grad(Xd, td, params)
    hist = hif.mlp_train(Xd, td, params, steps=1500, batch=256, lr=2e-3, seed=9)
    l1, _ = hif.mlp_grad(Xd, td, params)
    assert len(hist) == 1500 and np.all(np.isfinite(hist))
    assert l1 < 0.1 * l0


def _train_rank_model(dim, n, eps, seeds, lo, hi):
    import torch
    from paper_1307_2895_gb300 import hif
    Xs, ts = [], []
    for s in seeds:
        a, b = inputs.high_contrast_coefficients(dim, n, seed=s, low=lo, high=hi)
        F = hif.factor(dim, n, a, b, eps)
        try:
            f, r, _ = F.front_log()
        finally:
            F.free()
        Xs.append(f)
        ts.append(np.log1p(r.astype(np.float32)))
    X = torch.tensor(np.concatenate(Xs), device="cuda")
    t = torch.tensor(np.concatenate(ts), device="cuda")
    params = torch.tensor(_init_params(7), device="cuda")
    hist = hif.mlp_train(X, t, params, steps=3000, batch=512, lr=2e-3, seed=1)
    return params, hist


@pytest.mark.parametrize("mode", ["rand", "learned"])
def test_randomized_id_keeps_solver_target(hiflib, mode):
    from paper_1307_2895_gb300 import hif
    dim, n, eps = 2, 128, 1e-6
    a, b = inputs.high_contrast_coefficients(dim, n, seed=2, low=1e-3, high=1e3)
    kw = {}
    if mode == "learned":
        kw["rank_model"], _ = _train_rank_model(dim, n, eps, [3, 4], 1e-3, 1e3)
    F = hif.factor(dim, n, a, b, eps, id_mode=mode, seed=5, **kw)
    try:
        st = F.stats()
        x, info = F.solve(inputs.rhs(dim, n, 2, seed=7), tol=1e-12, maxit=300)
    finally:
        F.free()
    assert st["sketched_fronts"] > 0
    assert info["converged"] and info["relres_max"] <= 1e-12


def test_learned_rank_gain_over_model_free_sketch(hiflib):
    """What the trained network gains over the randomized ID without it: on a
    held-out coefficient field its rank estimate is closer to the pivoted-QR
    rank than the model-free guess ceil(|c|/2) (less than half the mean
    error), and the sketches it sizes fall back to pivoted QR no more often;
    both keep the 1e-12 solver target."""
    import torch
    from paper_1307_2895_gb300 import hif
    dim, n, eps, lo, hi = 2, 256, 1e-6, 1e-3, 1e3
    params, hist = _train_rank_model(dim, n, eps, [3, 4], lo, hi)
    assert hist[-50:].mean() < 0.25 * hist[:5].mean()
    a, b = inputs.high_contrast_coefficients(dim, n, seed=2, low=lo, high=hi)
    F = hif.factor(dim, n, a, b, eps)
    try:
        f, r, sz = F.front_log()
    finally:
        F.free()
    pred = hif.mlp_predict(torch.tensor(f, device="cuda"), params).cpu().numpy()
    k_mlp = np.maximum(np.ceil(np.expm1(np.clip(pred, 0, 12))), 1)
    k_free = np.maximum((sz + 1) // 2, 1)
    err_mlp, err_free = np.abs(k_mlp - r).mean(), np.abs(k_free - r).mean()
    assert err_mlp < 0.5 * err_free, (err_mlp, err_free)
    rhs = inputs.rhs(dim, n, 2, seed=7)
    res = {}
    for mode in ("rand", "learned"):
        kw = {"rank_model": params} if mode == "learned" else {}
        G = hif.factor(dim, n, a, b, eps, id_mode=mode, seed=5, **kw)
        try:
            st = G.stats()
            _, info = G.solve(rhs, tol=1e-12, maxit=300)
        finally:
            G.free()
        assert info["converged"] and info["relres_max"] <= 1e-12
        res[mode] = st
    assert res["learned"]["fallback_fronts"] <= res["rand"]["fallback_fronts"]
