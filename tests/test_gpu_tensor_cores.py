"""Tensor-core (tcgen05, TF32) products of the FP32 elimination against the oracle.

hif_schur_update_f32 computes U - G G^T on FP32 blocks.  The expected value
is the oracle's Lemma 2.1 elimination (``oracle.hifde.eliminate``) of p from
a random SPD matrix [[A_pp, A_pq], [A_qp, A_qq]]: B_qq = A_qq - A_qp A_pp^-1
A_pq.  The test forms G = A_qp L^-T (L L^T = A_pp) in FP64 and rounds G and
A_qq to FP32.

Error bound, elementwise, with S = |G||G|^T.  Each operand value is split
into TF32 parts by repeated round-to-nearest.
  * split = 3: x = x0 + x1 + x2 exactly.  The six products kept are exact
    in FP32; the three dropped ones are below 2^-33 |x||y| together.  FP32
    accumulation over k terms adds at most one ulp per addition, i.e.
    (k + 2) 2^-23 S with the input rounding of G.  Rounding A_qq adds
    2^-24 |A_qq|.  The test allows twice that sum, and requires the split-3
    error to be 16x below the plain-TF32 error on the same inputs.
  * split = 2: the second part enters the MMA with its TF32 rounding,
    2^-21 |x| per operand, hence 2 2^-21 S per product.
  * split = 1 (plain TF32): 2^-10 relative per operand, hence 2 2^-10 S per
    product, plus the same accumulation and input terms.

A dropped remainder term, a wrong swizzle or a transposed operand each
breaks the split-3 bound by a wide margin.  Sizes span several 128 x 64
output blocks with ragged tails in both dimensions and in k.

End to end, the mixed-precision multifrontal factorization (eps = 0) through
the tiled path with the tensor cores solves as accurately as the same path
with FP32 on the SIMT pipes, and with skeletonization PCG reaches 1e-12.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs

pytestmark = pytest.mark.gpu

U24 = 2.0 ** -24


def _oracle_schur(m, k, seed):
    """Random SPD [[A_pp, A_pq], [A_qp, A_qq]] (|p| = k, |q| = m); the oracle's
    Lemma 2.1 elimination of p gives B_qq."""
    rng = np.random.default_rng(seed)
    n = k + m
    X = rng.standard_normal((n, n + 8))
    A = X @ X.T / (n + 8) + 0.5 * np.eye(n)
    act = hifde.ActiveMatrix(sp.csr_matrix(A))
    p = list(range(k))
    rec = hifde.eliminate(act, p)
    q = rec.q.tolist()
    assert q == list(range(k, n))
    Bqq = act.block(q, q)
    Aqq = A[k:, k:]
    G = np.linalg.solve(rec.L, rec.Aqp.T).T          # A_qp L^-T
    return G, Aqq, Bqq


@pytest.mark.parametrize("m,k", [(1, 1), (64, 32), (100, 33), (200, 7), (257, 300), (130, 64)])
@pytest.mark.parametrize("split", [3, 2, 1])
def test_schur_update_matches_oracle(hiflib, m, k, split):
    import torch
    from paper_1307_2895_gb300 import hif
    nb = 3
    Gs, Aqqs, Bqqs = zip(*[_oracle_schur(m, k, seed=100 * m + k + b) for b in range(nb)])
    G = torch.tensor(np.stack(Gs), dtype=torch.float32, device="cuda").contiguous()
    U = torch.tensor(np.stack(Aqqs), dtype=torch.float32, device="cuda").contiguous()
    U0 = U.clone()
    hif.schur_update(G, U, split=split)
    got = U.double().cpu().numpy()
    for b in range(nb):
        S = np.abs(Gs[b]) @ np.abs(Gs[b]).T
        per_product = {3: 3 * 2.0 ** -33, 2: 2 * 2.0 ** -21, 1: 2 * 2.0 ** -10}[split]
        # accumulation: one FP32 ulp per addition (tensor-core adders may truncate)
        bound = 2 * ((per_product + (k + 2) * 2 * U24) * S + U24 * np.abs(Aqqs[b]))
        err = np.abs(got[b] - Bqqs[b])
        assert (err <= bound).all(), (b, float((err / bound).max()))
    if split == 3 and m * k >= 1000:
        # the remainder products are there: far below the plain-TF32 error
        hif.schur_update(G, U0, split=1)
        e1 = max(np.abs(U0[b].double().cpu().numpy() - Bqqs[b]).max() for b in range(nb))
        e3 = max(np.abs(got[b] - Bqqs[b]).max() for b in range(nb))
        assert 16 * e3 < e1, (e3, e1)


def test_schur_update_empty_and_args(hiflib):
    import torch
    from paper_1307_2895_gb300 import hif
    G = torch.zeros((2, 0, 5), dtype=torch.float32, device="cuda")
    U = torch.zeros((2, 0, 0), dtype=torch.float32, device="cuda")
    hif.schur_update(G, U)                       # m = 0: nothing to do
    G = torch.zeros((1, 3, 0), dtype=torch.float32, device="cuda")
    U = torch.ones((1, 3, 3), dtype=torch.float32, device="cuda")
    hif.schur_update(G, U)                       # k = 0: U unchanged
    assert (U == 1).all()
    with pytest.raises(hif.HifError):
        hif.schur_update(torch.zeros((1, 4, 4), dtype=torch.float32, device="cuda"),
                         torch.zeros((1, 4, 4), dtype=torch.float32, device="cuda"), split=4)


def _contrast(dim, n):
    return inputs.high_contrast_coefficients(dim, n, seed=11, low=1e-2, high=1e2)


@pytest.mark.parametrize("dim,n,field", [(3, 12, "lap"), (3, 16, "contrast"), (2, 64, "contrast")])
def test_mixed_tiled_tensor_cores_vs_simt(hiflib, dim, n, field):
    """MF (eps = 0: no skeletonization, F = A up to arithmetic) in mixed
    precision with every cell through the tiled elimination: F^-1 f from the
    tensor-core products (three-part split) is as close to the dense solve as
    from the SIMT FP32 products."""
    from paper_1307_2895_gb300 import hif
    a, b = _contrast(dim, n) if field == "contrast" else inputs.constant_coefficients(dim, n)
    A = stencil.assemble(dim, n, a, b)
    f = inputs.rhs(dim, n, 2, seed=5)
    xd = np.linalg.solve(A.toarray(), f)
    errs = {}
    for tc in (0, -1):
        G = hif.factor(dim, n, a, b, 0.0, variant="mf", precision="mixed", big_cell=1, tensor_cores=tc)
        try:
            y = G.apply(f)
        finally:
            G.free()
        errs[tc] = np.linalg.norm(y - xd) / np.linalg.norm(xd)
    assert errs[0] <= 2 * errs[-1] + 1e-7, errs


@pytest.mark.parametrize("tc", [0, 2])
def test_mixed_tensor_cores_pcg(hiflib, tc):
    """3D 31^3 contrast 1e4 in mixed precision with the large cells and the
    redundant blocks of the large fronts on the tensor cores (three- and
    two-part TF32 splits): PCG reaches 1e-12, re-checked in extended
    precision."""
    from paper_1307_2895_gb300 import hif
    dim, n, eps = 3, 32, 1e-6
    a, b = _contrast(dim, n)
    f = inputs.rhs(dim, n, 2)
    G = hif.factor(dim, n, a, b, eps, precision="mixed", big_cell=128, tensor_cores=tc)
    try:
        xh, xl, info = G.solve(f, tol=1e-12, maxit=200, want_lo=True)
    finally:
        G.free()
    assert info["converged"] and info["relres_max"] <= 1e-12
    assert stencil.residual_ext(dim, n, a, b, f, xh, xl).max() <= 2e-12
