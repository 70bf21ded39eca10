"""hif_residual_norms_noalloc: the residual-norm entry point for callers that
cannot allocate device memory (e.g. code inside another library's allocator
callback, or code that must not let an allocation synchronize the device).

It must return the same squared residual norms as the existing entry points
(hif_matvec for A x, then the norms of f - A x), on two calls in a row (the
second call reuses the library's fixed scratch left by the first), and must
not change the device's free memory.  This file is collected last on purpose.
"""
import pytest

from paper_1307_2895_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_residual_norms_match_existing_entry_point(hiflib):
    import torch
    from paper_1307_2895_gb300 import hif

    dim, n, nrhs = 2, 64, 5
    a_np, b_np = inputs.high_contrast_coefficients(dim, n, seed=4, low=1e-2, high=1e2)
    dev = torch.device("cuda", 0)
    a = torch.from_numpy(a_np).to(dev)
    b = torch.from_numpy(b_np).to(dev)
    f = torch.from_numpy(inputs.rhs(dim, n, nrhs, seed=1)).to(dev)
    x = torch.from_numpy(inputs.rhs(dim, n, nrhs, seed=2)).to(dev) * 1e-3

    G = hif.factor(dim, n, a, b, 1e-6)
    try:
        ax = G.matvec(x)                       # existing entry point: y = A x
    finally:
        G.free()
    ref = ((f - ax) ** 2).sum(dim=0)

    out = torch.zeros(nrhs, dtype=torch.float64, device=dev)
    hif.residual_norms_noalloc(dim, n, a, b, f, x, out)
    torch.cuda.synchronize()
    first = out.clone()
    free_before = torch.cuda.mem_get_info(dev)[0]
    out.fill_(-1.0)
    hif.residual_norms_noalloc(dim, n, a, b, f, x, out)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info(dev)[0]
    second = out.clone()

    rel1 = ((first - ref).abs() / ref).max().item()
    rel2 = ((second - ref).abs() / ref).max().item()
    assert rel1 <= 1e-12, rel1
    assert rel2 <= 1e-12, rel2
    assert free_after == free_before


def test_noalloc_rejects_sizes_beyond_its_scratch(hiflib):
    import torch
    from paper_1307_2895_gb300 import hif

    dim, n = 2, 16
    a_np, b_np = inputs.constant_coefficients(dim, n)
    dev = torch.device("cuda", 0)
    a = torch.from_numpy(a_np).to(dev)
    b = torch.from_numpy(b_np).to(dev)
    f = torch.zeros((n - 1) ** 2, 17, dtype=torch.float64, device=dev)
    out = torch.zeros(17, dtype=torch.float64, device=dev)
    with pytest.raises(hif.HifError) as e:
        hif.residual_norms_noalloc(dim, n, a, b, f, f, out)
    assert e.value.code == hif.HIF_ERR_ARG and "16" in str(e.value)
