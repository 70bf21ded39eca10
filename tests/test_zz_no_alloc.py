"""hif_residual_norms_noalloc: the residual-norm entry point for callers that
cannot allocate device memory (e.g. code inside another library's allocator
callback, or code that must not let an allocation synchronize the device).

It must return the squared residual norms ||f_r - A x_r||^2 of the stencil
operator: checked against the oracle's assembled A (A x on the CPU) and
against the existing entry point hif_matvec, on two calls in a row (the
second call reuses the library's fixed scratch left by the first), without
changing the device's free memory.  2D and 3D (the 3D bond indices are their
own formulas), and the full 16-column width of the scratch.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from oracle import stencil
from paper_1307_2895_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,n,nrhs", [(2, 64, 5), (3, 16, 16)])
def test_noalloc_residual_norms_match_oracle_and_existing_entry_point(hiflib, dim, n, nrhs):
    import torch
    from paper_1307_2895_gb300 import hif

    a_np, b_np = inputs.high_contrast_coefficients(dim, n, seed=4, low=1e-2, high=1e2)
    f_np = inputs.rhs(dim, n, nrhs, seed=1)
    x_np = inputs.rhs(dim, n, nrhs, seed=2) * 1e-3
    A = stencil.assemble(dim, n, a_np, b_np)
    ref = ((f_np - A @ x_np) ** 2).sum(axis=0)          # oracle: assembled A on the CPU

    dev = torch.device("cuda", 0)
    a = torch.from_numpy(a_np).to(dev)
    b = torch.from_numpy(b_np).to(dev)
    f = torch.from_numpy(f_np).to(dev)
    x = torch.from_numpy(x_np).to(dev)

    G = hif.factor(dim, n, a, b, 1e-6)
    try:
        ax = G.matvec(x)                       # existing entry point: y = A x
    finally:
        G.free()
    ref_entry = ((f - ax) ** 2).sum(dim=0).cpu().numpy()

    out = torch.zeros(nrhs, dtype=torch.float64, device=dev)
    hif.residual_norms_noalloc(dim, n, a, b, f, x, out)
    torch.cuda.synchronize()
    first = out.cpu().numpy()
    free_before = torch.cuda.mem_get_info(dev)[0]
    out.fill_(-1.0)
    hif.residual_norms_noalloc(dim, n, a, b, f, x, out)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info(dev)[0]
    second = out.cpu().numpy()

    for got in (first, second):
        assert np.max(np.abs(got - ref) / ref) <= 1e-12
        assert np.max(np.abs(got - ref_entry) / ref_entry) <= 1e-12
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


def test_noalloc_refuses_host_memory_on_the_gpu(hiflib):
    """A host array reaching the C entry point is an argument error there, not
    a device fault (the binding's own checks are bypassed on purpose)."""
    import torch
    from paper_1307_2895_gb300 import hif

    dim, n = 2, 16
    a_np, b_np = inputs.constant_coefficients(dim, n)
    dev = torch.device("cuda", 0)
    a = torch.from_numpy(a_np).to(dev)
    b = torch.from_numpy(b_np).to(dev)
    f = torch.zeros((n - 1) ** 2, 2, dtype=torch.float64, device=dev)
    out_host = np.zeros(2)
    lib = hif.load()
    rc = lib.hif_residual_norms_noalloc(dim, n, a.data_ptr(), b.data_ptr(), f.data_ptr(), f.data_ptr(), 2, 2,
                                        out_host.ctypes.data, None)
    assert rc == hif.HIF_ERR_ARG and b"rnorm2" in lib.hif_last_error()
