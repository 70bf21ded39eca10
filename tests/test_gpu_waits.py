"""Failure detection of the bounded device waits, without a fault: each wait
runs on an object that nothing completes (a bulk-copy phase whose bytes never
come, a group barrier whose partner block never arrives, a tensor-core
barrier on which no MMA commits), with a short bound.  It must give up,
report HIF_ERR_TIMEOUT with its own message through the same status bits as
in the factorization and the sweeps, and leave the context usable: a
factorization and F^-1 x right after it still match the oracle.
"""
import numpy as np
import pytest

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which,limit,words", [
    ("bulk", 1 << 12, "bulk copy"),
    ("group", 1 << 10, "group-barrier"),
    ("mma", 1_000_000, "tensor-core MMAs"),      # 1 ms of the global timer
])
def test_bounded_wait_gives_up_and_reports(hiflib, which, limit, words):
    from paper_1307_2895_gb300 import hif
    with pytest.raises(hif.HifError) as e:
        hif.wait_selftest(which, limit)
    assert e.value.code == hif.HIF_ERR_TIMEOUT
    assert words in str(e.value)
    dim, n, eps = 2, 32, 1e-6
    a, b = inputs.constant_coefficients(dim, n)
    x = inputs.rhs(dim, n, 2, seed=3)
    G = hif.factor(dim, n, a, b, eps, precision="fp64")
    try:
        y = G.apply(x)
    finally:
        G.free()
    o = hifde.factor(stencil.assemble(dim, n, a, b), dim, n, eps).apply_inverse(x)
    assert np.linalg.norm(y - o) <= 1e-10 * np.linalg.norm(o)
