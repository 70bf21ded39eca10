"""The sweep autotuner: a solve with autotuning records one choice per
launch shape it met, every choice is one of the candidates, and the solution
is that of the built-in shapes (each output element is computed by one
thread whatever the block size; the shared boundary rows are summed with
atomics, so agreement is to rounding)."""
import numpy as np
import pytest

from paper_1307_2895_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_autotune_records_choices_and_keeps_results(hiflib):
    from paper_1307_2895_gb300 import hif
    a, b = inputs.high_contrast_coefficients(2, 128, seed=11, low=1e-2, high=1e2)
    f = inputs.rhs(2, 128, 4, seed=2)
    ys = {}
    for tune in (False, True):
        G = hif.factor(2, 128, a, b, 1e-6, precision="fp32_apply", autotune=tune)
        try:
            ys[tune] = G.apply(f, inverse=True)
            _, info = G.solve(f, tol=1e-12)
            assert info["converged"]
        finally:
            G.free()
    tab = hif.autotune_table()
    mine = tab[(tab[:, 1] == 4) & (tab[:, 2] == 4)]
    assert len(mine) >= 8              # up and down launches of the levels seen
    assert set(mine[:, 7]) <= {0, 64, 128, 256, 512}
    assert set(mine[:, 8]) <= {-1, 0}
    assert np.linalg.norm(ys[True] - ys[False]) <= 1e-5 * np.linalg.norm(ys[False])
