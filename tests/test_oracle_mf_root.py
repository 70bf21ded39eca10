"""The size of MF's top separator (Algorithm 3.1) against the paper's mf2 /
mf3 columns (tests/golden/paper_mf_root_sizes.txt), on the CPU.

The root of nested dissection on an (n-1)^dim grid is the last level's cross
of separators: two lines of n-1 DOFs sharing one in 2D, 2(n-1) - 1; three
planes of (n-1)^2 DOFs in 3D, pairwise sharing a line of n-1 and all three
one point, 3(n-1)^2 - 3(n-1) + 1 by inclusion-exclusion.  Both closed forms
reproduce every size the paper prints; the oracle reproduces them at 63^2
and 127^2 and the paper's own 31^3 case.
"""
import os

import pytest

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_mf_root_sizes.txt")


def _closed_form(dim, n):
    m = n - 1
    return 2 * m - 1 if dim == 2 else 3 * m * m - 3 * m + 1


def _rows():
    with open(GOLDEN) as fh:
        return [tuple(int(v) for v in ln.split()) for ln in fh if ln.strip() and not ln.startswith("#")]


def test_closed_form_matches_paper():
    rows = _rows()
    assert len(rows) == 5
    for dim, n, sL in rows:
        assert _closed_form(dim, n) == sL, (dim, n, sL)


@pytest.mark.parametrize("dim,n", [(2, 64), (2, 128), (3, 32)])
def test_oracle_mf_root(dim, n):
    a, b = inputs.constant_coefficients(dim, n)
    F = hifde.factor(stencil.assemble(dim, n, a, b), dim, n, 0.0)
    assert len(F.root) == _closed_form(dim, n)
    if (dim, n) == (3, 32):
        assert (3, 32, len(F.root)) in _rows()          # the paper's 31^3 value itself
