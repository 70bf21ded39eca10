"""The host symbolic stage of HIF-DE in 3D with edge skeletonization
(csrc/symbolic3x.cpp, Section 4.5) against the oracle's factorization
(oracle.hifde.factor3x), on the CPU.

A small harness (tests/host/symbolic3x_check.cpp, compiled here with g++)
builds every level's algebraic cells, face groups and edge groups from the
clique pattern of A_l, skeletonizing each group with the skeleton the
oracle's ID chose for it.  Its index sets must equal the oracle's, which
follows the stored entries of the numerical A_l:

* per level, the peeled cells (the oracle's eliminated sets p, in order) and
  their neighbours q = p^N at elimination (Lemma 2.1);
* the face groups, then the edge groups (the oracle's front sets c, in key
  order), and the neighbour set c^N of each, whose block A_{c^N, c} the ID
  compresses (recorded from the oracle's own neighbour queries);
* the DOFs left for the root (s_L).

The cases: 15^3 with edges from level 0 (one level) at two tolerances;
31^3 with edges from level 1 (two levels); 31^3 with a high-contrast field
and edges from level 0.  Only the last one makes the pattern decide
anything: with edges from level 1 on a uniform grid, every group lies in
the neighbour clique of an adjacent cell and no DOF of a level-1 cell is
coupled to another cell, while with level-0 edges the fill-in of the edge
skeletons couples level-1 cells, so the peel removes DOFs (asserted) and a
dropped skeleton clique or a skipped peel changes the groups.  A skeleton
that is not in its group is rejected without changing the pattern.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import hifde, stencil
from paper_1307_2895_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1307_2895_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("symbolic3x") / "symbolic3x_check")
    cmd = [gxx, "-std=c++17", "-O2", "-pthread", "-I", CSRC, os.path.join(ROOT, "tests", "host", "symbolic3x_check.cpp"),
           os.path.join(CSRC, "symbolic3x.cpp"), os.path.join(CSRC, "host_pool.cpp"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    return exe


def _skeletons(F, edge_start):
    """int32 stream of the oracle's skeletons, per level: faces, then edges."""
    out = []
    for k, lev in enumerate(F.levels):
        ell, is_edges = k // 2, k % 2 == 1
        if is_edges and ell < edge_start:
            assert not lev.fronts
            continue
        out.append(len(lev.fronts))
        for fr in lev.fronts:
            out.append(len(fr.sk))
            out.extend(sorted(fr.sk.tolist()))
    return np.asarray(out, dtype=np.int32)


def _run(harness, tmp_path, n, edge_start, skel):
    s = str(tmp_path / "skel.bin")
    o = str(tmp_path / "out.bin")
    skel.tofile(s)
    rc = subprocess.run([harness, str(n), "8", str(edge_start), s, o]).returncode
    v = np.fromfile(o, dtype=np.int32)
    return rc, v


def _parse(v, L, edge_start):
    k = 0

    def take(m):
        nonlocal k
        r = v[k:k + m]
        k += m
        return r

    def lst():
        return take(int(take(1)[0])).tolist()

    levels = []
    for ell in range(L):
        cells = []
        for _ in range(int(take(1)[0])):
            p = lst()
            cells.append((p, lst()))
        faces = [(lst(), lst()) for _ in range(int(take(1)[0]))]
        edges = [(lst(), lst()) for _ in range(int(take(1)[0]))] if ell >= edge_start else []
        levels.append((cells, faces, edges))
    root = lst()
    assert k == v.size
    return levels, root


def _compare(F, levels, root, queried):
    for ell, (cells, faces, edges) in enumerate(levels):
        lc, le = F.levels[2 * ell], F.levels[2 * ell + 1]
        assert len(cells) == len(lc.cells), f"level {ell}: cell count"
        for (p, q), rec in zip(cells, lc.cells):
            assert p == rec.p.tolist(), f"level {ell}: cell differs"
            assert q == rec.q.tolist(), f"level {ell}: neighbours differ"
        for kind, groups, lev in (("face", faces, lc), ("edge", edges, le)):
            assert [fr.c.tolist() for fr in lev.fronts] == [c for c, _ in groups], f"level {ell}: {kind} groups differ"
            for c, N in groups:
                assert queried[tuple(c)] == N, f"level {ell}: {kind} group neighbours differ"
    assert root == F.root.tolist()


def _recording_neighbors(monkeypatch):
    """Wrap the oracle's neighbour query to keep c -> c^N of every call."""
    seen = {}
    orig = hifde.ActiveMatrix.neighbors

    def rec(self, c):
        out = orig(self, c)
        seen[tuple(int(v) for v in c)] = list(out)
        return out

    monkeypatch.setattr(hifde.ActiveMatrix, "neighbors", rec)
    return seen


def _case(harness, tmp_path, monkeypatch, A, n, eps, edge_start):
    queried = _recording_neighbors(monkeypatch)
    F = hifde.factor3x(A, n, eps, edge_start=edge_start)
    rc, v = _run(harness, tmp_path, n, edge_start, _skeletons(F, edge_start))
    assert rc == 0
    levels, root = _parse(v, F.L, edge_start)
    _compare(F, levels, root, queried)
    return F


@pytest.mark.parametrize("eps", [1e-3, 1e-9])
def test_one_level_edges_from_level0(harness, tmp_path, monkeypatch, eps):
    n = 16
    a, b = inputs.constant_coefficients(3, n)
    _case(harness, tmp_path, monkeypatch, stencil.assemble(3, n, a, b), n, eps, 0)


def test_two_levels_edges_from_level1(harness, tmp_path, monkeypatch):
    n = 32
    a, b = inputs.constant_coefficients(3, n)
    F = _case(harness, tmp_path, monkeypatch, stencil.assemble(3, n, a, b), n, 1e-3, 1)
    assert F.L == 2 and len(F.levels[3].fronts) > 0


def test_high_contrast_two_levels(harness, tmp_path, monkeypatch):
    n = 32
    a, b = inputs.high_contrast_coefficients(3, n, seed=5, low=1e-2, high=1e2)
    F = _case(harness, tmp_path, monkeypatch, stencil.assemble(3, n, a, b), n, 1e-6, 0)
    # level 1 (S = 16): the Voronoi members are the DOFs active at its start
    # with no coordinate on the plane 16; the peel removed some of them
    act1 = F.root.tolist()
    for lev in F.levels[2:]:
        act1 += [g for rec in lev.cells for g in rec.p.tolist()]
        act1 += [g for fr in lev.fronts for g in fr.rd.tolist()]
    X = stencil.coords(3, n)[np.asarray(act1)]
    members = int((X != 16).all(axis=1).sum())
    kept = sum(len(rec.p) for rec in F.levels[2].cells)
    assert members - kept > 0


def test_rejects_foreign_skeleton(harness, tmp_path):
    n = 16
    a, b = inputs.constant_coefficients(3, n)
    F = hifde.factor3x(stencil.assemble(3, n, a, b), n, 1e-3, edge_start=0)
    skel = _skeletons(F, 0).copy()
    # the first face group's first skeleton DOF replaced by a DOF of no group:
    # one that a level-0 cell eliminated
    gone = int(F.levels[0].cells[0].p[0])
    assert skel[0] > 0 and skel[1] > 0
    skel[2] = gone
    rc, _ = _run(harness, tmp_path, n, 0, skel)
    assert rc == 4


@pytest.mark.parametrize("n", [4, 5, 10])
def test_smallest_and_ragged_grids(harness, tmp_path, monkeypatch, n):
    """One-level trees: n = 4 (cells of one DOF), and n = 5 and 10, which are
    not 2^L m (the last cells and groups are cut short), with edges from
    level 0."""
    a, b = inputs.high_contrast_coefficients(3, n, seed=5, low=1e-2, high=1e2)
    _case(harness, tmp_path, monkeypatch, stencil.assemble(3, n, a, b), n, 1e-6, 0)
