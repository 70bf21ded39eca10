"""The host tree and block-index builder (geometry.cpp, on the host thread
pool) against the definitions of Sections 3.1, 4.1 and 4.3, on the CPU.

A small harness (tests/host/builder_check.cpp, compiled here with g++)
runs build_cells / build_fronts / build_child_map on a given alive set.  The
references below are computed independently in numpy, with the separator
positions of the oracle (oracle.hifde.level_separators):

* cell interiors I: alive DOFs with no coordinate on a level separator,
  grouped by the interval of each coordinate (x fastest cell index);
* cell boundaries B: alive DOFs with a separator coordinate, in every cell
  whose closed box contains them;
* fronts: after the interiors leave, alive DOFs with exactly one separator
  coordinate, grouped by that separator and the intervals of the others;
  N = (B of the two adjacent cells) minus c, and pos1 / pos2 = positions of
  [c ; N] in those two boundaries;
* child maps: position of each DOF of a level-l cell in the boundary of
  each of its 2^dim children at level l - 1.

The grids (511^2, 63^3) are large enough for the builders' parallel paths;
n = 40 and 3D n = 24 have rounded separators; n = 4 (cells of one DOF) and
2D n = 5 are the smallest trees (one level).  Level 1 starts from an alive set with the
level-0 interiors and a pseudo-random 30% of the front DOFs removed, as
skeletonization removes redundant DOFs.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import hifde, stencil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1307_2895_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("builder") / "builder_check")
    cmd = [gxx, "-std=c++17", "-O2", "-pthread", "-I", CSRC, os.path.join(ROOT, "tests", "host", "builder_check.cpp"),
           os.path.join(CSRC, "geometry.cpp"), os.path.join(CSRC, "host_pool.cpp"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    return exe


def _write_ids(path, ids):
    arr = np.asarray(ids, dtype=np.int32)
    with open(path, "wb") as f:
        np.array([arr.size], dtype=np.int32).tofile(f)
        arr.tofile(f)


def _run(harness, tmp_path, dim, n, level, alive, prev_alive=None):
    a = str(tmp_path / "alive.bin")
    o = str(tmp_path / "out.bin")
    _write_ids(a, alive)
    args = [harness, str(dim), str(n), str(level), a, o]
    if prev_alive is not None:
        p = str(tmp_path / "prev.bin")
        _write_ids(p, prev_alive)
        args.append(p)
    subprocess.run(args, check=True)
    v = np.fromfile(o, dtype=np.int32)
    k = 0

    def take(m):
        nonlocal k
        r = v[k:k + m]
        k += m
        return r

    def lst():
        m = int(take(1)[0])
        return take(m).tolist()

    cells = [(lst(), lst()) for _ in range(int(take(1)[0]))]
    fronts = []
    for _ in range(int(take(1)[0])):
        axis, p1, p2 = take(3).tolist()
        c, N = lst(), lst()
        fronts.append(dict(axis=axis, P1=p1, P2=p2, c=c, N=N, pos1=take(len(c) + len(N)).tolist(),
                           pos2=take(len(c) + len(N)).tolist()))
    maps = []
    if prev_alive is not None:
        for I, B in cells:
            child = take(8).tolist()
            maps.append((child, take(8 * (len(I) + len(B))).reshape(-1, 8)))
    assert k == v.size
    return cells, fronts, maps


def _reference(dim, n, level, alive):
    L = hifde.tree_levels(n, 8)
    seps = hifde.level_separators(n, L, level)
    nc = len(seps) + 1
    X = stencil.coords(dim, n)[alive]
    on = np.isin(X, seps)
    iv = np.searchsorted(seps, X)                 # interval (interior) or ordinal (on a separator)
    ncells = nc ** dim
    I = [[] for _ in range(ncells)]
    B = [[] for _ in range(ncells)]
    for g, x_on, x_iv in zip(alive, on, iv):
        if not x_on.any():
            lin = 0
            for a in reversed(range(dim)):
                lin = lin * nc + int(x_iv[a])
            I[lin].append(int(g))
            continue
        choices = [(int(x_iv[a]), int(x_iv[a]) + 1) if x_on[a] else (int(x_iv[a]),) for a in range(dim)]
        for combo in np.array(np.meshgrid(*choices, indexing="ij")).reshape(dim, -1).T:
            lin = 0
            for a in reversed(range(dim)):
                lin = lin * nc + int(combo[a])
            B[lin].append(int(g))
    for c in range(ncells):
        B[c].sort()
    interior = {g for cell in I for g in cell}
    fronts = {}
    for g, x_on, x_iv in zip(alive, on, iv):
        if int(g) in interior or int(x_on.sum()) != 1:
            continue
        axis = int(np.nonzero(x_on)[0][0])
        cells = []
        for side in (0, 1):
            lin = 0
            for a in reversed(range(dim)):
                lin = lin * nc + (int(x_iv[a]) + side if a == axis else int(x_iv[a]))
            cells.append(lin)
        fronts.setdefault((axis, cells[0], cells[1]), []).append(int(g))
    return I, B, fronts


def _check(dim, n, level, alive, cells, fronts, ref):
    I, B, rfronts = ref
    assert len(cells) == len(I)
    for c, (ci, cb) in enumerate(cells):
        assert ci == I[c], f"cell {c}: interior differs"
        assert cb == B[c], f"cell {c}: boundary differs"
    assert len(fronts) == len(rfronts)
    for F in fronts:
        key = (F["axis"], F["P1"], F["P2"])
        assert F["c"] == rfronts[key], f"front {key}: DOFs differ"
        cs = set(F["c"])
        b1, b2 = B[F["P1"]], B[F["P2"]]
        assert F["N"] == sorted((set(b1) | set(b2)) - cs)
        p1 = {g: i for i, g in enumerate(b1)}
        p2 = {g: i for i, g in enumerate(b2)}
        allg = F["c"] + F["N"]
        assert F["pos1"] == [p1.get(g, -1) for g in allg]
        assert F["pos2"] == [p2.get(g, -1) for g in allg]


def _level1_alive(dim, n, cells0, fronts0, seed=7):
    """Level-0 interiors gone, and about 30% of every level-0 front."""
    N = (n - 1) ** dim
    dead = np.zeros(N, dtype=bool)
    for I, _ in cells0:
        dead[I] = True
    rng = np.random.default_rng(seed)
    for F in fronts0:
        c = np.asarray(F["c"])
        dead[c[rng.random(c.size) < 0.3]] = True
    return np.nonzero(~dead)[0].astype(np.int64)


@pytest.mark.parametrize("dim,n", [(2, 512), (3, 64), (2, 40), (3, 24), (2, 4), (3, 4), (2, 5)])
def test_builder_matches_definitions(harness, tmp_path, dim, n):
    alive0 = np.arange((n - 1) ** dim, dtype=np.int64)
    cells0, fronts0, _ = _run(harness, tmp_path, dim, n, 0, alive0)
    _check(dim, n, 0, alive0, cells0, fronts0, _reference(dim, n, 0, alive0))
    if hifde.tree_levels(n, 8) < 2:
        return                                   # one level: no level 1 to build
    alive1 = _level1_alive(dim, n, cells0, fronts0)
    cells1, fronts1, maps1 = _run(harness, tmp_path, dim, n, 1, alive1, prev_alive=alive0)
    _check(dim, n, 1, alive1, cells1, fronts1, _reference(dim, n, 1, alive1))
    # child maps: each DOF of a level-1 cell found in its children's level-0 boundaries
    for (I, B), (child, m) in zip(cells1, maps1):
        kids = [c for c in child if c >= 0]
        assert len(kids) == 2 ** dim
        pos = [{g: i for i, g in enumerate(cells0[k][1])} for k in kids]
        for row, g in zip(m, I + B):
            assert row[:2 ** dim].tolist() == [p.get(g, -1) for p in pos]
            assert (row[2 ** dim:] == -1).all()


@pytest.mark.parametrize("dim,n", [(2, 40), (3, 24)])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_builder_level1_other_removals(harness, tmp_path, dim, n, seed):
    """Level 1 after other pseudo-random removals of level-0 front DOFs, on
    the grids with rounded separators."""
    alive0 = np.arange((n - 1) ** dim, dtype=np.int64)
    cells0, fronts0, _ = _run(harness, tmp_path, dim, n, 0, alive0)
    alive1 = _level1_alive(dim, n, cells0, fronts0, seed=seed)
    cells1, fronts1, _ = _run(harness, tmp_path, dim, n, 1, alive1, prev_alive=alive0)
    _check(dim, n, 1, alive1, cells1, fronts1, _reference(dim, n, 1, alive1))
