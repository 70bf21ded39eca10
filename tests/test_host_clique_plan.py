"""The clique form of A_l for HIF-DE in 3D with edge skeletonization
(Section 4.5), driven by the host symbolic stage (csrc/symbolic3x.cpp),
against the oracle's factorization (oracle.hifde.factor3x), on the CPU.

A_l is held as a sum of dense matrices, one per live clique: at the start
one clique per interior stencil bond ([[w, -w], [-w, w]], w = a / h^2, on its
two nodes) and one per DOF (b plus its bonds to the boundary).  The symbolic
stage says which cliques each block is gathered from and which clique each
result goes to; a small numpy model of the matrices follows it:

* a cell p (Lemma 2.1): F = the sum of the cliques touching p, on [p; q]
  (each lies in p and q = p^N); the new clique on q holds
  F_qq - F_qp F_pp^-1 F_pq, and the absorbed cliques die;
* a group c (Lemma 2.4): the cliques touching c give A_{c^N, c} (the block
  the ID compresses) and A_cc, all groups of a fractional level before any is
  skeletonized; with the oracle's skeleton s and T, the new clique on s
  holds -B_sr B_rr^-1 B_rs, and r leaves every clique (its entries dropped);
* the root: the sum of the live cliques on s_L.

Every block is also gathered through the flat plan of its batch (all cells
of a level, all groups of a fractional level: Symbolic3x::gather_plan),
applied as a gather launch would apply it; the result must equal the direct
sum bit for bit.

Each gathered block must equal the oracle's at the same step (1e-9 of its
largest entry; the two sum the same terms in other orders): A_pp (as
L L^T) and A_qp of every cell, the ID block of every group (recorded from the
oracle's own calls), B_sr and B_rr (as L L^T), and the root matrix D.  Cases,
on a high-contrast field: 15^3 with edges from level 0 (one level); 23^3
(two levels) with edges from level 1, and from level 0, where the level-0
edge cliques make the peel remove 249 DOFs from level 1's cells; the
planted mistakes of the module's last test
(a cell gathered without one of its cliques, cliques that keep r after a
skeletonization) fail it.
"""
import ctypes
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
def capi(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    so = str(tmp_path_factory.mktemp("s3x") / "libs3x.so")
    cmd = [gxx, "-std=c++17", "-O2", "-shared", "-fPIC", "-pthread", "-I", CSRC,
           os.path.join(ROOT, "tests", "host", "symbolic3x_capi.cpp"), os.path.join(CSRC, "symbolic3x.cpp"),
           os.path.join(CSRC, "host_pool.cpp"), "-o", so]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(so)
    vp, i, ip = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)
    sig = {"s3x_new": ([i, i, i], vp), "s3x_free": ([vp], None), "s3x_levels": ([vp], i),
           "s3x_count": ([vp], i), "s3x_size": ([vp, i], i), "s3x_copy": ([vp, i, ip], None),
           "s3x_add_clique": ([vp, ip, i], i), "s3x_cells": ([vp, i], None), "s3x_groups": ([vp, i, i], None),
           "s3x_neighbors": ([vp, ip, i], None), "s3x_touching": ([vp, ip, i], None),
           "s3x_members": ([vp, i], None), "s3x_active": ([vp], None), "s3x_eliminate": ([vp, ip, i], i),
           "s3x_skeletonize": ([vp, ip, i, ip, i], i), "s3x_gather_plan": ([vp, i, ip, ip, ip, ip], i)}
    for name, (args, res) in sig.items():
        getattr(lib, name).argtypes = args
        getattr(lib, name).restype = res
    return lib


class Plan:
    """The symbolic stage through the C shim (explicit stencil: cliques only)."""

    def __init__(self, lib, n):
        self.lib = lib
        self.h = lib.s3x_new(n, 8, 0)

    def close(self):
        self.lib.s3x_free(self.h)

    @staticmethod
    def _arr(v):
        a = (ctypes.c_int * max(1, len(v)))(*[int(x) for x in v])
        return a, len(v)

    def _lists(self):
        out = []
        for k in range(self.lib.s3x_count(self.h)):
            m = self.lib.s3x_size(self.h, k)
            buf = (ctypes.c_int * max(1, m))()
            self.lib.s3x_copy(self.h, k, buf)
            out.append(list(buf[:m]))
        return out

    def add(self, members):
        return self.lib.s3x_add_clique(self.h, *self._arr(members))

    def cells(self, l):
        self.lib.s3x_cells(self.h, l)
        return self._lists()

    def groups(self, l, kind):
        self.lib.s3x_groups(self.h, l, kind)
        return self._lists()

    def neighbors(self, c):
        self.lib.s3x_neighbors(self.h, *self._arr(c))
        return self._lists()[0]

    def touching(self, c):
        self.lib.s3x_touching(self.h, *self._arr(c))
        return self._lists()[0]

    def members(self, cid):
        self.lib.s3x_members(self.h, cid)
        return self._lists()[0]

    def active(self):
        self.lib.s3x_active(self.h)
        return self._lists()[0]

    def gather_plan(self, keys, orders):
        """(ok, dim, start, clique, map_start, map) of one batch of gathers."""
        def flat(lists):
            off = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(int)
            return self._arr([g for x in lists for g in x])[0], self._arr(off)[0]
        kf, ko = flat(keys)
        of, oo = flat(orders)
        ok = self.lib.s3x_gather_plan(self.h, len(keys), kf, ko, of, oo)
        return (ok == 1,) + tuple(self._lists())

    def eliminate(self, p):
        return self.lib.s3x_eliminate(self.h, *self._arr(p))

    def skeletonize(self, c, s):
        a, na = self._arr(c)
        b, nb = self._arr(s)
        return self.lib.s3x_skeletonize(self.h, a, na, b, nb)


def _initial_cliques(n, a_stag, b):
    """(members, matrix) of every interior bond and every DOF's diagonal."""
    m = n - 1
    inv_h2 = float(n) ** 2
    sizes = [m * m * n] * 3
    offs = np.cumsum([0] + sizes)
    idx = np.arange(m ** 3).reshape(m, m, m)                  # [z][y][x]
    diag = np.asarray(b, dtype=np.float64).reshape(m, m, m).copy()
    out = []
    for axis in range(3):
        ax = 2 - axis                                          # numpy axis of this coordinate
        shape = [m, m, m]
        shape[ax] = n
        w = np.asarray(a_stag[offs[axis]:offs[axis + 1]], dtype=np.float64).reshape(shape) * inv_h2

        def sl(v):
            t = [slice(None)] * 3
            t[ax] = v
            return tuple(t)

        diag[sl(0)] += w[sl(0)]                                # bond to the lower boundary
        diag[sl(m - 1)] += w[sl(n - 1)]                        # bond to the upper boundary
        for wi, i0, i1 in zip(w[sl(slice(1, m))].ravel(), idx[sl(slice(0, m - 1))].ravel(),
                              idx[sl(slice(1, m))].ravel()):
            out.append(([int(i0), int(i1)], np.array([[wi, -wi], [-wi, wi]])))
    for i, d in enumerate(diag.ravel()):
        out.append(([i], np.array([[d]])))
    return out


def _gather(store, ids, order):
    pos = {g: k for k, g in enumerate(order)}
    F = np.zeros((len(order), len(order)))
    for cid in ids:
        mem, M = store[cid]
        ix = [pos[g] for g in mem]
        F[np.ix_(ix, ix)] += M
    return F


def _gather_batch(store, plan_out):
    """What a gather launch computes from the flat plan: one block per target."""
    ok, dim, start, clique, map_start, mp = plan_out
    assert ok
    blocks = []
    for t, d in enumerate(dim):
        F = np.zeros((d, d))
        for k in range(start[t], start[t + 1]):
            M = store[clique[k]][1]
            ix = mp[map_start[k]:map_start[k] + M.shape[0]]
            F[np.ix_(ix, ix)] += M
        blocks.append(F)
    return blocks


def _close(X, Y, what):
    scale = max(np.abs(Y).max(), 1e-300)
    assert np.abs(X - Y).max() <= 1e-9 * scale, (what, np.abs(X - Y).max() / scale)


def _compact(plan, store, ids):
    """Cliques that lost members in the plan lose the same rows / columns."""
    for cid in ids:
        mem, M = store[cid]
        new = plan.members(cid)
        if not new:
            del store[cid]
            continue
        keep = [k for k, g in enumerate(mem) if g in set(new)]
        assert [mem[k] for k in keep] == new
        store[cid] = (new, M[np.ix_(keep, keep)])


def _run(capi, n, eps, edge_start, field_seed, plant=None):
    a, b = inputs.high_contrast_coefficients(3, n, seed=field_seed, low=1e-2, high=1e2)
    A = stencil.assemble(3, n, a, b)
    recorded = []
    orig_id = hifde.interp_decomp

    def rec_id(M, e):
        recorded.append(np.array(M))
        return orig_id(M, e)

    hifde.interp_decomp = rec_id
    try:
        F = hifde.factor3x(A, n, eps, edge_start=edge_start)
    finally:
        hifde.interp_decomp = orig_id

    plan = Plan(capi, n)
    try:
        store = {}
        for mem, M in _initial_cliques(n, a, b):
            cid = plan.add(mem)
            store[cid] = (mem, M)
        k_id = 0
        for ell in range(plan.lib.s3x_levels(plan.h)):
            lc = F.levels[2 * ell]
            cells = plan.cells(ell)
            assert len(cells) == len(lc.cells)
            qs = [plan.neighbors(p) for p in cells]   # kept cells are never coupled: one batch
            batch = _gather_batch(store, plan.gather_plan(cells, [p + q for p, q in zip(cells, qs)]))
            for p, q, rec, Fb in zip(cells, qs, lc.cells, batch):
                assert p == rec.p.tolist() and q == rec.q.tolist()
                ids = plan.touching(p)
                Fm = _gather(store, ids if plant != "drop_contribution" else ids[:-1], p + q)
                assert plant or np.array_equal(Fb, Fm)
                k = len(p)
                _close(Fm[:k, :k], rec.L @ rec.L.T, "A_pp")
                if q:
                    _close(Fm[k:, :k], rec.Aqp, "A_qp")
                U = Fm[k:, k:] - Fm[k:, :k] @ np.linalg.solve(Fm[:k, :k], Fm[:k, k:])
                for cid in ids:                        # absorbed into the new clique
                    del store[cid]
                new = plan.eliminate(p)
                if q:
                    store[new] = (q, U)
            for kind, lev in ((1, F.levels[2 * ell]), (2, F.levels[2 * ell + 1])):
                if kind == 2 and ell < edge_start:
                    continue
                groups = plan.groups(ell, kind)
                assert [fr.c.tolist() for fr in lev.fronts] == groups
                gathered = []
                Ns = [plan.neighbors(c) for c in groups]
                batch = _gather_batch(store, plan.gather_plan(groups, [c + N for c, N in zip(groups, Ns)]))
                for c, N, Fb in zip(groups, Ns, batch):  # every ID block from the same A_l
                    ids = plan.touching(c)
                    Fm = _gather(store, ids, c + N)
                    assert np.array_equal(Fb, Fm)
                    _close(Fm[len(c):, :len(c)], recorded[k_id], "A_{c^N, c}")
                    k_id += 1
                    gathered.append((ids, Fm[:len(c), :len(c)]))
                for c, fr, (ids, Acc) in zip(groups, lev.fronts, gathered):
                    where = {g: i for i, g in enumerate(c)}
                    si = [where[g] for g in fr.sk.tolist()]
                    ri = [where[g] for g in fr.rd.tolist()]
                    if ri:
                        Ass, Asr, Arr = Acc[np.ix_(si, si)], Acc[np.ix_(si, ri)], Acc[np.ix_(ri, ri)]
                        T = fr.T
                        Bsr = Asr - Ass @ T
                        Brr = Arr - T.T @ Asr - Asr.T @ T + T.T @ Ass @ T
                        _close(Brr, fr.L @ fr.L.T, "B_rr")
                        if si:
                            _close(Bsr, fr.Bsr, "B_sr")
                        delta = -Bsr @ np.linalg.solve(Brr, Bsr.T)
                    new = plan.skeletonize(c, fr.sk.tolist())
                    assert new != -2
                    if new >= 0:
                        store[new] = (fr.sk.tolist(), delta)
                    if ri and plant != "no_compact":
                        _compact(plan, store, ids)
        root = plan.active()
        assert root == F.root.tolist()
        live = [cid for cid in store if plan.members(cid)]
        _close(_gather(store, live, root), F.D, "root D")
        assert k_id == len(recorded)
    finally:
        plan.close()


@pytest.mark.parametrize("n,edge_start", [(16, 0), (24, 1), (24, 0)])
def test_clique_plan_reproduces_oracle_blocks(capi, n, edge_start):
    _run(capi, n, 1e-6, edge_start, field_seed=5)


@pytest.mark.parametrize("plant", ["drop_contribution", "no_compact"])
def test_clique_plan_planted_mistakes_fail(capi, plant):
    with pytest.raises((AssertionError, KeyError, ValueError)):
        _run(capi, 16, 1e-6, 0, field_seed=5, plant=plant)


def test_gather_plan_refuses_a_block_that_misses_a_member(capi):
    """A target whose order lacks a member of a clique touching its keys
    (here a cell gathered on p alone, without q) is refused."""
    n = 16
    a, b = inputs.high_contrast_coefficients(3, n, seed=5, low=1e-2, high=1e2)
    plan = Plan(capi, n)
    try:
        for mem, _ in _initial_cliques(n, a, b):
            plan.add(mem)
        p = plan.cells(0)[0]
        q = plan.neighbors(p)
        assert q
        assert plan.gather_plan([p], [p + q])[0]
        assert not plan.gather_plan([p], [p])[0]
    finally:
        plan.close()
