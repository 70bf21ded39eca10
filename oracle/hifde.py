"""MF and HIF-DE, written out step by step in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Slow on purpose: the
active matrix A_l is a dict of sparse rows, every block operation is a plain
dense numpy call, and the loops follow the paper's order.

What each function follows:

* :func:`tree_levels`, :func:`separators` -- the cell partition of Section 3.1
  (separators every ``2^l m h``); grids whose ``n`` is not ``2^L m`` use the
  rounded separator positions ``round(i n / 2^L)``.
* :func:`eliminate` -- Lemma 2.1 (sparse elimination), with ``A_pp`` factored by
  Cholesky, ``A_pp = L L^T`` (so ``D_p = I``), as Section 5 does for SPD ``A``.
* :func:`interp_decomp` -- Lemma 2.2 / Corollary 2.3: ID by column-pivoted
  Householder QR, rank chosen adaptively from the pivot magnitudes (Section 2.2).
* :func:`skeletonize` -- Lemma 2.4 (skeletonization) with the implicit
  truncation of ``A_{q, r}`` described after it.
* :func:`factor` -- Algorithm 3.1 (MF, ``eps = 0``) and Algorithm 4.1 (HIF-DE in
  2D, and in 3D with face skeletonization, Section 4.2), with the accelerated
  compression of Section 4.3 (fronts hold only the strict interior of an edge
  or face; the ID compresses ``(A_{l+1/2})_{c^N, c}``).
* :func:`svd_skel`, :func:`skeletonize_svd` -- Section 4.4: the SVD
  ``A_{N,c} = U Sigma V^T`` in place of the ID, ``Q_c = diag(V, I)``, the
  directions with singular values ``<= eps sigma_1`` eliminated (Lemma 2.1 on
  ``B_{p1 p1}`` of ``V^T A_cc V``) and their interactions with ``N``
  dropped; the kept directions live on in the slots of the first ``k`` DOFs
  of ``c`` with interactions ``A_{N,c} V_2`` (``factor(..., skel="svd")``).
* :func:`eliminate_two_sided`, :func:`skeletonize_two_sided` -- the
  unsymmetric generalization of Section 6: two-sided elimination operators
  ``R_p`` and ``S_p`` from ``A_pp = L U`` (LU without pivoting, L unit lower),
  and the ID of the stacked ``[A_{N,c}; A_{c,N}^T]``, whose ``T`` serves both
  sides (``factor(..., two_sided=True)``).
* :func:`factor3x` -- the 3D variant with edge skeletonization (Section 4.5,
  Algorithm 4.2): cells built algebraically from Voronoi cells about the cell
  centers, faces and edges as Voronoi cells about the face and edge centers.
* :func:`Factor.apply_inverse`, :func:`Factor.apply` -- Eq. (4.2):
  ``F^-1 = V_0 V_1/2 ... D^-1 ... V_1/2^T V_0^T`` and ``F`` itself.
* :func:`pcg` -- preconditioned CG of Section 5 (relative residual 1e-12).
* :func:`fgmres` -- GMRES (Saad and Schultz, 1986), which Section 5 uses with
  the preconditioner ``F^-1`` where the system is not SPD; the right
  preconditioned flexible form (``z_j = F^-1 v_j`` kept).
* :func:`power_estimates` -- the a posteriori estimates ``e_a``, ``e_s`` of
  Section 5 by power iteration to 1e-2 relative precision.

Readings where the paper leaves a choice:

* index sets are ordered by ascending global index; the skeleton set is kept
  in pivot order; ``T`` has rows in skeleton order and columns in ascending
  redundant order;
* pivot = the remaining column with the smallest original position whose
  squared residual norm is at least ``(1 - 1e-10)`` times the largest one;
  residual norms are recomputed at every step (no downdating);
* rank = number of pivots with ``|R_ii| > eps |R_11|``, stopping at the first
  failure; an empty or zero block has rank 0;
* all fronts of one fractional level compress blocks of ``A_{l+1/2}`` (the
  matrix before any front of that level is skeletonized);
* corners (2D) and cell edges / corners (3D) belong to no front (Section 4.3);
* SVD skeletonization (Section 4.4): rank = number of singular values
  ``> eps sigma_1``; V's columns in descending singular-value order; the
  ``k`` kept directions take the slots of the first ``k`` DOFs of ``c``
  (ascending ids), the others those of the rest; when nothing or everything
  is dropped (``k = 0`` or ``k = |c|``) no rotation is made (``V = I``: the
  factorization does not depend on the basis of a block that is wholly kept
  or wholly eliminated).  Every front of a level takes its SVD from
  ``A_{l+1/2}`` and the rotations of all fronts apply to it together: the
  rotations of different fronts act on disjoint index sets and commute, and
  each front's eliminated directions couple only to its own kept ones.  (The
  paper's front loop is sequential; with the ID the two orders agree
  exactly, with the SVD they differ by the truncated interactions.)

* two-sided variant (Section 6): rows and columns of a front share one ID
  (of the stacked block), so the transform is ``Q_c^T A Q_c`` as in the
  symmetric case; the redundant DOFs are eliminated by LU against the
  skeletons (``B_ss <- A_ss - B_sr B_rr^-1 B_rs``); the root by LU.  For a
  symmetric ``A`` the stacked block's pivoted QR picks the same skeletons as
  ``A_{N,c}``'s (its column norms are those of ``A_{N,c}`` times sqrt(2)).

Parity status: MF, the stencil, Lemma 2.1, Lemma 2.4, the ID, the SVD
skeletonization (exact F = A when nothing is truncated, V orthogonal, the
truncated interactions within eps sigma_1, ||A - F|| of order eps), the
two-sided variant (MF exact against a dense solve, exact without truncation,
the symmetric factor recovered for a symmetric A, ||A - F|| of order eps),
F and F^-1 are
pinned by the ``-m "not gpu"`` tests (dense LU, closed forms, exact low rank,
LAPACK's pivoted QR, invariants); the power estimates by the exact 2-norms of
dense A - F, A and I - A F^-1 on small grids; PCG by scipy's preconditioned
CG, iterate by iterate; F itself by the closed-form eigenpairs of the
Laplacian (F v = lambda v to O(eps), the lowest modes included).
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List

import numpy as np
import scipy.linalg as sla

PIVOT_TIE_REL = 1e-10


# --------------------------------------------------------------------------
# geometry (Section 3.1, 3.2)
# --------------------------------------------------------------------------

def tree_levels(n: int, leaf: int = 8) -> int:
    """Tree depth L: ``n = 2^L m`` with leaf width ``m``; otherwise the nearest
    integer to ``log2(n / leaf)``, at least 1."""
    return max(1, int(round(np.log2(n / leaf))))


def separators(n: int, L: int) -> np.ndarray:
    """Separator positions ``p_i = round(i n / 2^L)`` (half up), i = 1..2^L-1.

    For ``n = 2^L m`` these are the multiples of ``m`` of Section 3.1."""
    i = np.arange(1, 2 ** L, dtype=np.int64)
    return (2 * i * n + 2 ** L) // (2 ** (L + 1))


def level_separators(n: int, L: int, ell: int) -> np.ndarray:
    """Positions of the level-``ell`` separators: every ``2^ell``-th one."""
    p = separators(n, L)
    i = np.arange(1, 2 ** L)
    return p[(i % (2 ** ell)) == 0]


def _interval_index(x: np.ndarray, seps: np.ndarray) -> np.ndarray:
    """Index of the open interval between consecutive separators containing x
    (x not on a separator)."""
    return np.searchsorted(seps, x)


# --------------------------------------------------------------------------
# active matrix A_l: dict of sparse symmetric rows
# --------------------------------------------------------------------------

class ActiveMatrix:
    """Symmetric sparse matrix stored as ``rows[i] = {j: A_ij}`` (both halves).

    The structural pattern is what the paper's neighbour set refers to:
    ``c^N = {i not in c : A_ic != 0}`` (Section 2) with "nonzero" meaning stored.
    """

    def __init__(self, A_csr):
        A = A_csr.tocsr()
        self.rows: Dict[int, Dict[int, float]] = {}
        for i in range(A.shape[0]):
            lo, hi = A.indptr[i], A.indptr[i + 1]
            self.rows[i] = dict(zip(A.indices[lo:hi].tolist(), A.data[lo:hi].tolist()))

    def active(self) -> List[int]:
        return sorted(self.rows)

    def block(self, r: List[int], c: List[int]) -> np.ndarray:
        out = np.zeros((len(r), len(c)))
        for a, i in enumerate(r):
            row = self.rows[i]
            for b, j in enumerate(c):
                v = row.get(j)
                if v is not None:
                    out[a, b] = v
        return out

    def neighbors(self, c: List[int]) -> List[int]:
        cs = set(c)
        nb = set()
        for i in c:
            nb.update(self.rows[i].keys())
        return sorted(nb - cs)

    def add_block(self, r: List[int], c: List[int], M: np.ndarray) -> None:
        for a, i in enumerate(r):
            row = self.rows[i]
            for b, j in enumerate(c):
                row[j] = row.get(j, 0.0) + M[a, b]

    def set_block(self, r: List[int], c: List[int], M: np.ndarray) -> None:
        for a, i in enumerate(r):
            row = self.rows[i]
            for b, j in enumerate(c):
                row[j] = M[a, b]

    def remove(self, dofs: List[int]) -> None:
        """Decouple and drop ``dofs`` (rows and columns)."""
        ds = set(dofs)
        touched = set()
        for i in dofs:
            touched.update(self.rows[i].keys())
        for j in touched - ds:
            row = self.rows[j]
            for i in dofs:
                row.pop(i, None)
        for i in dofs:
            del self.rows[i]


# --------------------------------------------------------------------------
# Lemma 2.1: sparse elimination
# --------------------------------------------------------------------------

def ldl_signed(A: np.ndarray):
    """A = L diag(s) L^T with L lower triangular and s_j = +-1: the LDL^T
    decomposition with 1 x 1 pivots taken in order, its D = diag(s) |D| split
    as |D|^(1/2) into L (so L = L_unit |D|^(1/2)).  Right-looking: pivot d_jj,
    s_j = sign(d_jj), l_jj = |d_jj|^(1/2), column below divided by s_j l_jj
    (so that s_j l_ij l_jj is the entry), trailing block minus s_j l l^T.
    Raises LinAlgError on a zero pivot."""
    n = A.shape[0]
    W = np.array(A, dtype=np.float64, copy=True)
    L = np.zeros((n, n))
    s = np.ones(n)
    for j in range(n):
        d = W[j, j]
        if d == 0.0 or not np.isfinite(d):
            raise np.linalg.LinAlgError("zero pivot in the LDL^T decomposition")
        s[j] = 1.0 if d > 0 else -1.0
        L[j, j] = np.sqrt(abs(d))
        L[j + 1:, j] = W[j + 1:, j] / (s[j] * L[j, j])
        W[j + 1:, j + 1:] -= s[j] * np.outer(L[j + 1:, j], L[j + 1:, j])
    return L, s


def factor_block(M: np.ndarray):
    """A diagonal block's factor (Section 5: Cholesky when SPD, an LDL^T
    decomposition otherwise): (L, s) with M = L diag(s) L^T, s = None when
    the Cholesky decomposition exists (all signs +1)."""
    try:
        return np.linalg.cholesky(M), None
    except np.linalg.LinAlgError:
        return ldl_signed(M)


@dataclasses.dataclass
class CellRecord:
    """Elimination operator S_p of Lemma 2.1 with A_pp = L D_p L^T, D_p =
    diag(sgn) (sgn None: D_p = I, the Cholesky case).  The up step applies
    D_p^-1 = D_p to the eliminated values, so that F^-1 is the product of
    the up steps, the root and the down steps."""
    p: np.ndarray      # eliminated indices (ascending)
    q: np.ndarray      # neighbour indices c^N (ascending)
    L: np.ndarray      # lower triangular factor of A_pp
    Aqp: np.ndarray    # A_qp at the time of elimination
    sgn: np.ndarray = None   # diagonal of D_p (+-1), None when all +1


def _sgn(rec, v):
    return v if rec.sgn is None else rec.sgn.reshape((-1,) + (1,) * (v.ndim - 1)) * v


def eliminate(A: ActiveMatrix, p: List[int]) -> CellRecord:
    """Lemma 2.1 with q = p^N: B_qq = A_qq - A_qp A_pp^{-1} A_qp^T; p decoupled."""
    q = A.neighbors(p)
    App = A.block(p, p)
    Aqp = A.block(q, p)
    L, sgn = factor_block(App)
    if q:
        # A_qp A_pp^{-1} A_qp^T through the factor: (A_qp L^-T) D_p (A_qp L^-T)^T
        Y = sla.solve_triangular(L, Aqp.T, lower=True)        # L^-1 A_qp^T
        A.add_block(q, q, -(Y.T @ (Y if sgn is None else sgn[:, None] * Y)))
    A.remove(p)
    return CellRecord(np.array(p, dtype=np.int64), np.array(q, dtype=np.int64), L, Aqp, sgn)


def apply_S_T(rec: CellRecord, x: np.ndarray) -> None:
    """x <- D_p^-1 S_p^T x on p and S_p^T x on q (in place, x may have several
    columns).  S_p^T = [[L^-1, 0], [-A_qp A_pp^-1, I]] on (p, q)."""
    if isinstance(rec, TwoSidedRecord):
        apply_R_T(rec, x)
        return
    xp = _sgn(rec, sla.solve_triangular(rec.L, x[rec.p], lower=True))
    if len(rec.q):
        x[rec.q] -= rec.Aqp @ sla.solve_triangular(rec.L, xp, lower=True, trans="T")
    x[rec.p] = xp


def apply_S(rec: CellRecord, x: np.ndarray) -> None:
    """x <- S_p x:  x_p <- L^-T (x_p - D_p^-1 L^-1 A_qp^T x_q)."""
    if isinstance(rec, TwoSidedRecord):
        apply_S2(rec, x)
        return
    xp = x[rec.p]
    if len(rec.q):
        xp = xp - _sgn(rec, sla.solve_triangular(rec.L, rec.Aqp.T @ x[rec.q], lower=True))
    x[rec.p] = sla.solve_triangular(rec.L, xp, lower=True, trans="T")


def apply_S_inv(rec: CellRecord, x: np.ndarray) -> None:
    """x <- S_p^{-1} x with S_p^{-1} = [[L^T, D_p^-1 L^-1 A_qp^T], [0, I]] (the
    inverse of apply_S)."""
    if isinstance(rec, TwoSidedRecord):
        apply_S2_inv(rec, x)
        return
    xp = rec.L.T @ x[rec.p]
    if len(rec.q):
        xp = xp + _sgn(rec, sla.solve_triangular(rec.L, rec.Aqp.T @ x[rec.q], lower=True))
    x[rec.p] = xp


def apply_S_inv_T(rec: CellRecord, x: np.ndarray) -> None:
    """The inverse of apply_S_T: x_q += A_qp L^-T x_p; x_p <- L D_p x_p."""
    if isinstance(rec, TwoSidedRecord):
        apply_R_inv_T(rec, x)
        return
    xp = x[rec.p].copy()
    if len(rec.q):
        x[rec.q] += rec.Aqp @ sla.solve_triangular(rec.L, xp, lower=True, trans="T")
    x[rec.p] = rec.L @ _sgn(rec, xp)


# --------------------------------------------------------------------------
# Section 6: two-sided elimination (unsymmetric A)
# --------------------------------------------------------------------------

def lu_nopivot(A: np.ndarray):
    """A = L U with L unit lower triangular and U upper triangular, pivots
    taken in order (right-looking).  Raises LinAlgError on a zero pivot."""
    n = A.shape[0]
    W = np.array(A, dtype=np.float64, copy=True)
    L = np.eye(n)
    U = np.zeros((n, n))
    for j in range(n):
        d = W[j, j]
        if d == 0.0 or not np.isfinite(d):
            raise np.linalg.LinAlgError("zero pivot in the LU decomposition")
        U[j, j:] = W[j, j:]
        L[j + 1:, j] = W[j + 1:, j] / d
        W[j + 1:, j + 1:] -= np.outer(L[j + 1:, j], W[j, j + 1:])
    return L, U


@dataclasses.dataclass
class TwoSidedRecord:
    """R_p^T = [[L^-1, 0], [-A_qp A_pp^-1, I]] and S_p = [[U^-1, -A_pp^-1
    A_pq], [0, I]] with A_pp = L U, so that R_p^T A S_p = diag(I, B_qq),
    B_qq = A_qq - A_qp A_pp^-1 A_pq."""
    p: np.ndarray
    q: np.ndarray
    L: np.ndarray
    U: np.ndarray
    Aqp: np.ndarray
    Apq: np.ndarray


def _lsolve(L, v):
    return sla.solve_triangular(L, v, lower=True, unit_diagonal=True)


def _usolve(U, v):
    return sla.solve_triangular(U, v, lower=False)


def eliminate_two_sided(A: ActiveMatrix, p: List[int]) -> TwoSidedRecord:
    """Lemma 2.1 with two-sided operators: B_qq = A_qq - A_qp A_pp^-1 A_pq."""
    q = A.neighbors(p)
    L, U = lu_nopivot(A.block(p, p))
    Aqp = A.block(q, p)
    Apq = A.block(p, q)
    if q:
        A.add_block(q, q, -(Aqp @ _usolve(U, _lsolve(L, Apq))))
    A.remove(p)
    return TwoSidedRecord(np.array(p, dtype=np.int64), np.array(q, dtype=np.int64), L, U, Aqp, Apq)


def apply_R_T(rec: TwoSidedRecord, x: np.ndarray) -> None:
    """x <- R_p^T x:  y_p = L^-1 x_p;  x_q -= A_qp U^-1 y_p;  x_p = y_p."""
    y = _lsolve(rec.L, x[rec.p])
    if len(rec.q):
        x[rec.q] -= rec.Aqp @ _usolve(rec.U, y)
    x[rec.p] = y


def apply_S2(rec: TwoSidedRecord, x: np.ndarray) -> None:
    """x <- S_p x:  x_p <- U^-1 (x_p - L^-1 A_pq x_q)."""
    xp = x[rec.p]
    if len(rec.q):
        xp = xp - _lsolve(rec.L, rec.Apq @ x[rec.q])
    x[rec.p] = _usolve(rec.U, xp)


def apply_S2_inv(rec: TwoSidedRecord, x: np.ndarray) -> None:
    """x <- S_p^-1 x with S_p^-1 = [[U, L^-1 A_pq], [0, I]]."""
    xp = rec.U @ x[rec.p]
    if len(rec.q):
        xp = xp + _lsolve(rec.L, rec.Apq @ x[rec.q])
    x[rec.p] = xp


def apply_R_inv_T(rec: TwoSidedRecord, x: np.ndarray) -> None:
    """x <- R_p^-T x with R_p^-T = [[L, 0], [A_qp U^-1, I]]."""
    xp = x[rec.p].copy()
    if len(rec.q):
        x[rec.q] += rec.Aqp @ _usolve(rec.U, xp)
    x[rec.p] = rec.L @ xp


# --------------------------------------------------------------------------
# Lemma 2.2 / Corollary 2.3: interpolative decomposition
# --------------------------------------------------------------------------

@dataclasses.dataclass
class IDResult:
    sk: np.ndarray        # skeleton column positions, pivot order
    rd: np.ndarray        # redundant column positions, ascending
    T: np.ndarray         # k x |rd|:  M[:, rd] ~ M[:, sk] T
    pivots: np.ndarray    # |R_ii| for i < k, plus the first rejected one (if any)
    near_threshold: bool  # a pivot ratio within 1e-8 (relative) of eps


def interp_decomp(M: np.ndarray, eps: float) -> IDResult:
    """Adaptive-rank ID of M (m x n) by column-pivoted Householder QR.

    Step i works on the residual rows i..m-1.  Residual column norms are
    recomputed at every step.  The pivot is the remaining column of smallest
    original position whose squared norm is within a factor (1 - 1e-10) of
    the largest; the iteration stops when |R_ii| <= eps |R_11|.  Then
    T = R_11^{-1} R_12 (Lemma 2.2)."""
    m, n = M.shape
    R = np.array(M, dtype=np.float64, copy=True)
    remaining = list(range(n))
    chosen: List[int] = []
    pivots: List[float] = []
    nu1sq = None
    near = False
    for i in range(min(m, n)):
        sq = {j: float(np.dot(R[i:, j], R[i:, j])) for j in remaining}
        mx = max(sq.values())
        if nu1sq is None:
            nu1sq = mx
        if mx == 0.0:
            break
        ratio = np.sqrt(mx / nu1sq)
        if abs(ratio - eps) <= 1e-8 * eps:
            near = True
        pivots.append(np.sqrt(mx))
        if mx <= eps * eps * nu1sq:
            break
        piv = min(j for j in remaining if sq[j] >= (1.0 - PIVOT_TIE_REL) * mx)
        chosen.append(piv)
        remaining.remove(piv)
        x = R[i:, piv].copy()
        alpha = -np.sqrt(sq[piv]) if x[0] >= 0 else np.sqrt(sq[piv])
        v = x.copy()
        v[0] -= alpha
        vv = float(np.dot(v, v))
        if vv > 0.0:
            for j in remaining:
                R[i:, j] -= (2.0 * np.dot(v, R[i:, j]) / vv) * v
        R[i:, piv] = 0.0
        R[i, piv] = alpha
    k = len(chosen)
    rd = np.array(remaining, dtype=np.int64)
    if k and len(rd):
        R11 = R[:k, chosen]
        R12 = R[:k, remaining]
        T = sla.solve_triangular(R11, R12, lower=False)
    else:
        T = np.zeros((k, len(rd)))
    return IDResult(np.array(chosen, dtype=np.int64), rd, T, np.array(pivots), near)


# --------------------------------------------------------------------------
# Lemma 2.4: skeletonization
# --------------------------------------------------------------------------

@dataclasses.dataclass
class FrontRecord:
    """U_c = Q_c S_r of Lemma 2.4 (S_r is Lemma 2.1 with p = r, q = s)."""
    c: np.ndarray      # front indices (ascending)
    sk: np.ndarray     # skeleton indices (global, pivot order)
    rd: np.ndarray     # redundant indices (global, ascending)
    T: np.ndarray      # k x |rd|
    L: np.ndarray      # lower triangular factor of B_rr (B_rr = L D L^T)
    Bsr: np.ndarray    # B_sr
    near_threshold: bool = False
    sgn: np.ndarray = None   # diagonal of D (+-1), None when B_rr is SPD


def skeletonize(A: ActiveMatrix, c: List[int], idr: IDResult) -> FrontRecord:
    """Z_c(A) of Lemma 2.4: Q_c^T A Q_c with A_{q,r} truncated, then Lemma 2.1
    on the redundant set r (whose only remaining neighbours are the skeletons)."""
    c_arr = np.array(c, dtype=np.int64)
    sk = c_arr[idr.sk]
    rd = c_arr[idr.rd]
    sk_l, rd_l = sk.tolist(), rd.tolist()
    Ass = A.block(sk_l, sk_l)
    Asr = A.block(sk_l, rd_l)
    Arr = A.block(rd_l, rd_l)
    T = idr.T
    Brr = Arr - T.T @ Asr - Asr.T @ T + T.T @ Ass @ T
    Bsr = Asr - Ass @ T
    L, sgn = factor_block(Brr) if len(rd_l) else (np.zeros((0, 0)), None)
    if len(rd_l) and len(sk_l):
        Y = sla.solve_triangular(L, Bsr.T, lower=True)          # L^-1 B_sr^T
        A.set_block(sk_l, sk_l, Ass - Y.T @ (Y if sgn is None else sgn[:, None] * Y))
    A.remove(rd_l)
    return FrontRecord(c_arr, sk, rd, T, L, Bsr, idr.near_threshold, sgn)


def _front_as_cell(fr: FrontRecord) -> CellRecord:
    if isinstance(fr, TwoSidedFrontRecord):
        return TwoSidedRecord(fr.rd, fr.sk, fr.L, fr.U, fr.Bsr, fr.Brs)
    return CellRecord(fr.rd, fr.sk, fr.L, fr.Bsr, fr.sgn)


@dataclasses.dataclass
class TwoSidedFrontRecord:
    """Section 6's front: Q_c from the ID of [A_{N,c}; A_{c,N}^T] (one T for
    rows and columns), then the two-sided elimination of r against s."""
    c: np.ndarray
    sk: np.ndarray
    rd: np.ndarray
    T: np.ndarray
    L: np.ndarray      # B_rr = L U
    U: np.ndarray
    Bsr: np.ndarray
    Brs: np.ndarray
    near_threshold: bool = False
    sgn: np.ndarray = None


def skeletonize_two_sided(A: ActiveMatrix, c: List[int], idr: IDResult) -> TwoSidedFrontRecord:
    """Q_c^T A Q_c with A_{q,r} and A_{r,q} truncated, then the two-sided
    elimination of r: B_ss <- B_ss - B_sr B_rr^-1 B_rs."""
    c_arr = np.array(c, dtype=np.int64)
    sk = c_arr[idr.sk]
    rd = c_arr[idr.rd]
    sk_l, rd_l = sk.tolist(), rd.tolist()
    Ass = A.block(sk_l, sk_l)
    Asr = A.block(sk_l, rd_l)
    Ars = A.block(rd_l, sk_l)
    Arr = A.block(rd_l, rd_l)
    T = idr.T
    Brr = Arr - T.T @ Asr - Ars @ T + T.T @ Ass @ T
    Bsr = Asr - Ass @ T
    Brs = Ars - T.T @ Ass
    if len(rd_l):
        L, U = lu_nopivot(Brr)
    else:
        L, U = np.zeros((0, 0)), np.zeros((0, 0))
    if len(rd_l) and len(sk_l):
        A.set_block(sk_l, sk_l, Ass - Bsr @ _usolve(U, _lsolve(L, Brs)))
    A.remove(rd_l)
    return TwoSidedFrontRecord(c_arr, sk, rd, T, L, U, Bsr, Brs, idr.near_threshold)


def apply_U_T(fr: FrontRecord, x: np.ndarray) -> None:
    """x <- U_c^T x = S_r^T Q_c^T x;  Q_c^T: x_r <- x_r - T^T x_s (ID), x_c <- V^T x_c (SVD)."""
    if len(fr.rd) == 0:
        return
    if isinstance(fr, SVDFrontRecord):
        _rotate(fr, x, True)
        apply_S_T(_svd_as_cell(fr), x)
        return
    if len(fr.sk):
        x[fr.rd] -= fr.T.T @ x[fr.sk]
    apply_S_T(_front_as_cell(fr), x)


def apply_U(fr: FrontRecord, x: np.ndarray) -> None:
    """x <- U_c x = Q_c S_r x;  Q_c: x_s <- x_s - T x_r (ID), x_c <- V x_c (SVD)."""
    if len(fr.rd) == 0:
        return
    if isinstance(fr, SVDFrontRecord):
        apply_S(_svd_as_cell(fr), x)
        _rotate(fr, x, False)
        return
    apply_S(_front_as_cell(fr), x)
    if len(fr.sk):
        x[fr.sk] -= fr.T @ x[fr.rd]


def apply_U_inv(fr: FrontRecord, x: np.ndarray) -> None:
    """x <- U_c^{-1} x = S_r^{-1} Q_c^{-1} x;  Q_c^{-1}: x_s <- x_s + T x_r (ID),
    x_c <- V^T x_c (SVD: Q_c^{-1} = Q_c^T)."""
    if len(fr.rd) == 0:
        return
    if isinstance(fr, SVDFrontRecord):
        _rotate(fr, x, True)
        apply_S_inv(_svd_as_cell(fr), x)
        return
    if len(fr.sk):
        x[fr.sk] += fr.T @ x[fr.rd]
    apply_S_inv(_front_as_cell(fr), x)


def apply_U_inv_T(fr: FrontRecord, x: np.ndarray) -> None:
    """x <- U_c^{-T} x = Q_c^{-T} S_r^{-T} x;  Q_c^{-T}: x_r <- x_r + T^T x_s (ID),
    x_c <- V x_c (SVD)."""
    if len(fr.rd) == 0:
        return
    if isinstance(fr, SVDFrontRecord):
        apply_S_inv_T(_svd_as_cell(fr), x)
        _rotate(fr, x, False)
        return
    apply_S_inv_T(_front_as_cell(fr), x)
    if len(fr.sk):
        x[fr.rd] += fr.T.T @ x[fr.sk]


# --------------------------------------------------------------------------
# Section 4.4: skeletonization by the SVD
# --------------------------------------------------------------------------

@dataclasses.dataclass
class SVDResult:
    V: np.ndarray         # |c| x |c| orthogonal, columns by descending singular value
    sigma: np.ndarray     # singular values, descending (min(m, |c|) of them)
    k: int                # number of singular values > eps sigma_1
    near_threshold: bool  # a ratio sigma_i / sigma_1 within 1e-8 (relative) of eps


def svd_skel(M: np.ndarray, eps: float) -> SVDResult:
    """M = U Sigma V^T (LAPACK's SVD, the full V); k = #{sigma_i > eps sigma_1};
    an empty or zero block has rank 0."""
    m, n = M.shape
    if m == 0 or n == 0:
        return SVDResult(np.eye(n), np.zeros(0), 0, False)
    _, sig, Vt = np.linalg.svd(M, full_matrices=True)
    if sig[0] == 0.0:
        return SVDResult(np.eye(n), sig, 0, False)
    ratio = sig / sig[0]
    k = int(np.count_nonzero(ratio > eps))
    near = bool(np.any(np.abs(ratio - eps) <= 1e-8 * eps))
    return SVDResult(Vt.T.copy(), sig, k, near)


@dataclasses.dataclass
class SVDFrontRecord:
    """U_c = Q_c S_p1 with Q_c = diag(V, I) (Section 4.4's lemma) and S_p1 the
    elimination (Lemma 2.1) of the dropped directions p1 against the kept
    ones p2 only.  Slots: p2 = c[:k] (``sk``), p1 = c[k:] (``rd``); V = None
    when no rotation is made."""
    c: np.ndarray
    sk: np.ndarray
    rd: np.ndarray
    V: np.ndarray      # |c| x |c| or None
    L: np.ndarray      # factor of B_p1p1 (B = V^T A_cc V)
    Bsr: np.ndarray    # B_p2p1
    near_threshold: bool = False
    sgn: np.ndarray = None


def skeletonize_svd(A: ActiveMatrix, c: List[int], sv: SVDResult) -> SVDFrontRecord:
    """Q_c^T A Q_c with the interactions of the dropped directions truncated,
    then Lemma 2.1 on them (their only remaining neighbours are the kept
    directions): B~_p2p2 = B_p2p2 - B_p2p1 B_p1p1^-1 B_p1p2."""
    c_arr = np.array(c, dtype=np.int64)
    nc, k = len(c), sv.k
    V = sv.V if 0 < k < nc else None
    if V is not None:
        nb = A.neighbors(c)
        if nb:
            X = A.block(nb, c) @ V                              # A_{N,c} V
            A.set_block(nb, c, X)
            A.set_block(c, nb, X.T)
        A.set_block(c, c, V.T @ A.block(c, c) @ V)
    sk, rd = c_arr[:k], c_arr[k:]
    sk_l, rd_l = sk.tolist(), rd.tolist()
    B_ss = A.block(sk_l, sk_l)
    B_sr = A.block(sk_l, rd_l)
    B_rr = A.block(rd_l, rd_l)
    L, sgn = factor_block(B_rr) if len(rd_l) else (np.zeros((0, 0)), None)
    if len(rd_l) and len(sk_l):
        Y = sla.solve_triangular(L, B_sr.T, lower=True)
        A.set_block(sk_l, sk_l, B_ss - Y.T @ (Y if sgn is None else sgn[:, None] * Y))
    A.remove(rd_l)
    return SVDFrontRecord(c_arr, sk, rd, V, L, B_sr, sv.near_threshold, sgn)


def _rotate(fr: SVDFrontRecord, x: np.ndarray, transpose: bool) -> None:
    if fr.V is not None:
        x[fr.c] = (fr.V.T if transpose else fr.V) @ x[fr.c]


def _svd_as_cell(fr: SVDFrontRecord) -> CellRecord:
    return CellRecord(fr.rd, fr.sk, fr.L, fr.Bsr, fr.sgn)


# --------------------------------------------------------------------------
# Algorithms 3.1 / 4.1
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Level:
    """One level of the factorization: V_l (cells) then V_{l+1/2} (fronts)."""
    ell: int
    cells: List[CellRecord]
    fronts: List[FrontRecord]
    front_keys: List[tuple]


@dataclasses.dataclass
class Factor:
    dim: int
    n: int
    L: int
    eps: float
    levels: List[Level]
    root: np.ndarray           # s_L (ascending)
    D: np.ndarray              # A_L restricted to s_L
    Dchol: np.ndarray          # its lower triangular factor (D = Dchol diag(Dsgn) Dchol^T)
    sketched: int = 0          # fronts whose sketched ID passed the check
    fallback: int = 0          # fronts whose sketched ID failed it
    Dsgn: np.ndarray = None    # signs of D's LDL^T decomposition (None: Cholesky)
    DU: np.ndarray = None      # two-sided variant: D = Dchol DU (Dchol unit lower), None otherwise

    # ---- Eq. (4.2): F^-1 = V_0 V_1/2 ... D^-1 ... V_1/2^T V_0^T
    def apply_inverse(self, b: np.ndarray) -> np.ndarray:
        x = np.array(b, dtype=np.float64, copy=True)
        for lev in self.levels:                       # V^T, finest first
            for rec in lev.cells:
                apply_S_T(rec, x)
            for fr in lev.fronts:
                apply_U_T(fr, x)
        if len(self.root) and self.DU is not None:
            x[self.root] = _usolve(self.DU, _lsolve(self.Dchol, x[self.root]))
        elif len(self.root):
            y = sla.solve_triangular(self.Dchol, x[self.root], lower=True)
            if self.Dsgn is not None:
                y = self.Dsgn.reshape((-1,) + (1,) * (y.ndim - 1)) * y
            x[self.root] = sla.solve_triangular(self.Dchol, y, lower=True, trans="T")
        for lev in reversed(self.levels):             # V, coarsest first
            for fr in lev.fronts:
                apply_U(fr, x)
            for rec in lev.cells:
                apply_S(rec, x)
        return x

    # ---- F = V_0^-T ... V_{L-1/2}^-T D V_{L-1/2}^-1 ... V_0^-1
    def apply(self, b: np.ndarray) -> np.ndarray:
        x = np.array(b, dtype=np.float64, copy=True)
        for lev in self.levels:                       # V^-1, finest first
            for rec in lev.cells:
                apply_S_inv(rec, x)
            for fr in lev.fronts:
                apply_U_inv(fr, x)
        if len(self.root):
            x[self.root] = self.D @ x[self.root]
        for lev in reversed(self.levels):             # V^-T, coarsest first
            for fr in lev.fronts:
                apply_U_inv_T(fr, x)
            for rec in lev.cells:
                apply_S_inv_T(rec, x)
        return x

    # ---- structure for parity checks
    def skeleton_structure(self):
        """Per fractional level: {front key: (c, sk in pivot order, rank)} and |s_L|."""
        out = []
        for lev in self.levels:
            d = {}
            for key, fr in zip(lev.front_keys, lev.fronts):
                d[key] = (fr.c.tolist(), fr.sk.tolist(), len(fr.sk))
            out.append(d)
        return out, len(self.root)


def _front_key(dim, x, on_sep, seps):
    """Front identity: (axis with the separator coordinate, separator ordinal,
    interval index along each other axis)."""
    axis = int(np.nonzero(on_sep)[0][0])
    ordinal = int(np.searchsorted(seps, x[axis]))
    others = tuple(int(_interval_index(np.array([x[a]]), seps)[0]) for a in range(dim) if a != axis)
    return (axis, ordinal) + others


def factor(A_csr, dim: int, n: int, eps: float, leaf: int = 8,
           skip_levels: int = 0, sketch=None, sketch_power: int = 0, skel: str = "id",
           two_sided: bool = False) -> Factor:
    """Algorithm 4.1 (HIF-DE; ``eps > 0``) or Algorithm 3.1 (MF; ``eps == 0``).

    Level l: eliminate the active DOFs strictly inside each level-l cell
    (Lemma 2.1, cells in ascending linear index, x fastest).  Level l + 1/2
    (skipped when ``eps == 0`` or ``l < skip_levels``): group the active DOFs
    with exactly one coordinate on a level-l separator by front (2D edge or
    3D face interior), compute every front's ID from ``A_{l+1/2}``, then
    skeletonize the fronts (Lemma 2.4).  Finally ``D = A_L`` on ``s_L``.

    ``sketch`` (optional) supplies the random numbers of the randomized ID
    (Section 4.3): ``sketch(l, c, rows)`` returns the Gaussian sampling
    matrix for front ``c`` (ascending DOF ids) whose ID block has the rows
    ``rows`` (ascending DOF ids), or None to use the pivoted-QR ID.  A
    sketched ID that fails :func:`oracle.learned.randomized_id`'s check falls
    back to the pivoted-QR ID of the block itself (``sketch_power`` power
    iterations on the sketch).  The counts of accepted and rejected sketches
    are kept on the result.

    ``skel="svd"`` skeletonizes the fronts by the SVD (Section 4.4,
    :func:`skeletonize_svd`) instead of the ID.  ``two_sided=True`` is the
    unsymmetric variant of Section 6 (two-sided elimination by LU, the ID of
    the stacked ``[A_{N,c}; A_{c,N}^T]``, the root by LU)."""
    from .stencil import coords as _coords
    if skel not in ("id", "svd"):
        raise ValueError(f"skel must be 'id' or 'svd', not {skel!r}")
    if skel == "svd" and sketch is not None:
        raise ValueError("the randomized ID and the SVD skeletonization are exclusive")
    if two_sided and (skel != "id" or sketch is not None):
        raise ValueError("the two-sided variant uses the pivoted-QR ID")
    A = ActiveMatrix(A_csr)
    X = _coords(dim, n)
    L = tree_levels(n, leaf)
    levels: List[Level] = []
    n_sketched = n_fallback = 0
    for ell in range(L):
        seps = level_separators(n, L, ell)
        act = np.array(A.active(), dtype=np.int64)
        Xa = X[act]
        on = np.isin(Xa, seps)
        non = on.sum(axis=1)
        # ---- level l: cells
        inside = act[non == 0]
        cell_dofs: Dict[int, List[int]] = {}
        if len(inside):
            iv = np.searchsorted(seps, X[inside])              # interval per axis
            ncell = len(seps) + 1
            lin = np.zeros(len(inside), dtype=np.int64)
            for a in reversed(range(dim)):
                lin = lin * ncell + iv[:, a]
            for d, cidx in zip(inside.tolist(), lin.tolist()):
                cell_dofs.setdefault(cidx, []).append(d)
        elim = eliminate_two_sided if two_sided else eliminate
        cells = [elim(A, sorted(cell_dofs[k])) for k in sorted(cell_dofs)]
        # ---- level l + 1/2: fronts
        fronts: List[FrontRecord] = []
        keys: List[tuple] = []
        if eps > 0 and ell >= skip_levels:
            act = np.array(A.active(), dtype=np.int64)
            Xa = X[act]
            on = np.isin(Xa, seps)
            one = act[on.sum(axis=1) == 1]
            groups: Dict[tuple, List[int]] = {}
            for d in one.tolist():
                key = _front_key(dim, X[d], np.isin(X[d], seps), seps)
                groups.setdefault(key, []).append(d)
            keys = sorted(groups)
            ids = []
            for key in keys:                           # all IDs from A_{l+1/2}
                c = sorted(groups[key])
                nb = A.neighbors(c)
                M = A.block(nb, c)
                if skel == "svd":
                    ids.append(svd_skel(M, eps))
                    continue
                if two_sided:                          # rows and columns: one ID (Section 6)
                    ids.append(interp_decomp(np.vstack([M, A.block(c, nb).T]), eps))
                    continue
                Phi = sketch(ell, c, nb) if sketch is not None else None
                idr = None
                if Phi is not None:
                    from .learned import randomized_id
                    ids_s, ok = randomized_id(M, eps, Phi, sketch_power)
                    if ok:
                        idr = ids_s
                        n_sketched += 1
                    else:
                        n_fallback += 1
                if idr is None:
                    idr = interp_decomp(M, eps)
                    if Phi is not None and ids_s.near_threshold:
                        idr = dataclasses.replace(idr, near_threshold=True)
                ids.append(idr)
            for key, idr in zip(keys, ids):
                if skel == "svd":
                    fronts.append(skeletonize_svd(A, sorted(groups[key]), idr))
                elif two_sided:
                    fronts.append(skeletonize_two_sided(A, sorted(groups[key]), idr))
                else:
                    fronts.append(skeletonize(A, sorted(groups[key]), idr))
        levels.append(Level(ell, cells, fronts, keys))
    root = np.array(A.active(), dtype=np.int64)
    D = A.block(root.tolist(), root.tolist())
    if two_sided:
        DL, DU = lu_nopivot(D) if len(root) else (np.zeros((0, 0)), np.zeros((0, 0)))
        return Factor(dim, n, L, eps, levels, root, D, DL, n_sketched, n_fallback, None, DU)
    Dchol, Dsgn = factor_block(D) if len(root) else (np.zeros((0, 0)), None)
    return Factor(dim, n, L, eps, levels, root, D, Dchol, n_sketched, n_fallback, Dsgn)


# --------------------------------------------------------------------------
# Section 4.5: HIF-DE in 3D with edge skeletonization
# --------------------------------------------------------------------------

def _nearest(x2: np.ndarray, pos2: np.ndarray):
    """Per entry of x2: index of the nearest of the sorted positions pos2,
    the squared distance, and whether a second position is as near (all in
    doubled grid units, so exact in integers)."""
    j = np.clip(np.searchsorted(pos2, x2), 0, len(pos2) - 1)
    jl = np.clip(j - 1, 0, len(pos2) - 1)
    dj = (x2 - pos2[j]) ** 2
    dl = (x2 - pos2[jl]) ** 2
    best = np.where(dl < dj, jl, j)
    dbest = np.minimum(dl, dj)
    tie = (dl == dj) & (jl != j)
    return best, dbest, tie


def _voronoi(X: np.ndarray, families):
    """Nearest center among the union of center families, each a Cartesian
    product of per-axis position lists (doubled units); returns (family, index
    tuple) per DOF, or None where two or more centers are nearest (such DOFs
    join no group)."""
    X2 = 2 * X
    dist, idx, tied = [], [], []
    for axes in families:
        d = np.zeros(len(X), dtype=np.int64)
        t = np.zeros(len(X), dtype=bool)
        ii = []
        for a, pos2 in enumerate(axes):
            b, db, tb = _nearest(X2[:, a], pos2)
            d += db
            t |= tb
            ii.append(b)
        dist.append(d)
        idx.append(np.stack(ii, axis=1))
        tied.append(t)
    D = np.stack(dist, axis=1)
    dmin = D.min(axis=1)
    out = []
    for r in range(len(X)):
        fams = np.nonzero(D[r] == dmin[r])[0]
        if len(fams) != 1 or tied[fams[0]][r]:
            out.append(None)
        else:
            f = int(fams[0])
            out.append((f,) + tuple(int(v) for v in idx[f][r]))
    return out


def _groups(A: ActiveMatrix, X: np.ndarray, families) -> Dict[tuple, List[int]]:
    act = np.array(A.active(), dtype=np.int64)
    keys = _voronoi(X[act], families)
    g: Dict[tuple, List[int]] = {}
    for d, k in zip(act.tolist(), keys):
        if k is not None:
            g.setdefault(k, []).append(d)
    return g


def _skeletonize_groups(A: ActiveMatrix, groups: Dict[tuple, List[int]], eps: float):
    """All IDs from the current matrix, then every group skeletonized
    (one fractional level)."""
    keys = sorted(groups)
    ids = []
    for key in keys:
        c = sorted(groups[key])
        ids.append(interp_decomp(A.block(A.neighbors(c), c), eps))
    fronts = [skeletonize(A, sorted(groups[key]), idr) for key, idr in zip(keys, ids)]
    return fronts, keys


def factor3x(A_csr, n: int, eps: float, leaf: int = 8, edge_start: int = 1) -> Factor:
    """HIF-DE in 3D with edge skeletonization (Section 4.5, Algorithm 4.2), for
    ``n = 2^L leaf``.  With S = 2^l leaf and K = 2^(L-l), at each level l:

    * level l: Voronoi cells of the active DOFs about the cell centers
      ((j - 1/2) S per axis, j = 1..K); then, cell by cell in ascending linear
      index (x fastest), the DOFs with a stored entry in the column of a DOF
      of another current cell are removed from their cell; each cell left is
      eliminated (Lemma 2.1);
    * level l + 1/3: Voronoi cells about the face centers (j S on the face's
      normal axis, j = 1..K-1; (j - 1/2) S on the other two), skeletonized
      (Lemma 2.4, all IDs from A_{l+1/3});
    * level l + 2/3: the same about the edge centers (j S on two axes,
      (j - 1/2) S along the edge).

    A DOF equidistant to two or more nearest centers joins no group and stays
    active.  Edge skeletonization runs from level ``edge_start`` on (the
    paper's rule of thumb: skip it while it would not pay for the thicker
    separators it causes; by default it starts at level 1).  Each l gives two entries of ``levels`` (cells and
    faces, then the edges), so that F and F^-1 apply them in the algorithm's
    order."""
    from .stencil import coords as _coords
    A = ActiveMatrix(A_csr)
    X = _coords(3, n)
    L = tree_levels(n, leaf)
    m = n // (2 ** L)
    levels: List[Level] = []
    for ell in range(L):
        S, K = m * 2 ** ell, 2 ** (L - ell)
        centers = np.array([(2 * j - 1) * S for j in range(1, K + 1)], dtype=np.int64)
        planes = np.array([2 * j * S for j in range(1, K)], dtype=np.int64)
        # ---- level l: algebraic cells
        cell_groups = _groups(A, X, [(centers, centers, centers)])
        member = {}
        lin_of = {}
        for key, dofs in cell_groups.items():
            lin = key[1] + K * (key[2] + K * key[3])
            lin_of[key] = lin
            for d in dofs:
                member[d] = lin
        kept: Dict[int, List[int]] = {}
        for key in sorted(cell_groups, key=lambda k: lin_of[k]):
            lin = lin_of[key]
            keep = []
            for i in sorted(cell_groups[key]):
                ext = any(member.get(j, lin) != lin for j in A.rows[i] if j != i)
                if ext:
                    del member[i]
                else:
                    keep.append(i)
            kept[lin] = keep
        cells = [eliminate(A, kept[lin]) for lin in sorted(kept) if kept[lin]]
        # ---- level l + 1/3: faces
        faces = [(planes, centers, centers), (centers, planes, centers), (centers, centers, planes)]
        ffr, fkeys = _skeletonize_groups(A, _groups(A, X, faces), eps)
        levels.append(Level(ell, cells, ffr, fkeys))
        # ---- level l + 2/3: edges
        edges = [(centers, planes, planes), (planes, centers, planes), (planes, planes, centers)]
        efr, ekeys = _skeletonize_groups(A, _groups(A, X, edges), eps) if ell >= edge_start else ([], [])
        levels.append(Level(ell, [], efr, ekeys))
    root = np.array(A.active(), dtype=np.int64)
    D = A.block(root.tolist(), root.tolist())
    Dchol, Dsgn = factor_block(D) if len(root) else (np.zeros((0, 0)), None)
    return Factor(3, n, L, eps, levels, root, D, Dchol, 0, 0, Dsgn)


# --------------------------------------------------------------------------
# Section 5: PCG and the power-method error estimates
# --------------------------------------------------------------------------

def pcg(A_csr, F: Factor, b: np.ndarray, tol: float = 1e-12, maxit: int = 200):
    """Preconditioned CG with M^-1 = F^-1 on each column of b (textbook
    recurrences).  When the recursive residual reaches tol, the true residual
    b - A x is computed; if it is still above tol, CG restarts from it.
    Returns (x, iters, relres) with relres the true FP64 relative residual."""
    b2 = b.reshape(b.shape[0], -1)
    X = np.zeros_like(b2)
    iters, relres = [], []
    for col in range(b2.shape[1]):
        bb = b2[:, col]
        nb = np.linalg.norm(bb)
        x = np.zeros_like(bb)
        r = bb.copy()
        it = 0
        restarts = 0
        while it < maxit:
            z = F.apply_inverse(r)
            p = z.copy()
            rz = float(r @ z)
            while np.linalg.norm(r) > tol * nb and it < maxit:
                q = A_csr @ p
                alpha = rz / float(p @ q)
                x += alpha * p
                r = r - alpha * q
                it += 1
                z = F.apply_inverse(r)
                rz_new = float(r @ z)
                p = z + (rz_new / rz) * p
                rz = rz_new
            r = bb - A_csr @ x
            if np.linalg.norm(r) <= tol * nb or restarts >= 5:
                break
            restarts += 1
        X[:, col] = x
        iters.append(it)
        relres.append(np.linalg.norm(bb - A_csr @ x) / nb)
    return X.reshape(b.shape), iters, relres


def fgmres(A, apply_minv, b: np.ndarray, tol: float = 1e-12, maxit: int = 200, restart: int = 50):
    """Right-preconditioned flexible GMRES(restart) on each column of b.

    One cycle from the residual r (beta = ||r||): v_0 = r / beta; for
    j = 0, 1, ...: z_j = M^-1 v_j, w = A z_j, modified Gram-Schmidt
    h_ij = <w, v_i>, w -= h_ij v_i (i <= j), h_{j+1,j} = ||w||,
    v_{j+1} = w / h_{j+1,j}; y minimizes ||beta e_1 - H_j y|| (numpy lstsq)
    and the cycle stops when that residual is at most tol ||b|| (or at a
    breakdown h_{j+1,j} = 0, or after `restart` steps); then x += Z y and
    the next cycle starts from the true residual b - A x.  ``A`` is anything
    with ``A @ v``; ``apply_minv(v)`` applies M^-1.  Returns (x, iters,
    relres) like :func:`pcg`, iters counting the steps j."""
    b2 = b.reshape(b.shape[0], -1)
    X = np.zeros_like(b2)
    iters, relres = [], []
    for col in range(b2.shape[1]):
        bb = b2[:, col]
        nb = np.linalg.norm(bb)
        x = np.zeros_like(bb)
        r = bb.copy()
        it = 0
        while it < maxit:
            beta = np.linalg.norm(r)
            if beta <= tol * nb:
                break
            V = [r / beta]
            Z = []
            H = np.zeros((restart + 1, restart))
            y = np.zeros(0)
            for j in range(restart):
                Z.append(apply_minv(V[j]))
                w = A @ Z[j]
                for i in range(j + 1):
                    H[i, j] = w @ V[i]
                    w = w - H[i, j] * V[i]
                H[j + 1, j] = np.linalg.norm(w)
                it += 1
                e1 = np.zeros(j + 2)
                e1[0] = beta
                y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
                res = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y)
                if H[j + 1, j] == 0.0 or res <= tol * nb or it >= maxit:
                    break
                V.append(w / H[j + 1, j])
            x = x + np.column_stack(Z) @ y
            r = bb - A @ x
        X[:, col] = x
        iters.append(it)
        relres.append(np.linalg.norm(bb - A @ x) / nb)
    return X.reshape(b.shape), iters, relres


def power_norm(op, x0: np.ndarray, rtol: float = 1e-2, maxit: int = 200) -> float:
    """||op|| by power iteration ||op x|| / ||x|| from x0, stopped at rtol
    relative change (Section 5)."""
    x = x0 / np.linalg.norm(x0)
    est = 0.0
    for _ in range(maxit):
        y = op(x)
        ny = float(np.linalg.norm(y))
        if ny == 0.0:
            return 0.0
        if est > 0 and abs(ny - est) <= rtol * ny:
            return ny
        est = ny
        x = y / ny
    return est


def power_estimates(A_csr, F: Factor, x0: np.ndarray):
    """(e_a, e_s): e_a ~ ||A - F|| / ||A||,  e_s ~ ||I - A F^-1||
    (the latter through (I - F^-1 A)(I - A F^-1), whose norm is its square)."""
    nA = power_norm(lambda v: A_csr @ v, x0)
    nE = power_norm(lambda v: A_csr @ v - F.apply(v), x0)

    def MtM(v):
        w = v - A_csr @ F.apply_inverse(v)
        return w - F.apply_inverse(A_csr @ w)

    es = np.sqrt(power_norm(MtM, x0))
    return nE / nA, es
