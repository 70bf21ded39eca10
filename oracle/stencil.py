"""Five-point (2D) and seven-point (3D) variable-coefficient stencil.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 3.1 (2D) and Section 3.2 (3D): at every interior node ``x_j``

    (1/h^2) * sum_e [ a_{j-e/2} (u_j - u_{j-e}) + a_{j+e/2} (u_j - u_{j+e}) ] + b_j u_j = f_j

with ``a`` sampled on the staggered grid, ``b`` at the nodes, ``h = 1/n`` and zero
Dirichlet values at the boundary nodes (a neighbour on the boundary contributes
only to the diagonal).  Unknowns are ordered lexicographically with x fastest.

``residual_ext`` evaluates f - A x in that bond form with every product and
sum in numpy longdouble, from the FP64 coefficients themselves: the CSR
matrix of ``assemble`` rounds each diagonal entry (a sum of 2 dim bond terms
and b) to FP64, which on an ill-conditioned problem alone moves the relative
residual of an accurate solution far above 1e-12.

``rhs_from_bc`` moves nonzero Dirichlet values to the right-hand side.

``convection`` is the central difference of a constant convection term
``beta . grad u``: ``(beta_e / 2h) (u_{j+e} - u_{j-e})`` per axis, zero
Dirichlet values at the boundary; skew-symmetric, so ``assemble(...) +
convection(...)`` is the unsymmetric operator (with an SPD symmetric part) of
the two-sided variant the paper's Section 6 sketches.

Pinned by: the closed-form eigenpairs of the constant-coefficient Laplacian
(``tests/test_oracle_stencil.py``) and symmetry / row-sum identities;
``rhs_from_bc`` by harmonic quadratics, which the stencil reproduces exactly,
and by one-dimensional solutions of constant flux under a variable
coefficient, along each axis; the
bond-form residual by agreement with the CSR product where the diagonal is
exact in FP64, and by exact solutions of small systems refined in longdouble.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _stag_blocks(dim, n, a_stag):
    m = n - 1
    if dim == 2:
        shapes = [(m, n), (n, m)]
    else:
        shapes = [(m, m, n), (m, n, m), (n, m, m)]
    out, off = [], 0
    for s in shapes:
        size = int(np.prod(s))
        out.append(np.asarray(a_stag[off:off + size], dtype=np.float64).reshape(s))
        off += size
    assert off == len(a_stag), "a_stag has the wrong length"
    return out


def assemble(dim: int, n: int, a_stag, b) -> sp.csr_matrix:
    """Sparse matrix A of the stencil above, as a CSR matrix (N x N, FP64)."""
    m = n - 1
    N = m ** dim
    inv_h2 = float(n) ** 2
    blocks = _stag_blocks(dim, n, a_stag)
    idx = np.arange(N).reshape((m,) * dim)     # axis order (.., j2, j1): x fastest
    rows, cols, vals = [], [], []
    diag = np.asarray(b, dtype=np.float64).reshape((m,) * dim).copy()
    for axis in range(dim):                    # axis 0 = x, 1 = y, 2 = z
        arr_axis = dim - 1 - axis              # numpy axis of this coordinate
        a = blocks[axis] * inv_h2              # shape has n along arr_axis
        # bond between node j and j+e sits at staggered index j (0..n-1) along arr_axis
        lo = [slice(None)] * dim
        hi = [slice(None)] * dim
        lo[arr_axis] = slice(0, m)             # bond to the lower neighbour: a_{j-e/2}
        hi[arr_axis] = slice(1, n)             # bond to the upper neighbour: a_{j+e/2}
        diag += a[tuple(lo)] + a[tuple(hi)]
        # off-diagonal coupling between interior nodes j and j+e (bond index j+1 .. )
        inner = [slice(None)] * dim
        inner[arr_axis] = slice(1, m)          # bonds strictly between two interior nodes
        w = a[tuple(inner)]
        left = [slice(None)] * dim
        right = [slice(None)] * dim
        left[arr_axis] = slice(0, m - 1)
        right[arr_axis] = slice(1, m)
        i0 = idx[tuple(left)].ravel()
        i1 = idx[tuple(right)].ravel()
        rows += [i0, i1]
        cols += [i1, i0]
        vals += [-w.ravel(), -w.ravel()]
    rows.append(np.arange(N))
    cols.append(np.arange(N))
    vals.append(diag.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    return A.tocsr()


def convection(dim: int, n: int, beta) -> sp.csr_matrix:
    """C x = (beta . grad) x by central differences, (beta_e / 2h)(x_{j+e} -
    x_{j-e}) for each axis e (x fastest), neighbours on the boundary dropped
    (zero Dirichlet values).  C^T = -C."""
    m = n - 1
    N = m ** dim
    idx = np.arange(N).reshape((m,) * dim)
    rows, cols, vals = [], [], []
    for axis in range(dim):
        arr_axis = dim - 1 - axis
        c = float(beta[axis]) * n / 2.0                 # beta_e / (2h), h = 1/n
        lo = [slice(None)] * dim
        hi = [slice(None)] * dim
        lo[arr_axis] = slice(0, m - 1)
        hi[arr_axis] = slice(1, m)
        i_lo, i_hi = idx[tuple(lo)].ravel(), idx[tuple(hi)].ravel()
        rows += [i_lo, i_hi]
        cols += [i_hi, i_lo]
        vals += [np.full(i_lo.size, c), np.full(i_hi.size, -c)]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def rhs_from_bc(dim: int, n: int, a_stag, g, f) -> np.ndarray:
    """Right-hand side for nonzero Dirichlet values ``g`` on the boundary nodes.

    In the stencil equation above, a neighbour x_k of the interior node x_j
    that lies on the boundary contributes ``-(1/h^2) a_{jk} u_k`` with the known
    value ``u_k = g_k``; moved to the right, it adds ``(1/h^2) a_{jk} g_k`` to
    ``f_j``.  ``g``: values at all ``(n+1)^dim`` grid nodes (coordinates 0..n, x
    fastest; only boundary nodes are read), shape ``((n+1)^dim,)`` or
    ``((n+1)^dim, nrhs)``; ``f``: ``(N,)`` or ``(N, nrhs)``.  Per node the terms
    are added axis by axis, the lower neighbour before the upper one."""
    m = n - 1
    inv_h2 = float(n) ** 2
    blocks = _stag_blocks(dim, n, a_stag)
    g = np.asarray(g, dtype=np.float64)
    out = np.array(f, dtype=np.float64, copy=True)
    X = coords(dim, n)
    for j in range(X.shape[0]):
        c = [int(v) for v in X[j]]
        for axis in range(dim):
            for side, bond, bcoord in ((c[axis] == 1, 0, 0), (c[axis] == m, n - 1, n)):
                if not side:
                    continue
                # the bond coefficient: numpy axes run z, y, x; bond index on `axis`
                at = tuple(bond if (dim - 1 - p) == axis else c[dim - 1 - p] - 1 for p in range(dim))
                a = blocks[axis][at]
                k = list(c)
                k[axis] = bcoord
                lin = sum(k[q] * (n + 1) ** q for q in range(dim))
                out[j] += inv_h2 * a * g[lin]
    return out


def coords(dim: int, n: int) -> np.ndarray:
    """Integer grid coordinates (j1, j2[, j3]) of every unknown, shape (N, dim)."""
    m = n - 1
    g = np.meshgrid(*[np.arange(1, n)] * dim, indexing="ij")
    # meshgrid 'ij' gives axis0 = first coordinate; our order is x fastest
    out = np.stack([gi.transpose(*reversed(range(dim))).ravel() for gi in g], axis=1)
    return out.astype(np.int64)


def apply_ext(dim: int, n: int, a_stag, b, x) -> np.ndarray:
    """A x in the bond form of Section 3.1 / 3.2, in numpy longdouble.
    x: (N, nrhs) (any float dtype); returns (N, nrhs) longdouble."""
    m = n - 1
    L = np.longdouble
    x = np.asarray(x).astype(L)
    nr = x.shape[1]
    xg = x.reshape((m,) * dim + (nr,))             # axis order (.., j2, j1, rhs)
    n2 = L(n) * L(n)
    Ax = np.asarray(b, dtype=np.float64).astype(L).reshape((m,) * dim)[..., None] * xg
    for axis, blk in enumerate(_stag_blocks(dim, n, a_stag)):
        arr_axis = dim - 1 - axis
        a = blk.astype(L)[..., None] * n2          # bond values, n along arr_axis
        pad = [(0, 0)] * (dim + 1)
        pad[arr_axis] = (1, 1)
        xp = np.pad(xg, pad)                       # zero Dirichlet values
        lo = [slice(None)] * (dim + 1)
        hi = [slice(None)] * (dim + 1)
        lo[arr_axis] = slice(0, m)
        hi[arr_axis] = slice(2, m + 2)
        alo = [slice(None)] * (dim + 1)
        ahi = [slice(None)] * (dim + 1)
        alo[arr_axis] = slice(0, m)
        ahi[arr_axis] = slice(1, n)
        Ax = Ax + a[tuple(alo)] * (xg - xp[tuple(lo)]) + a[tuple(ahi)] * (xg - xp[tuple(hi)])
    return Ax.reshape(x.shape)


def residual_ext(dim: int, n: int, a_stag, b, f, x_hi, x_lo=None) -> np.ndarray:
    """Per-column relative residual ||f - A (x_hi + x_lo)||_2 / ||f||_2 with A
    applied in the bond form (``apply_ext``) in numpy longdouble.
    f, x_hi, x_lo: (N,) or (N, nrhs) in the lexicographic order (x fastest)."""
    f2 = np.asarray(f, dtype=np.float64)
    if f2.ndim == 1:
        f2 = f2[:, None]
    L = np.longdouble
    x = np.asarray(x_hi, dtype=np.float64).reshape(f2.shape).astype(L)
    if x_lo is not None:
        x = x + np.asarray(x_lo, dtype=np.float64).reshape(f2.shape).astype(L)
    r = f2.astype(L) - apply_ext(dim, n, a_stag, b, x)
    return np.linalg.norm(r.astype(np.float64), axis=0) / np.linalg.norm(f2, axis=0)
