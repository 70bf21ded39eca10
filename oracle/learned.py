"""Randomized ID and the rank-prediction MLP, in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* :func:`randomized_id` -- the randomized ID mentioned in Section 4.3 (and
  again at the end of Section 4.5): choose the skeletons from ``Phi M``
  instead of ``M``, with ``Phi`` a Gaussian sampling matrix of ``ell`` rows
  (passed in as an input), fit T to ``M`` itself by least squares, then
  accept the result only if the interpolation residual of ``M`` passes the
  pivoted QR's own stopping rule for those skeletons: every column of
  ``M_r - M_s T`` has norm at most ``eps`` times the largest column norm of
  ``M`` (in a pivoted QR these are |R_{k+1,k+1}| and |R_11|, Section 2.2);
  otherwise the caller falls back to the pivoted-QR ID of ``M`` (Lemma 2.2).
  Given the same ``Phi`` (the GPU's counter-based stream, rebuilt on the
  host), its skeletons and decisions are compared with the GPU's front by
  front.
* :class:`MLP` -- the rank predictor: three layers of width 64 with ReLU,
  target log(1 + k), Huber loss (delta 1), mean over samples.  Forward and
  backward written out; gradients are pinned by central finite differences
  in ``tests/test_oracle_learned.py``.

Parity status: the MLP gradients are pinned (finite differences); the
randomized ID is pinned by exact low-rank cases (it must recover the rank and
interpolate to rounding), by its fallback on an undersized sketch, and, in a
whole factorization, by the identity sketch (which makes it the pivoted-QR
ID at ``SKETCH_RANK_TOL * eps``).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .hifde import interp_decomp

HUBER_DELTA = 1.0


# The sketch's skeletons are chosen at this fraction of eps: a Gaussian
# sketch's pivots track those of M only to a modest factor, so the pivoted QR
# of Y at eps itself stops a few columns early for M.
SKETCH_RANK_TOL = 0.1


def randomized_id(M: np.ndarray, eps: float, Phi: np.ndarray, power: int = 0):
    """ID of M from the sketch Y = Phi M (M^T M)^power (the power iterations
    the end of Section 4.5 suggests for inaccurate sketches): the skeletons
    and rank of the pivoted-QR ID of Y at (SKETCH_RANK_TOL * eps)^(2 power +
    1) (Y's singular values are M's to that power), then T by least squares
    on M itself (T minimizes every column norm of M_r - M_s T).  Returns
    (IDResult, ok) where ok says the residual check passed (column norms, see
    the module docstring) and the sketch was not saturated (k < ell).  The
    result's near_threshold flag is also set when the largest residual column
    norm lies within 1e-8 (relative) of the acceptance bound, a decision that
    rounding order could flip."""
    Y = Phi @ M
    for _ in range(power):
        Y = (Y @ M.T) @ M
    idy = interp_decomp(Y, (SKETCH_RANK_TOL * eps) ** (2 * power + 1))
    k, ell = len(idy.sk), Phi.shape[0]
    if k >= ell:
        return idy, False
    if k:
        T = np.linalg.lstsq(M[:, idy.sk], M[:, idy.rd], rcond=None)[0]
    else:
        T = np.zeros((0, len(idy.rd)))
    idr = dataclasses.replace(idy, T=T)
    E = M[:, idr.rd] - M[:, idr.sk] @ T
    e = np.linalg.norm(E, axis=0).max() if E.size else 0.0
    bound = eps * np.linalg.norm(M, axis=0).max()
    ok = bool(e <= bound)
    if abs(e - bound) <= 1e-8 * bound:
        idr = dataclasses.replace(idr, near_threshold=True)
    return idr, ok


class MLP:
    """y = W3 relu(W2 relu(W1 x + b1) + b2) + b3, hidden width H."""

    def __init__(self, params):
        self.W1, self.b1, self.W2, self.b2, self.W3, self.b3 = [np.asarray(p, dtype=np.float64) for p in params]

    @staticmethod
    def unpack(flat: np.ndarray, nin: int, H: int = 64):
        """Split the flat parameter vector (layout: W1 (H x nin) row-major, b1,
        W2 (H x H), b2, W3 (1 x H), b3)."""
        sizes = [H * nin, H, H * H, H, H, 1]
        out, off = [], 0
        for s in sizes:
            out.append(np.asarray(flat[off:off + s], dtype=np.float64))
            off += s
        W1, b1, W2, b2, W3, b3 = out
        return MLP([W1.reshape(H, nin), b1, W2.reshape(H, H), b2, W3.reshape(1, H), b3])

    def flat(self) -> np.ndarray:
        return np.concatenate([self.W1.ravel(), self.b1, self.W2.ravel(), self.b2, self.W3.ravel(), self.b3])

    def forward(self, X: np.ndarray):
        Z1 = X @ self.W1.T + self.b1
        H1 = np.maximum(Z1, 0.0)
        Z2 = H1 @ self.W2.T + self.b2
        H2 = np.maximum(Z2, 0.0)
        y = (H2 @ self.W3.T + self.b3)[:, 0]
        return y, (X, Z1, H1, Z2, H2)

    def loss_and_grad(self, X: np.ndarray, t: np.ndarray):
        """Mean Huber loss of (y - t) and its gradient (flat, same layout)."""
        y, (X, Z1, H1, Z2, H2) = self.forward(X)
        d = y - t
        n = len(t)
        loss = np.where(np.abs(d) <= HUBER_DELTA, 0.5 * d * d,
                        HUBER_DELTA * (np.abs(d) - 0.5 * HUBER_DELTA)).mean()
        g = np.clip(d, -HUBER_DELTA, HUBER_DELTA) / n          # dL/dy
        gW3 = g[None, :] @ H2                                   # 1 x H
        gb3 = np.array([g.sum()])
        gH2 = g[:, None] * self.W3                              # n x H
        gZ2 = gH2 * (Z2 > 0)
        gW2 = gZ2.T @ H1
        gb2 = gZ2.sum(axis=0)
        gH1 = gZ2 @ self.W2
        gZ1 = gH1 * (Z1 > 0)
        gW1 = gZ1.T @ X
        gb1 = gZ1.sum(axis=0)
        grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
        return loss, grad
