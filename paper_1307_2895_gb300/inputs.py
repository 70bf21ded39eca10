"""Seeded synthetic inputs for HIF-DE workloads.

This module only *generates data*: coefficient fields, nodal reaction terms,
right-hand sides and random start vectors.  It holds none of the method's
arithmetic (no stencil, no elimination, no skeletonization), so both the CUDA
path and the CPU oracle may consume what it produces.

Layouts (shared by every consumer):

* Grid: ``n`` intervals per axis, interior nodes ``j = 1..n-1`` per axis,
  ``N = (n-1)**d`` unknowns, lexicographic order with x fastest.
* ``a_stag`` (staggered coefficient, Section 3.1 and 3.2 stencils): the
  concatenation ``ax.ravel() ++ ay.ravel() [++ az.ravel()]`` where, in 2D,
  ``ax[j2-1, j1] = a((j1+1/2)h, j2 h)`` has shape ``(n-1, n)`` and
  ``ay[j2, j1-1] = a(j1 h, (j2+1/2)h)`` has shape ``(n, n-1)``.  In 3D,
  ``ax`` has shape ``(n-1, n-1, n)`` indexed ``[j3-1, j2-1, j1]``, ``ay`` shape
  ``(n-1, n, n-1)`` indexed ``[j3-1, j2, j1-1]`` and ``az`` shape
  ``(n, n-1, n-1)`` indexed ``[j3, j2-1, j1-1]``.  Every block has
  ``n*(n-1)**(d-1)`` entries.
* ``b``: nodal values, ``(n-1)**d`` entries, x fastest.

Random numbers come from splitmix64 (Steele, Lea, Flood 2014), a published
counter-based generator, so the same seed gives the same field on any host.
The quantized high-contrast field follows the recipe of Example 2 in
Section 5.1 (uniform samples, Gaussian smoothing of width 4h, two-level
quantization) with the threshold and contrast given per workload.
"""
from __future__ import annotations

import math

import numpy as np

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Return ``count`` outputs of splitmix64 for counters ``offset+1 .. offset+count``.

    The state after ``i`` steps is ``seed + i * 0x9E3779B97F4A7C15`` (mod 2^64),
    and each output is the published mixing function of that state.
    """
    with np.errstate(over="ignore"):
        gamma = np.uint64(0x9E3779B97F4A7C15)
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = (np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * gamma) & _MASK64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK64
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of splitmix64 outputs."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def standard_normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normal doubles by the Box-Muller transform of splitmix64 uniforms."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m, 2 * offset)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:count]


def splitmix64_at(seed: int, counters) -> np.ndarray:
    """splitmix64 outputs number ``counters`` (each >= 1) of the stream seeded
    with ``seed`` (array-valued counterpart of :func:`splitmix64`)."""
    with np.errstate(over="ignore"):
        c = np.asarray(counters, dtype=np.uint64)
        z = (np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + c * np.uint64(0x9E3779B97F4A7C15)) & _MASK64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK64
        return z ^ (z >> np.uint64(31))


def sketch_matrix(seed: int, level: int, nglob: int, c0: int, ell: int, rows) -> np.ndarray:
    """Gaussian sampling matrix of the randomized ID drawn by the CUDA path for
    one front (random numbers of the method, generated here from the same
    published definitions so that a checker can rebuild them).

    The front is identified by its fractional level and its smallest DOF id
    ``c0``; its key is splitmix64 output number ``level * nglob + c0 + 1`` of
    the stream seeded with ``seed``.  Entry (r, i) belongs to sketch row r and
    to the DOF ``rows[i]`` (global id): with e = r * nglob + rows[i], it is
    the cosine branch of the Box-Muller transform of u1 = 1 - U(2e + 1) and
    u2 = U(2e + 2), where U(c) is the top 53 bits of output c of the stream
    seeded with the key, over 2^53.  Returns an (ell, len(rows)) array."""
    key = int(splitmix64_at(seed, [level * nglob + c0 + 1])[0])
    rows = np.asarray(rows, dtype=np.uint64)
    e = (np.arange(ell, dtype=np.uint64)[:, None] * np.uint64(nglob) + rows[None, :]).ravel()
    u1 = 1.0 - (splitmix64_at(key, 2 * e + np.uint64(1)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    u2 = (splitmix64_at(key, 2 * e + np.uint64(2)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(6.283185307179586 * u2)
    return z.reshape(ell, len(rows))


def num_dofs(dim: int, n: int) -> int:
    return (n - 1) ** dim


def stag_shapes(dim: int, n: int):
    """Shapes of the staggered blocks ax, ay(, az) in the layout described above."""
    m = n - 1
    if dim == 2:
        return [(m, n), (n, m)]
    if dim == 3:
        return [(m, m, n), (m, n, m), (n, m, m)]
    raise ValueError("dim must be 2 or 3")


def constant_coefficients(dim: int, n: int, a: float = 1.0, b: float = 0.0):
    """a(x) = a, b(x) = b (Examples 1 and 4)."""
    size = sum(int(np.prod(s)) for s in stag_shapes(dim, n))
    return np.full(size, float(a)), np.full(num_dofs(dim, n), float(b))


def helmholtz_coefficients(dim: int, n: int, dofs_per_wavelength: float, perturb: float = 0.0,
                           seed: int = 0):
    """a(x) = 1, b(x) = -k^2 with k = 2 pi kappa and kappa = n / dofs_per_wavelength
    wavelengths across the domain (Examples 3 and 6 keep 32 and 8 DOFs per
    wavelength as n grows).  The operator is indefinite once k^2 exceeds the
    Laplacian's smallest eigenvalue d pi^2.

    ``perturb`` > 0 replaces a(x) = 1 by 1 + perturb (2 U - 1) with i.i.d.
    U[0,1) samples (stream ``seed``) on the staggered points: the grid's
    symmetries then no longer make columns of a front exactly equal in norm."""
    kappa = n / float(dofs_per_wavelength)
    k = 2.0 * math.pi * kappa
    a, b = constant_coefficients(dim, n, a=1.0, b=-k * k)
    if perturb > 0.0:
        a = 1.0 + perturb * (2.0 * uniform01(seed, a.size) - 1.0)
    return a, b


def _gaussian_taps(sigma: float, radius: int) -> np.ndarray:
    k = np.arange(-radius, radius + 1, dtype=np.float64)
    w = np.exp(-0.5 * (k / sigma) ** 2)
    return w / w.sum()


def _smooth_reflect(field: np.ndarray, taps: np.ndarray) -> np.ndarray:
    """Separable correlation with ``taps`` along every axis, reflecting boundary
    (``d c b a | a b c d``)."""
    r = (len(taps) - 1) // 2
    out = field
    for ax in range(field.ndim):
        pad = [(0, 0)] * field.ndim
        pad[ax] = (r, r)
        p = np.pad(out, pad, mode="symmetric")
        acc = np.zeros_like(out)
        length = out.shape[ax]
        for t, w in enumerate(taps):
            sl = [slice(None)] * field.ndim
            sl[ax] = slice(t, t + length)
            acc += w * p[tuple(sl)]
        out = acc
    return out


def high_contrast_coefficients(dim: int, n: int, seed: int, low: float, high: float,
                               threshold: float = 0.5, width_h: float = 4.0):
    """Quantized high-contrast field (Example 2 recipe, Section 5.1).

    1. i.i.d. U[0,1) samples on the half-step lattice (spacing h/2, ``2n+1``
       points per axis), which contains every staggered point.
    2. Separable normalized Gaussian smoothing of width ``width_h * h``
       (``2*width_h`` lattice units), truncated at four widths, reflecting
       boundary.
    3. Values above ``threshold`` become ``high``, the others ``low``.  The
       recipe splits at the median of the smoothed values; 0.5, the mean of
       U[0,1), about which the smoothed field is symmetric, is the default
       here, so one realization's high share is near but not exactly one half
       (51.9% for the 511 x 511 field of seed 2).

    Returns ``(a_stag, b)`` with ``b = 0``.
    """
    m2 = 2 * n + 1
    u = uniform01(seed, m2 ** dim).reshape((m2,) * dim)  # axis order (.., x) with x last
    sigma = 2.0 * width_h
    taps = _gaussian_taps(sigma, int(math.ceil(4 * sigma)))
    s = _smooth_reflect(u, taps)
    q = np.where(s > threshold, high, low)
    # staggered point (j1+1/2, j2) sits at lattice index (2*j1+1, 2*j2)
    if dim == 2:
        ax = q[2:2 * n:2, 1:2 * n:2]            # rows j2=1..n-1, cols j1+1/2 for j1=0..n-1
        ay = q[1:2 * n:2, 2:2 * n:2]            # rows j2+1/2 for j2=0..n-1, cols j1=1..n-1
        blocks = [ax, ay]
    else:
        ax = q[2:2 * n:2, 2:2 * n:2, 1:2 * n:2]
        ay = q[2:2 * n:2, 1:2 * n:2, 2:2 * n:2]
        az = q[1:2 * n:2, 2:2 * n:2, 2:2 * n:2]
        blocks = [ax, ay, az]
    for blk, shp in zip(blocks, stag_shapes(dim, n)):
        assert blk.shape == shp, (blk.shape, shp)
    a_stag = np.concatenate([np.ascontiguousarray(x).ravel() for x in blocks])
    return a_stag, np.zeros(num_dofs(dim, n))


def rhs(dim: int, n: int, nrhs: int, seed: int = 0) -> np.ndarray:
    """Standard normal right-hand sides, shape ``(N, nrhs)`` row-major (column r
    is right-hand side r)."""
    N = num_dofs(dim, n)
    return standard_normal(seed, N * nrhs).reshape(nrhs, N).T.copy()


def power_start(dim: int, n: int, seed: int = 0) -> np.ndarray:
    """Standard uniform start vector for the power-method error estimates."""
    return uniform01(seed, num_dofs(dim, n))


# ---- named workloads -------------------------------------------------------

def workload(name: str):
    """Named synthetic workloads (shapes and recipes of the paper's examples).

    Returns a dict with ``dim, n, a_stag, b, eps, nrhs``.
    """
    if name == "laplace2d_n64":          # Example 1 shape, 63x63 interior
        a, b = constant_coefficients(2, 64)
        return dict(dim=2, n=64, a_stag=a, b=b, eps=1e-6, nrhs=1)
    if name == "contrast2d_n512":        # Example 2 recipe, 511x511, contrast 1e6
        a, _ = high_contrast_coefficients(2, 512, seed=2, low=1e-3, high=1e3)
        b = np.full(num_dofs(2, 512), 1e-3)
        return dict(dim=2, n=512, a_stag=a, b=b, eps=1e-6, nrhs=8)
    if name == "laplace3d_n64":          # Example 4 shape, 63^3
        a, b = constant_coefficients(3, 64)
        return dict(dim=3, n=64, a_stag=a, b=b, eps=1e-6, nrhs=4)
    if name == "contrast3d_n128":        # Example 5 recipe, 127^3, contrast 1e4
        a, b = high_contrast_coefficients(3, 128, seed=5, low=1e-2, high=1e2)
        return dict(dim=3, n=128, a_stag=a, b=b, eps=1e-6, nrhs=4)
    raise KeyError(name)


def batched_problems(nprob: int = 64, seed: int = 0, nmin: int = 127, nmax: int = 1023, nrhs: int = 32):
    """Independent 2D problems of the batched workload: interior edge sizes
    n - 1 = round(exp(U[ln nmin, ln nmax])) (log-uniform), each with its own
    quantized high-contrast field of contrast 10^k, k uniform in {2, 4, 6}
    (values 10^(-k/2) and 10^(k/2), the recipe of the 511^2 workload), b = 0.
    Returns a list of dicts with ``dim, n, a_stag, b, nrhs, seed``."""
    u = uniform01(seed, 2 * nprob)
    out = []
    for p in range(nprob):
        m = int(round(float(np.exp(np.log(nmin) + u[2 * p] * (np.log(nmax) - np.log(nmin))))))
        k = 2 * (1 + min(int(u[2 * p + 1] * 3), 2))
        n = m + 1
        a, b = high_contrast_coefficients(2, n, seed=1000 + p, low=10.0 ** (-k / 2), high=10.0 ** (k / 2))
        out.append(dict(dim=2, n=n, a_stag=a, b=b, nrhs=nrhs, seed=1000 + p, contrast=10.0 ** k))
    return out
