"""Pins of the oracle's stencil (Section 3.1 / 3.2) and of the input generators."""
import numpy as np
import scipy.sparse.linalg as spla
import pytest

from oracle import stencil
from paper_1307_2895_gb300 import inputs


def _mode(dim, n, idx):
    """Discrete sine mode prod_a sin(i_a pi x_a) on the interior nodes."""
    X = stencil.coords(dim, n) / n
    v = np.ones(X.shape[0])
    for a, i in enumerate(idx):
        v *= np.sin(i * np.pi * X[:, a])
    return v


@pytest.mark.parametrize("dim,n", [(2, 16), (2, 33), (3, 8), (3, 11)])
def test_closed_form_eigenpairs(dim, n):
    """a = 1, b = 0: A v = lambda v with lambda = (4/h^2) sum_a sin^2(i_a pi h / 2)."""
    a, b = inputs.constant_coefficients(dim, n)
    A = stencil.assemble(dim, n, a, b)
    h = 1.0 / n
    rng = np.random.default_rng(1)
    for _ in range(5):
        idx = rng.integers(1, n, size=dim)
        v = _mode(dim, n, idx)
        lam = (4.0 / h ** 2) * np.sum(np.sin(idx * np.pi * h / 2) ** 2)
        assert np.linalg.norm(A @ v - lam * v) <= 1e-10 * lam * np.linalg.norm(v)


def test_extreme_eigenvalues_2d():
    n = 16
    a, b = inputs.constant_coefficients(2, n)
    ev = np.linalg.eigvalsh(stencil.assemble(2, n, a, b).toarray())
    h = 1.0 / n
    assert ev[0] == pytest.approx(8.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2, rel=1e-12)
    assert ev[-1] == pytest.approx(8.0 / h ** 2 * np.sin((n - 1) * np.pi * h / 2) ** 2, rel=1e-12)


@pytest.mark.parametrize("dim,n", [(2, 12), (3, 7)])
def test_variable_coefficient_structure(dim, n):
    """Symmetric, diagonal = b + sum of the 2d adjacent bond values / h^2, and
    with b = 0 the row sums vanish away from the boundary."""
    a, _ = inputs.high_contrast_coefficients(dim, n, seed=3, low=1e-2, high=1e2)
    b = inputs.uniform01(9, (n - 1) ** dim)
    A = stencil.assemble(dim, n, a, b)
    assert abs(A - A.T).max() == 0.0
    A0 = stencil.assemble(dim, n, a, np.zeros_like(b))
    X = stencil.coords(dim, n)
    interior = np.all((X > 1) & (X < n - 1), axis=1)
    rs = np.asarray(A0.sum(axis=1)).ravel()
    assert np.max(np.abs(rs[interior])) <= 1e-9 * n * n * a.max()
    assert np.all(rs[~interior] > 0)
    # one explicit bond: between node (1,1,..) and (2,1,..) the coupling is -a((1+1/2)h, h, ..) n^2
    i0 = 0
    i1 = 1
    ax = a[: n * (n - 1) ** (dim - 1)].reshape(((n - 1),) * (dim - 1) + (n,))
    expect = -ax[(0,) * (dim - 1) + (1,)] * n * n
    assert A[i0, i1] == pytest.approx(expect, rel=1e-15)


def test_splitmix64_published_vectors():
    """splitmix64 outputs for seed 0 and 1234567 (published reference values)."""
    assert [int(v) for v in inputs.splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                          0x06C45D188009454F]
    assert [int(v) for v in inputs.splitmix64(1234567, 3)] == [6457827717110365317, 3203168211198807973,
                                                                9817491932198370423]


def test_generators_deterministic_and_shaped():
    a1, b1 = inputs.high_contrast_coefficients(2, 32, seed=5, low=1e-3, high=1e3)
    a2, _ = inputs.high_contrast_coefficients(2, 32, seed=5, low=1e-3, high=1e3)
    assert np.array_equal(a1, a2) and len(a1) == 2 * 32 * 31 and set(np.unique(a1)) <= {1e-3, 1e3}
    frac = np.mean(a1 > 1)
    assert 0.2 < frac < 0.8
    z = inputs.standard_normal(0, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    r = inputs.rhs(2, 16, 3)
    assert r.shape == (225, 3) and r.flags["C_CONTIGUOUS"]


@pytest.mark.parametrize("dim,n", [(2, 12), (3, 7)])
def test_residual_ext_matches_csr_where_exact(dim, n):
    """a = 1 (all diagonal entries exact in FP64): the longdouble bond-form
    residual equals f - A x with the CSR product carried out in longdouble."""
    a, b = inputs.constant_coefficients(dim, n)
    b = b + 0.5                                  # exact in FP64 as well
    A = stencil.assemble(dim, n, a, b)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((A.shape[0], 2))
    f = rng.standard_normal((A.shape[0], 2))
    L = np.longdouble
    prod = A.data.astype(L)[:, None] * x.astype(L)[A.indices]
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    Ax = np.zeros(x.shape, dtype=L)
    np.add.at(Ax, rows, prod)
    ref = np.linalg.norm((f.astype(L) - Ax).astype(np.float64), axis=0) / np.linalg.norm(f, axis=0)
    got = stencil.residual_ext(dim, n, a, b, f, x)
    assert np.allclose(got, ref, rtol=1e-12, atol=0)


def test_residual_ext_of_refined_solution():
    """Contrast 1e6, b = 1e-3: a direct FP64 solve refined twice with the
    longdouble bond-form residual reaches 1e-13 in the bond-form residual
    (the x86 80-bit longdouble, u ~ 1e-19, limits it to a few 1e-14);
    the same iterate measured with the FP64-assembled matrix does not (its
    rounded diagonal is a different operator at that level)."""
    import scipy.sparse.linalg as spla
    dim, n = 2, 32
    a, _ = inputs.high_contrast_coefficients(dim, n, seed=2, low=1e-3, high=1e3)
    b = np.full((n - 1) ** dim, 1e-3)
    A = stencil.assemble(dim, n, a, b)
    f = inputs.rhs(dim, n, 2, seed=1)
    lu = spla.splu(A.tocsc())
    L = np.longdouble
    x = lu.solve(f).astype(L)
    for _ in range(3):
        r = (f.astype(L) - stencil.apply_ext(dim, n, a, b, x)).astype(np.float64)
        x = x + lu.solve(r).astype(L)
    xh = x.astype(np.float64)
    xl = (x - xh.astype(L)).astype(np.float64)
    assert stencil.residual_ext(dim, n, a, b, f, xh, xl).max() <= 1e-13
    assert stencil.residual_ext(dim, n, a, b, f, xh).max() <= 1e-9


def _grid_values(dim, n, fn):
    """fn(x, y[, z]) at all (n+1)^dim nodes (coordinates 0..n, x fastest), h = 1/n."""
    c = np.meshgrid(*[np.arange(n + 1)] * dim, indexing="ij")
    c = [ci.transpose(*reversed(range(dim))).ravel() / n for ci in c]
    return fn(*c)


def _interior(dim, n, full):
    X = stencil.coords(dim, n)
    return full[sum(X[:, q] * (n + 1) ** q for q in range(dim))]


@pytest.mark.parametrize("dim,n", [(2, 16), (2, 21), (3, 12)])
def test_rhs_from_bc_harmonic_quadratic(dim, n):
    """a = 1, b = 0: the stencil's second differences are exact on quadratics,
    so with g = u for a harmonic quadratic u, A x = rhs_from_bc(g, 0) has the
    solution x = u at the interior nodes."""
    if dim == 2:
        u = lambda x, y: x * x - y * y + 0.3 * x * y + 0.5 * x - 0.2
    else:
        u = lambda x, y, z: x * x + y * y - 2 * z * z + 0.7 * x * z - 0.4 * y + 0.1
    a, b = inputs.constant_coefficients(dim, n)
    g = _grid_values(dim, n, u)
    rhs = stencil.rhs_from_bc(dim, n, a, g, np.zeros((n - 1) ** dim))
    x = spla.spsolve(stencil.assemble(dim, n, a, b).tocsc(), rhs)
    ui = _interior(dim, n, g)
    assert np.abs(x - ui).max() <= 1e-12 * np.abs(ui).max()


@pytest.mark.parametrize("dim,axis", [(2, 0), (2, 1), (3, 0), (3, 1), (3, 2)])
def test_rhs_from_bc_constant_flux(dim, axis):
    """b = 0, a along `axis` a function of the bond index alone, the other
    coefficients arbitrary: u_k = sum_{i<k} 1/a_{i+1/2} (unit flux through
    every bond, constant across the other axes) solves the equation at every
    interior node, so with g = u every boundary term, on every axis, must be
    moved to the right-hand side with its own bond coefficient."""
    n = 12
    m = n - 1
    rng = np.random.default_rng(3 + axis)
    prof = rng.uniform(0.1, 10.0, size=n)             # a at bonds k + 1/2, k = 0..n-1
    blocks = []
    for ax in range(dim):
        shape = [n if (dim - 1 - p) == ax else m for p in range(dim)]
        if ax == axis:
            view = [1] * dim
            view[dim - 1 - ax] = n
            blocks.append(np.broadcast_to(prof.reshape(view), shape).ravel())
        else:
            blocks.append(rng.uniform(0.1, 10.0, size=int(np.prod(shape))))
    a = np.concatenate(blocks)
    U = np.concatenate([[0.0], np.cumsum(1.0 / prof)])  # u at coordinates 0..n
    c = np.meshgrid(*[np.arange(n + 1)] * dim, indexing="ij")
    g = U[c[axis].transpose(*reversed(range(dim))).ravel()]
    rhs = stencil.rhs_from_bc(dim, n, a, g, np.zeros(m ** dim))
    x = spla.spsolve(stencil.assemble(dim, n, a, np.zeros(m ** dim)).tocsc(), rhs)
    ui = _interior(dim, n, g)
    assert np.abs(x - ui).max() <= 1e-11 * np.abs(ui).max()


def test_rhs_from_bc_zero_data_and_columns():
    dim, n = 2, 10
    a, b = inputs.high_contrast_coefficients(dim, n, seed=2, low=1e-2, high=1e2)
    f = np.arange(2 * (n - 1) ** dim, dtype=float).reshape(-1, 2)
    assert np.array_equal(stencil.rhs_from_bc(dim, n, a, np.zeros(((n + 1) ** dim, 2)), f), f)
    g = np.random.default_rng(0).standard_normal(((n + 1) ** dim, 2))
    both = stencil.rhs_from_bc(dim, n, a, g, f)
    for r in range(2):
        assert np.array_equal(both[:, r], stencil.rhs_from_bc(dim, n, a, g[:, r], f[:, r]))
