"""Python binding of the C ABI in ``include/hif.h`` (argument marshalling only).

Every step of the factorization, the apply and the CG solve runs in the CUDA
library ``_lib/libhif.so``; this module only converts arguments.  Arrays may
be numpy arrays (host memory) or torch tensors (host or CUDA); results come
back in the same kind of container as the input vector.  There is no CPU
fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

HIF_OK, HIF_ERR_ARG, HIF_ERR_NOT_SPD, HIF_ERR_NOCONV, HIF_ERR_TIMEOUT, HIF_ERR_CUDA, HIF_ERR_OOM, HIF_ERR_HOST = range(8)
VARIANTS = {"mf": 0, "hifde": 1, "hifde3x": 2}
ID_MODES = {"qr": 0, "rand": 1, "learned": 2}
SKELS = {"id": 0, "svd": 1}
MLP_FEATURES, MLP_PARAMS = 10, 4929
SOLVERS = {"auto": 0, "cg": 1, "gmres": 2}
PRECISIONS = {"fp64": 0, "mixed": 1, "fp32_apply": 2}
APPLY_F, APPLY_FINV = 0, 1


class HifError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hif error {code}: {msg}")
        self.code = code


class _Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("leaf", ctypes.c_int), ("variant", ctypes.c_int)]


class _Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("skip_levels", ctypes.c_int), ("id_mode", ctypes.c_int),
                ("oversample", ctypes.c_int), ("stream", ctypes.c_void_p), ("rank_model", ctypes.c_void_p),
                ("seed", ctypes.c_ulonglong), ("big_cell", ctypes.c_int), ("tensor_cores", ctypes.c_int),
                ("autotune", ctypes.c_int), ("edge_start", ctypes.c_int), ("sketch_power", ctypes.c_int),
                ("deterministic", ctypes.c_int), ("big_apply", ctypes.c_longlong), ("skel", ctypes.c_int),
                ("two_sided", ctypes.c_int), ("beta", ctypes.c_double * 3)]


class _SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer", ctypes.c_int), ("converged", ctypes.c_int),
                ("relres_max", ctypes.c_double), ("relres_fp64_max", ctypes.c_double),
                ("gmres_iters", ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("levels", ctypes.c_int),
                ("root_size", ctypes.c_int), ("n_cells", ctypes.c_int), ("n_fronts", ctypes.c_int),
                ("max_front_rank", ctypes.c_int), ("near_threshold_fronts", ctypes.c_int),
                ("clamped_pivots", ctypes.c_int), ("sketched_fronts", ctypes.c_int),
                ("fallback_fronts", ctypes.c_int), ("t_fronts_ms", ctypes.c_double),
                ("factor_bytes", ctypes.c_longlong), ("factor_flops", ctypes.c_double),
                ("apply_bytes", ctypes.c_double), ("t_factor_ms", ctypes.c_double),
                ("negative_pivots", ctypes.c_int), ("t_wall_ms", ctypes.c_double), ("t_wait_ms", ctypes.c_double)]


class _Profile(ctypes.Structure):
    _fields_ = [("sweep_ms", ctypes.c_double), ("sweep_launches", ctypes.c_longlong),
                ("sweep_bytes", ctypes.c_double)]


_LIB = None
EXPORTS = ["hif_factor", "hif_apply", "hif_solve", "hif_matvec", "hif_rhs_from_bc", "hif_stats", "hif_structure",
           "hif_profile", "hif_kernel_launches", "hif_residual_norms_noalloc", "hif_front_log", "hif_mlp_grad",
           "hif_mlp_train", "hif_mlp_predict", "hif_schur_update_f32", "hif_factor_batch", "hif_solve_batch",
           "hif_set_solver", "hif_estimate", "hif_autotune_table", "hif_wait_selftest", "hif_free", "hif_last_error"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load ``libhif.so`` (raises if it is not built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: build it with paper_1307_2895_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.hif_factor.argtypes = [ctypes.POINTER(_Grid), vp, vp, vp, d, ctypes.POINTER(_Opts), ctypes.POINTER(vp)]
    lib.hif_factor.restype = i
    lib.hif_apply.argtypes = [vp, i, vp, vp, i, i]
    lib.hif_apply.restype = i
    lib.hif_solve.argtypes = [vp, vp, vp, vp, i, i, d, i, ctypes.POINTER(_SolveInfo)]
    lib.hif_solve.restype = i
    lib.hif_matvec.argtypes = [vp, vp, vp, i, i]
    lib.hif_matvec.restype = i
    lib.hif_rhs_from_bc.argtypes = [ctypes.POINTER(_Grid), vp, vp, vp, i, i]
    lib.hif_rhs_from_bc.restype = i
    lib.hif_stats.argtypes = [vp, ctypes.POINTER(_Stats)]
    lib.hif_stats.restype = i
    lib.hif_structure.argtypes = [vp, vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]
    lib.hif_structure.restype = i
    lib.hif_profile.argtypes = [vp, i, ctypes.POINTER(_Profile)]
    lib.hif_profile.restype = i
    lib.hif_kernel_launches.argtypes = []
    lib.hif_kernel_launches.restype = ctypes.c_longlong
    lib.hif_wait_selftest.argtypes = [i, ctypes.c_longlong, vp]
    lib.hif_wait_selftest.restype = i
    lib.hif_residual_norms_noalloc.argtypes = [i, i, vp, vp, vp, vp, i, i, vp, vp]
    lib.hif_residual_norms_noalloc.restype = i
    lib.hif_front_log.argtypes = [vp, vp, vp, vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]
    lib.hif_front_log.restype = i
    lib.hif_mlp_grad.argtypes = [vp, vp, i, vp, vp, vp, vp]
    lib.hif_mlp_grad.restype = i
    lib.hif_mlp_train.argtypes = [vp, vp, i, vp, i, i, ctypes.c_float, ctypes.c_ulonglong, vp, vp]
    lib.hif_mlp_train.restype = i
    lib.hif_mlp_predict.argtypes = [vp, i, vp, vp, vp]
    lib.hif_mlp_predict.restype = i
    lib.hif_schur_update_f32.argtypes = [i, i, i, vp, vp, i, vp]
    lib.hif_schur_update_f32.restype = i
    lib.hif_factor_batch.argtypes = [i, ctypes.POINTER(_Grid), vp, vp, vp, ctypes.POINTER(_Opts), i, vp]
    lib.hif_factor_batch.restype = i
    lib.hif_solve_batch.argtypes = [i, vp, vp, vp, vp, d, i, ctypes.POINTER(_SolveInfo), i]
    lib.hif_solve_batch.restype = i
    lib.hif_set_solver.argtypes = [vp, i, i]
    lib.hif_set_solver.restype = i
    lib.hif_estimate.argtypes = [vp, vp, d, i, ctypes.POINTER(d), ctypes.POINTER(d)]
    lib.hif_estimate.restype = i
    lib.hif_autotune_table.argtypes = [vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]
    lib.hif_autotune_table.restype = i
    lib.hif_free.argtypes = [vp]
    lib.hif_free.restype = None
    lib.hif_last_error.argtypes = []
    lib.hif_last_error.restype = ctypes.c_char_p
    _LIB = lib
    return lib


def _check(rc: int, lib) -> None:
    if rc != HIF_OK:
        raise HifError(rc, lib.hif_last_error().decode())


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype: str = "float64"):
    """Raw address of a contiguous numpy array or torch tensor of the given dtype."""
    if x is None:
        return None
    if _is_torch(x):
        import torch
        if x.dtype != getattr(torch, dtype) or not x.is_contiguous():
            raise TypeError(f"tensors must be contiguous {dtype}")
        return x.data_ptr()
    if x.dtype != np.dtype(dtype) or not x.flags["C_CONTIGUOUS"]:
        raise TypeError(f"arrays must be C-contiguous {dtype}")
    return x.ctypes.data


def _as_2d(x):
    return x.reshape(x.shape[0], -1)


def _numel(x) -> int:
    return int(x.numel()) if _is_torch(x) else int(np.size(x))


def _need(x, count: int, what: str) -> None:
    """The library reads `count` elements from x: refuse any other length."""
    if x is not None and _numel(x) != count:
        raise ValueError(f"{what} has {_numel(x)} elements, expected {count}")


def _need_problem(dim: int, n: int, a_stag, b) -> None:
    if dim in (2, 3) and n >= 2:
        _need(a_stag, dim * n * (n - 1) ** (dim - 1), "a_stag")
        _need(b, (n - 1) ** dim, "b")


def _need_rows(x2, N: int, what: str) -> None:
    if x2.shape[0] != N:
        raise ValueError(f"{what} has {x2.shape[0]} rows, expected N = {N}")


def _empty_like(x, shape):
    if _is_torch(x):
        import torch
        return torch.empty(shape, dtype=torch.float64, device=x.device)
    return np.empty(shape, dtype=np.float64)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Factorization:
    """Handle of one factorization (``hif_factor``); free with :meth:`free`, or
    use it as a context manager (``with hif.factor(...) as F:``)."""

    def __init__(self, handle, lib, N: int):
        self._h = handle
        self._lib = lib
        self.N = N

    def _live(self):
        if not self._h:
            raise RuntimeError("factorization already freed")
        return self._h

    def apply(self, x, inverse: bool = True):
        """y = F^-1 x (inverse=True) or F x; x has shape (N,) or (N, nrhs)."""
        x2 = _as_2d(x)
        _need_rows(x2, self.N, "x")
        y = _empty_like(x, x2.shape)
        rc = self._lib.hif_apply(self._live(), APPLY_FINV if inverse else APPLY_F, _ptr(x2), _ptr(y),
                                 x2.shape[1], x2.shape[1])
        _check(rc, self._lib)
        return y.reshape(x.shape)

    def matvec(self, x):
        x2 = _as_2d(x)
        _need_rows(x2, self.N, "x")
        y = _empty_like(x, x2.shape)
        _check(self._lib.hif_matvec(self._live(), _ptr(x2), _ptr(y), x2.shape[1], x2.shape[1]), self._lib)
        return y.reshape(x.shape)

    def estimate(self, x0, rtol: float = 1e-2, maxit: int = 200):
        """hif_estimate: (e_a, e_s) by power iteration from x0 (Section 5)."""
        _need(x0, self.N, "x0")
        ea, es = ctypes.c_double(), ctypes.c_double()
        _check(self._lib.hif_estimate(self._live(), _ptr(x0), rtol, maxit, ctypes.byref(ea), ctypes.byref(es)),
               self._lib)
        return ea.value, es.value

    def set_solver(self, solver: str = "auto", restart: int = 0) -> None:
        """hif_set_solver: inner solver of later solves ("auto": CG with a
        GMRES fallback on breakdown, "cg", "gmres"), GMRES restart length."""
        _check(self._lib.hif_set_solver(self._live(), SOLVERS[solver], restart), self._lib)

    def solve(self, rhs, tol: float = 1e-12, maxit: int = 200, raise_on_noconv: bool = False,
              want_lo: bool = False, out=None):
        """PCG (or GMRES, see set_solver) with F^-1 as preconditioner
        (double-double refinement); returns
        (x, info dict) or (x_hi, x_lo, info) with ``want_lo``.  ``out`` (same
        shape as rhs, contiguous float64) receives x if given."""
        r2 = _as_2d(rhs)
        _need_rows(r2, self.N, "rhs")
        _need(out, self.N * r2.shape[1], "out")
        x = _empty_like(rhs, r2.shape) if out is None else out.reshape(r2.shape)
        xlo = _empty_like(rhs, r2.shape) if want_lo else None
        info = _SolveInfo()
        rc = self._lib.hif_solve(self._live(), _ptr(r2), _ptr(x), _ptr(xlo), r2.shape[1], r2.shape[1], tol,
                                 maxit, ctypes.byref(info))
        if rc != HIF_ERR_NOCONV or raise_on_noconv:
            _check(rc, self._lib)
        d = dict(iters=info.iters, outer=info.outer, converged=bool(info.converged),
                 relres_max=info.relres_max, relres_fp64_max=info.relres_fp64_max, gmres_iters=info.gmres_iters)
        if want_lo:
            return x.reshape(rhs.shape), xlo.reshape(rhs.shape), d
        return x.reshape(rhs.shape), d

    def profile(self, enable: bool = True) -> dict:
        """Sweep timing since the previous call (then reset); toggles recording."""
        p = _Profile()
        _check(self._lib.hif_profile(self._live(), 1 if enable else 0, ctypes.byref(p)), self._lib)
        return dict(sweep_ms=p.sweep_ms, sweep_launches=p.sweep_launches, sweep_bytes=p.sweep_bytes)

    def front_log(self):
        """(features n x 10, ranks, sizes) of every front: rank-MLP training data."""
        cnt = ctypes.c_longlong(0)
        _check(self._lib.hif_front_log(self._live(), None, None, None, 0, ctypes.byref(cnt)), self._lib)
        n = cnt.value
        feats = np.zeros((n, MLP_FEATURES), dtype=np.float32)
        ranks = np.zeros(n, dtype=np.int32)
        sizes = np.zeros(n, dtype=np.int32)
        _check(self._lib.hif_front_log(self._live(), feats.ctypes.data, ranks.ctypes.data, sizes.ctypes.data, n,
                                       ctypes.byref(cnt)), self._lib)
        return feats, ranks, sizes

    def stats(self) -> dict:
        s = _Stats()
        _check(self._lib.hif_stats(self._live(), ctypes.byref(s)), self._lib)
        return {name: getattr(s, name) for name, _ in _Stats._fields_}

    def structure(self):
        """[(level, c, skeletons in pivot order)], |s_L|."""
        need = ctypes.c_longlong(0)
        _check(self._lib.hif_structure(self._live(), None, 0, ctypes.byref(need)), self._lib)
        buf = np.zeros(need.value, dtype=np.int32)
        _check(self._lib.hif_structure(self._live(), buf.ctypes.data, need.value, ctypes.byref(need)),
               self._lib)
        out, p = [], 0
        while buf[p] != -1:
            lev, nc, k = int(buf[p]), int(buf[p + 1]), int(buf[p + 2])
            p += 3
            c = buf[p:p + nc].tolist()
            p += nc
            sk = buf[p:p + k].tolist()
            p += k
            out.append((lev, c, sk))
        return out, int(buf[p + 1])

    def free(self) -> None:
        if self._h:
            self._lib.hif_free(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc) -> None:
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def residual_norms_noalloc(dim: int, n: int, a_stag, b, f, x, out, stream=None) -> None:
    """hif_residual_norms_noalloc on CUDA tensors: out[r] = ||f_r - A x_r||^2.
    Allocates nothing on the device (the library's fixed scratch is used)."""
    lib = load()
    for v, what in ((a_stag, "a_stag"), (b, "b"), (f, "f"), (x, "x"), (out, "out")):
        if not (_is_torch(v) and v.is_cuda):
            raise TypeError(f"{what} must be a CUDA tensor (this entry point stages nothing)")
    f2, x2 = _as_2d(f), _as_2d(x)
    _need_problem(dim, n, a_stag, b)
    if dim in (2, 3) and n >= 2:
        _need_rows(f2, (n - 1) ** dim, "f")
    if tuple(x2.shape) != tuple(f2.shape):
        raise ValueError(f"x has shape {tuple(x2.shape)}, f has {tuple(f2.shape)}")
    _need(out, f2.shape[1], "out")
    rc = lib.hif_residual_norms_noalloc(dim, n, _ptr(a_stag), _ptr(b), _ptr(f2), _ptr(x2), f2.shape[1],
                                        f2.shape[1], _ptr(out), _stream_ptr(stream))
    _check(rc, lib)


def wait_selftest(which: str, limit: int, stream=None) -> None:
    """hif_wait_selftest: run one bounded device wait ("bulk", "group" or
    "mma") on an object nothing completes; raises HifError (HIF_ERR_TIMEOUT
    when the wait gave up, as it should)."""
    lib = load()
    _check(lib.hif_wait_selftest({"bulk": 0, "group": 1, "mma": 2}[which], int(limit), _stream_ptr(stream)), lib)


def kernel_launches() -> int:
    """Kernels launched by the CUDA library so far in this process."""
    return int(load().hif_kernel_launches())


def mlp_grad(X, target, params, stream=None):
    """(loss, grad) of the rank MLP on CUDA float32 tensors."""
    import torch
    lib = load()
    grad = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    rc = lib.hif_mlp_grad(_ptr(X, "float32"), _ptr(target, "float32"), X.shape[0], _ptr(params, "float32"),
                          _ptr(grad, "float32"), _ptr(loss, "float32"), _stream_ptr(stream))
    _check(rc, lib)
    return float(loss.item()), grad


def mlp_train(X, target, params, steps: int = 2000, batch: int = 1024, lr: float = 1e-3, seed: int = 0,
              stream=None):
    """Train the rank MLP in place (CUDA float32 tensors); returns the loss history."""
    import torch
    lib = load()
    hist = torch.empty(max(steps, 1), dtype=torch.float32, device=params.device)
    rc = lib.hif_mlp_train(_ptr(X, "float32"), _ptr(target, "float32"), X.shape[0], _ptr(params, "float32"),
                           steps, batch, lr, seed, _ptr(hist, "float32"), _stream_ptr(stream))
    _check(rc, lib)
    return hist[:steps].cpu().numpy()


def mlp_predict(X, params, stream=None):
    """BF16-weight inference of the rank MLP (CUDA float32 tensors)."""
    import torch
    lib = load()
    y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    _check(lib.hif_mlp_predict(_ptr(X, "float32"), X.shape[0], _ptr(params, "float32"), _ptr(y, "float32"),
                               _stream_ptr(stream)), lib)
    return y


def autotune_table():
    """hif_autotune_table: rows (op, elem_bytes, nrhs, nblocks, max_np, max_nq,
    is_front, threads, staged) of the sweep shapes chosen so far."""
    lib = load()
    n = ctypes.c_longlong()
    _check(lib.hif_autotune_table(None, 0, ctypes.byref(n)), lib)
    buf = np.zeros((max(n.value, 1), 9), dtype=np.int32)
    _check(lib.hif_autotune_table(buf.ctypes.data, n.value, ctypes.byref(n)), lib)
    return buf[:n.value]


def schur_update(G, U, split: int = 3, stream=None):
    """hif_schur_update_f32: U_b -= G_b G_b^T in place on the tensor cores
    (CUDA float32 tensors G of shape (nb, m, k) and U of shape (nb, m, m))."""
    lib = load()
    nb, m, k = G.shape
    if tuple(U.shape) != (nb, m, m):
        raise ValueError("U must have shape (nb, m, m)")
    _check(lib.hif_schur_update_f32(nb, m, k, _ptr(G, "float32"), _ptr(U, "float32"), split,
                                    _stream_ptr(stream)), lib)
    return U


def rhs_from_bc(dim: int, n: int, a_stag, bc_vals, f):
    """hif_rhs_from_bc: ``f`` plus the stencil's boundary terms for nonzero
    Dirichlet values.  ``bc_vals``: values at all ``(n+1)^dim`` grid nodes
    (coordinates 0..n, x fastest; only boundary nodes are read), shape
    ``((n+1)^dim,)`` or ``((n+1)^dim, nrhs)``; ``f``: ``(N,)`` or ``(N, nrhs)``.
    Host arrays (numpy, or CPU tensors); returns a new float64 numpy array of
    ``f``'s shape, the right-hand side of the problem with those boundary values."""
    lib = load()
    N = (n - 1) ** dim
    f_np = np.asarray(f.cpu() if _is_torch(f) else f, dtype=np.float64)
    out = np.array(f_np, dtype=np.float64, order="C", copy=True).reshape(N, -1)
    g = np.ascontiguousarray(bc_vals.cpu() if _is_torch(bc_vals) else bc_vals, dtype=np.float64)
    g = g.reshape((n + 1) ** dim, -1)
    a = np.ascontiguousarray(a_stag.cpu() if _is_torch(a_stag) else a_stag, dtype=np.float64).ravel()
    if a.size != dim * n * (n - 1) ** (dim - 1):
        raise ValueError("a_stag has the wrong length")
    if g.shape[1] != out.shape[1]:
        raise ValueError("bc_vals and f need the same number of columns")
    grid = _Grid(dim, n, 8, VARIANTS["hifde"])
    _check(lib.hif_rhs_from_bc(ctypes.byref(grid), a.ctypes.data, g.ctypes.data, out.ctypes.data, out.shape[1],
                               out.shape[1]), lib)
    return out.reshape(f_np.shape)


def factor(dim: int, n: int, a_stag, b, eps: float, variant: str = "hifde", precision: str = "fp64",
           leaf: int = 8, skip_levels: int = 0, stream=None, id_mode: str = "qr", rank_model=None,
           oversample: int = 10, seed: int = 0, big_cell: int = 0, tensor_cores: int = 0,
           autotune: bool = True, edge_start: int = 1, sketch_power: int = 0,
           deterministic: bool = False, big_apply: int = 0, skel: str = "id", two_sided: bool = False,
           beta=None) -> Factorization:
    """hif_factor: MF or HIF-DE of the stencil operator defined by (a_stag, b).
    tensor_cores (mixed precision): 0 three-part TF32 split (about FP32),
    2 two-part, 1 plain TF32, -1 FP32 on the SIMT pipes.  edge_start
    (hifde3x): the first level whose edges are skeletonized.  sketch_power:
    power iterations on the randomized ID's sketch.  deterministic:
    bit-reproducible applications (no floating-point atomics in the sweeps).
    big_apply: F^-1 applies blocks of at least this many factor elements
    (np (np + 2 nq)) with many thread blocks each (0: 2^20, -1: never).
    skel: the fronts' low-rank approximation, "id" (Lemma 2.2) or "svd"
    (Section 4.4).  two_sided: the unsymmetric variant (LU elimination, one
    ID of [A_{N,c}; A_{c,N}^T]) of the stencil plus the convection term
    beta . grad u (beta: dim values, two_sided only)."""
    lib = load()
    _need_problem(dim, n, a_stag, b)
    _need(rank_model, MLP_PARAMS, "rank_model")
    grid = _Grid(dim, n, leaf, VARIANTS[variant])
    if edge_start < 0:
        raise ValueError("edge_start must be >= 0")
    if beta is not None:
        beta = [float(v) for v in beta]
        if len(beta) != dim:
            raise ValueError(f"beta has {len(beta)} values, the grid has {dim} axes")
    opts = _Opts(PRECISIONS[precision], skip_levels, ID_MODES[id_mode], oversample, _stream_ptr(stream),
                 _ptr(rank_model, "float32"), seed, big_cell, tensor_cores, 0 if autotune else -1,
                 -1 if edge_start == 0 else edge_start, sketch_power, 1 if deterministic else 0, int(big_apply),
                 SKELS[skel], 1 if two_sided else 0,
                 (ctypes.c_double * 3)(*(list(beta) + [0.0] * (3 - len(beta))) if beta is not None else (0.0,) * 3))
    h = ctypes.c_void_p()
    rc = lib.hif_factor(ctypes.byref(grid), _ptr(a_stag), _ptr(b), None, float(eps), ctypes.byref(opts),
                        ctypes.byref(h))
    _check(rc, lib)
    return Factorization(h, lib, (n - 1) ** dim)


def factor_batch(problems, eps: float, variant: str = "hifde", precision: str = "fp64", leaf: int = 8,
                 nthreads: int = 8, big_cell: int = 0, tensor_cores: int = 0, autotune: bool = True):
    """hif_factor_batch: problems = [(dim, n, a_stag, b), ...], factored
    concurrently (one stream each); returns one Factorization per problem."""
    lib = load()
    m = len(problems)
    for d, n, a, b in problems:
        _need_problem(d, n, a, b)
    grids = (_Grid * m)(*[_Grid(d, n, leaf, VARIANTS[variant]) for d, n, _, _ in problems])
    pa = (ctypes.c_void_p * m)(*[_ptr(a) for _, _, a, _ in problems])
    pb = (ctypes.c_void_p * m)(*[_ptr(b) for _, _, _, b in problems])
    pe = (ctypes.c_double * m)(*([float(eps)] * m))
    opts = _Opts(PRECISIONS[precision], 0, ID_MODES["qr"], 10, None, None, 0, big_cell, tensor_cores,
                 0 if autotune else -1)
    hs = (ctypes.c_void_p * m)()
    rc = lib.hif_factor_batch(m, grids, pa, pb, pe, ctypes.byref(opts), nthreads, hs)
    facts = [Factorization(ctypes.c_void_p(hs[p]), lib, (problems[p][1] - 1) ** problems[p][0]) if hs[p] else None
             for p in range(m)]
    if rc != 0:
        for F in facts:
            if F is not None:
                F.free()
        _check(rc, lib)
    return facts


def solve_batch(facts, rhs_list, tol: float = 1e-12, maxit: int = 1000, nthreads: int = 8):
    """hif_solve_batch: one (N, nrhs) float64 right-hand side array per
    factorization, solved concurrently; returns [(x, info dict), ...]."""
    lib = load()
    m = len(facts)
    if len(rhs_list) != m:
        raise ValueError("one right-hand side array per factorization")
    r2 = [_as_2d(r) for r in rhs_list]
    for F, q in zip(facts, r2):
        _need_rows(q, F.N, "rhs")
    xs = [_empty_like(r, q.shape) for r, q in zip(rhs_list, r2)]
    hs = (ctypes.c_void_p * m)(*[F._live() for F in facts])
    pr = (ctypes.c_void_p * m)(*[_ptr(q) for q in r2])
    px = (ctypes.c_void_p * m)(*[_ptr(x) for x in xs])
    pn = (ctypes.c_int * m)(*[q.shape[1] for q in r2])
    infos = (_SolveInfo * m)()
    rc = lib.hif_solve_batch(m, hs, pr, px, pn, tol, maxit, infos, nthreads)
    if rc != HIF_ERR_NOCONV:
        _check(rc, lib)
    out = []
    for p in range(m):
        i = infos[p]
        out.append((xs[p].reshape(rhs_list[p].shape),
                    dict(iters=i.iters, outer=i.outer, converged=bool(i.converged), relres_max=i.relres_max,
                         relres_fp64_max=i.relres_fp64_max, gmres_iters=i.gmres_iters)))
    return out
