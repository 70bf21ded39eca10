"""The C-ABI library builds, loads and exports every entry point of
include/hif.h; argument errors come back as status codes (no GPU needed:
these calls return before any CUDA work), and on a machine without a GPU a
factorization with valid arguments fails cleanly at its first CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest
import torch

from paper_1307_2895_gb300 import hif

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hif.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|long long|const char\*)\s+(hif_\w+)\s*\(", src, re.M)))


def test_library_exports_header_symbols():
    lib = hif.load(build_if_missing=True)
    names = _declared()
    assert set(names) == set(hif.EXPORTS)
    for name in names:
        assert hasattr(lib, name), name


def test_argument_errors_without_gpu():
    lib = hif.load(build_if_missing=True)
    a, b = np.ones(2 * 16 * 15), np.zeros(225)
    h = ctypes.c_void_p()
    grid = hif._Grid(5, 16, 8, 1)
    rc = lib.hif_factor(ctypes.byref(grid), a.ctypes.data, b.ctypes.data, None, 1e-6, None, ctypes.byref(h))
    assert rc == hif.HIF_ERR_ARG and b"dim" in lib.hif_last_error()
    grid = hif._Grid(2, 16, 8, 1)
    rc = lib.hif_factor(ctypes.byref(grid), a.ctypes.data, b.ctypes.data, None, 0.0, None, ctypes.byref(h))
    assert rc == hif.HIF_ERR_ARG and b"eps" in lib.hif_last_error()
    rc = lib.hif_factor(ctypes.byref(grid), a.ctypes.data, b.ctypes.data, a.ctypes.data, 1e-6, None,
                        ctypes.byref(h))
    assert rc == hif.HIF_ERR_ARG
    assert lib.hif_apply(None, 1, None, None, 1, 1) == hif.HIF_ERR_ARG
    assert lib.hif_solve(None, None, None, None, 1, 1, 1e-12, 10, None) == hif.HIF_ERR_ARG
    st = hif._Stats()
    assert lib.hif_stats(None, ctypes.byref(st)) == hif.HIF_ERR_ARG
    lib.hif_free(None)


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1307_2895_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), f


def test_batch_argument_errors():
    """The batch entry points reject bad arguments before touching a GPU."""
    from paper_1307_2895_gb300 import hif
    lib = hif.load(build_if_missing=True)
    assert lib.hif_factor_batch(-1, None, None, None, None, None, 1, None) == hif.HIF_ERR_ARG
    assert lib.hif_solve_batch(-1, None, None, None, None, 1e-12, 10, None, 1) == hif.HIF_ERR_ARG
    assert lib.hif_factor_batch(0, None, None, None, None, None, 1, None) == 0


def test_schur_update_argument_errors_without_gpu():
    """hif_schur_update_f32 rejects bad sizes and splits before any CUDA call."""
    lib = hif.load(build_if_missing=True)
    assert lib.hif_schur_update_f32(1, 4, 4, None, None, 0, None) == hif.HIF_ERR_ARG
    assert lib.hif_schur_update_f32(1, 4, 4, None, None, 4, None) == hif.HIF_ERR_ARG
    assert lib.hif_schur_update_f32(-1, 4, 4, None, None, 3, None) == hif.HIF_ERR_ARG
    assert lib.hif_schur_update_f32(70000, 4, 4, None, None, 3, None) == hif.HIF_ERR_ARG
    assert lib.hif_schur_update_f32(1, 4, 4, None, None, 3, None) == hif.HIF_ERR_ARG   # NULL U
    assert lib.hif_schur_update_f32(3, 0, 4, None, None, 3, None) == hif.HIF_OK        # nothing to do


def test_estimate_and_solver_argument_errors_without_gpu():
    lib = hif.load(build_if_missing=True)
    ea, es = ctypes.c_double(), ctypes.c_double()
    assert lib.hif_estimate(None, None, 1e-2, 10, ctypes.byref(ea), ctypes.byref(es)) == hif.HIF_ERR_ARG
    assert lib.hif_set_solver(None, 0, 0) == hif.HIF_ERR_ARG


def test_autotune_table_without_gpu():
    lib = hif.load(build_if_missing=True)
    assert lib.hif_autotune_table(None, 0, None) == hif.HIF_ERR_ARG
    n = ctypes.c_longlong(-1)
    assert lib.hif_autotune_table(None, 0, ctypes.byref(n)) == hif.HIF_OK and n.value == 0



@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the failure path of a machine without a GPU")
def test_factor_failure_after_handle_creation_without_gpu():
    """Valid arguments on a machine without a GPU: the handle is created, the
    first CUDA call fails, and hif_factor frees the handle (its stream and
    events included) and returns HIF_ERR_CUDA with a NULL handle."""
    lib = hif.load(build_if_missing=True)
    n = 16
    a, b = np.ones(2 * n * (n - 1)), np.zeros((n - 1) ** 2)
    grid = hif._Grid(2, n, 8, 1)
    for _ in range(3):
        h = ctypes.c_void_p(1)
        rc = lib.hif_factor(ctypes.byref(grid), a.ctypes.data, b.ctypes.data, None, 1e-6, None, ctypes.byref(h))
        assert rc in (hif.HIF_ERR_CUDA, hif.HIF_ERR_OOM) and h.value is None
        assert lib.hif_last_error()


def test_factorization_context_manager_frees_once():
    """with ... as F frees the handle on exit (hif_free once), after which any
    use raises; a second free is a no-op."""
    calls = []

    class _Lib:
        def hif_free(self, h):
            calls.append(h)

    with hif.Factorization(ctypes.c_void_p(1234), _Lib(), 10) as F:
        assert F._live().value == 1234
    assert len(calls) == 1 and calls[0].value == 1234
    with pytest.raises(RuntimeError):
        F._live()
    F.free()
    assert len(calls) == 1


def test_binding_refuses_wrong_lengths_before_the_library():
    """The library reads as many elements as the grid implies; the binding
    raises ValueError for any other length before calling it."""
    n = 16
    a, b = np.ones(2 * n * (n - 1)), np.zeros((n - 1) ** 2)
    with pytest.raises(ValueError, match="a_stag"):
        hif.factor(2, n, a[:-1], b, 1e-6)
    with pytest.raises(ValueError, match="b has"):
        hif.factor(2, n, a, np.zeros((n - 1) ** 2 + 1), 1e-6)
    with pytest.raises(ValueError, match="rank_model"):
        hif.factor(2, n, a, b, 1e-6, id_mode="learned", rank_model=np.zeros(7, dtype=np.float32))
    with pytest.raises(ValueError, match="a_stag"):
        hif.factor_batch([(2, n, a, b), (2, n, a[:10], b)], 1e-6)
    with pytest.raises(ValueError, match="beta"):
        hif.factor(2, n, a, b, 1e-6, two_sided=True, beta=(1.0, 2.0, 3.0))

    class _NoLib:      # any library call would fail with AttributeError
        pass

    F = hif.Factorization(ctypes.c_void_p(1), _NoLib(), (n - 1) ** 2)
    bad = np.zeros(((n - 1) ** 2 + 3, 2))
    for call in (lambda: F.apply(bad), lambda: F.matvec(bad), lambda: F.solve(bad),
                 lambda: F.estimate(np.zeros(5)), lambda: F.solve(np.zeros((n - 1) ** 2), out=np.zeros(3))):
        with pytest.raises(ValueError):
            call()
    F._h = None        # nothing to free


def test_noalloc_refuses_host_pointers_without_gpu():
    """hif_residual_norms_noalloc dereferences its arrays on the device, so a
    host pointer is refused with HIF_ERR_ARG before any launch."""
    lib = hif.load(build_if_missing=True)
    n = 16
    a, b = np.ones(2 * n * (n - 1)), np.zeros((n - 1) ** 2)
    f = np.zeros(((n - 1) ** 2, 2))
    out = np.zeros(2)
    rc = lib.hif_residual_norms_noalloc(2, n, a.ctypes.data, b.ctypes.data, f.ctypes.data, f.ctypes.data, 2, 2,
                                        out.ctypes.data, None)
    assert rc == hif.HIF_ERR_ARG and b"not device memory" in lib.hif_last_error()


def test_noalloc_binding_refuses_host_arrays_and_wrong_lengths():
    n = 16
    a, b = np.ones(2 * n * (n - 1)), np.zeros((n - 1) ** 2)
    f = np.zeros(((n - 1) ** 2, 2))
    with pytest.raises(TypeError):
        hif.residual_norms_noalloc(2, n, a, b, f, f, np.zeros(2))


def test_wait_selftest_argument_errors_without_gpu():
    """hif_wait_selftest refuses an unknown wait and a bound outside 1 .. the
    real wait's own, before any CUDA call."""
    lib = hif.load(build_if_missing=True)
    assert lib.hif_wait_selftest(3, 100, None) == hif.HIF_ERR_ARG
    assert lib.hif_wait_selftest(0, 0, None) == hif.HIF_ERR_ARG
    assert lib.hif_wait_selftest(1, (1 << 22) + 1, None) == hif.HIF_ERR_ARG
    assert lib.hif_wait_selftest(2, 2_000_000_000, None) == hif.HIF_ERR_ARG


def test_sketch_power_argument_error_without_gpu():
    lib = hif.load(build_if_missing=True)
    a, b = np.ones(2 * 16 * 15), np.zeros(225)
    h = ctypes.c_void_p()
    grid = hif._Grid(2, 16, 8, 1)
    opts = hif._Opts(0, 0, 1, 10, None, None, 0, 0, 0, 0, 0, 3)
    rc = lib.hif_factor(ctypes.byref(grid), a.ctypes.data, b.ctypes.data, None, 1e-6, ctypes.byref(opts),
                        ctypes.byref(h))
    assert rc == hif.HIF_ERR_ARG and b"sketch_power" in lib.hif_last_error()


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding passes through the C ABI has the header's
    size and field offsets (a C++ program compiled with the host compiler
    prints them from include/hif.h)."""
    import shutil
    import subprocess
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    pairs = [("hif_grid", hif._Grid), ("hif_opts", hif._Opts), ("hif_solve_info", hif._SolveInfo),
             ("hif_stats_t", hif._Stats), ("hif_profile_t", hif._Profile)]
    lines = ['#include <cstddef>', '#include <cstdio>', '#include "hif.h"', 'int main() {']
    for cname, cls in pairs:
        lines.append(f'  std::printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  std::printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append('  return 0;\n}')
    src = tmp_path / "layout.cpp"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cxx, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in pairs:
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, f"{cname}.{fname}"
