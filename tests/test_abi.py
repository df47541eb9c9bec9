"""The C-ABI library builds, loads without a GPU, and exports every entry point
include/bmg.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "bmg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bmg_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__
    return __graft_entry__._builder().build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("bmg_setup", "bmg_solve", "bmg_free", "bmg_history", "bmg_dendy_interp", "bmg_rap",
                 "bmg_relax", "bmg_resid_restrict", "bmg_interp_correct", "bmg_residual",
                 "bmg_coarse_factor", "bmg_coarse_solve", "bmg_inner_cycle"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_imports_and_reports_errors_without_gpu(libpath):
    import paper_2502_05279_gb300 as bmg
    assert bmg.lib.bmg_strerror(-6).decode() == "not converged within maxit"
    assert bmg.lib.bmg_strerror(0).decode() == "ok"
    # argument validation happens on the host, before any CUDA call
    h = ctypes.c_void_p()
    st = bmg._lib.Stencil(9, None)
    assert bmg.lib.bmg_setup(ctypes.byref(st), 127, 127, None, ctypes.byref(h)) == bmg._lib.BMG_EINVAL
    st = bmg._lib.Stencil(7, ctypes.c_void_p(16))
    assert bmg.lib.bmg_setup(ctypes.byref(st), 127, 127, None, ctypes.byref(h)) == bmg._lib.BMG_EINVAL
    st = bmg._lib.Stencil(9, ctypes.c_void_p(16))
    # any 1 <= nx, ny <= 65535 is a valid grid (embedded in the next 2^m - 1 square); outside that range
    # the call fails before touching the device
    for nx, ny in ((0, 0), (-1, 5), (5, 0), (65536, 3), (3, 70000)):
        assert bmg.lib.bmg_setup(ctypes.byref(st), nx, ny, None, ctypes.byref(h)) == bmg._lib.BMG_EINVAL
        assert "outside" in bmg.lib.bmg_last_error().decode()
    o = bmg._lib.Opts()
    for bad in (15, 99, -1):   # valid: 0 auto, 1 rows, 2 .. 7 one-pass, 8 .. 11 two-sweep shapes, 12 .. 14 lines
        o.smoother = bad
        assert bmg.lib.bmg_setup(ctypes.byref(st), 127, 127, ctypes.byref(o), ctypes.byref(h)) == bmg._lib.BMG_EINVAL
        assert "smoother" in bmg.lib.bmg_last_error().decode()
    assert bmg.lib.bmg_solve(None, None, None, 1e-10, 10, None, None) == bmg._lib.BMG_EINVAL
    bmg.lib.bmg_free(None)


def test_batched_setup_validates_on_the_host(libpath):
    """bmg_setup_batched rejects bad batches before any device work: no
    problems, a size that is not 2^m - 1, mixed stencil kinds, Krylov
    acceleration, line relaxation, one-pass shapes above 3, two-sweep passes
    in FP64, and an unknown arithmetic mode; the handle stays NULL."""
    import paper_2502_05279_gb300 as bmg
    L = bmg._lib
    B = ctypes.c_void_p()
    nine = (L.Stencil * 2)(L.Stencil(9, ctypes.c_void_p(16)), L.Stencil(9, ctypes.c_void_p(32)))
    mixed = (L.Stencil * 2)(L.Stencil(9, ctypes.c_void_p(16)), L.Stencil(5, ctypes.c_void_p(32)))
    sizes = (ctypes.c_int * 2)(63, 127)

    def opts(**kw):
        o = L.Opts()
        for k, v in kw.items():
            setattr(o, k, v)
        return ctypes.byref(o)

    cases = [(0, nine, sizes, None, "bad argument"),
             (2, nine, (ctypes.c_int * 2)(63, 100), None, "2^m - 1"),
             (2, mixed, sizes, None, "differ in kind"),
             (2, nine, sizes, opts(krylov=1), "stationary"),
             (2, nine, sizes, opts(smoother=12), "line relaxation"),
             (2, nine, sizes, opts(smoother=6), "bad smoother"),
             (2, nine, sizes, opts(smoother=8), "FP32 only"),
             (2, nine, sizes, opts(arith=3), "bad arith")]
    for nprob, st, n, o, msg in cases:
        assert L.lib.bmg_setup_batched(nprob, st, n, o, ctypes.byref(B)) == L.BMG_EINVAL
        assert msg in L.lib.bmg_last_error().decode()
        assert B.value is None


def test_binding_checks_sizes_before_the_library(libpath):
    """The C ABI takes bare pointers, so the binding refuses tensors smaller
    than what the library would read or write through them, and too few or
    too many per-problem tensors for a batch, before any call."""
    import torch
    import paper_2502_05279_gb300 as bmg
    z = lambda *s: torch.zeros(s, dtype=torch.float64)
    with pytest.raises(ValueError, match="coef holds"):
        bmg.Hierarchy(9, z(3, 17, 17))                 # a 9-point stencil needs 5 planes
    with pytest.raises(ValueError, match="CUDA"):
        bmg.Hierarchy(5, z(3, 17, 17))                 # sizes fine: stops at the device check
    h = bmg.Hierarchy.__new__(bmg.Hierarchy)
    h.nx, h.ny, h.n, h._h = 20, 10, 31, None
    with pytest.raises(ValueError, match="rhs holds 252 values; 264 are needed"):
        h.solve(z(12, 21))
    with pytest.raises(ValueError, match="x holds"):
        h.time_cycles(z(12, 22), z(12, 21), 1)
    with pytest.raises(ValueError, match="r32 holds"):
        h.inner_cycle(torch.zeros((33, 32), dtype=torch.float32))
    b = bmg.Batch.__new__(bmg.Batch)
    b.ns, b._h = [7, 15], None
    with pytest.raises(ValueError, match="1 rhs tensors for 2 problems"):
        b.solve([z(9, 9)])
    with pytest.raises(ValueError, match="rhs holds 81 values; 289 are needed"):
        b.time_cycles([z(9, 9), z(9, 9)], [z(9, 9), z(17, 17)], 1)
    with pytest.raises(ValueError, match="coef holds"):
        bmg.relax(9, z(3, 9, 9), z(9, 9), z(9, 9))
    with pytest.raises(ValueError, match="f holds"):
        bmg.residual(5, z(3, 9, 9), z(9, 9), z(9, 8))
    with pytest.raises(ValueError, match="ci holds"):
        bmg.rap(z(5, 9, 9), z(8, 4, 4))
    with pytest.raises(ValueError, match="ec holds"):
        bmg.interp_correct(z(8, 5, 5), z(4, 5), z(9, 9))
    with pytest.raises(ValueError, match="L holds"):
        bmg.coarse_solve(z(8, 10), z(5, 5), z(5, 5))   # n = 3: L is 9 x 9


def test_release_library_has_no_debug_checks(libpath):
    """libbmg.so compiles every device bounds check to the constant true: it
    reports itself as a release build, never holds a record, and refuses the
    debug builds' test hook (no device call is made for any of this)."""
    import paper_2502_05279_gb300 as bmg
    assert not bmg.debug_build()
    assert bmg.debug_take() is None
    with pytest.raises(bmg.BmgError) as e:
        bmg.debug_shrink(1)
    assert e.value.code == bmg._lib.BMG_EINVAL
    assert bmg.lib.bmg_strerror(-8).decode() == "debug bounds check failed"
    assert bmg.lib.bmg_debug_site_name(1).decode() == "point Gauss-Seidel store"


def test_header_is_a_c_abi(libpath, tmp_path):
    """include/bmg.h compiles as strict C99 (-pedantic -Werror) and a C program
    links against the library and makes the calls that need no GPU."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "c_abi_check")
    libdir = os.path.dirname(libpath)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c_abi_check.c"), "-L", libdir, "-lbmg", f"-Wl,-rpath,{libdir}",
                        "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("ok ") == 7
