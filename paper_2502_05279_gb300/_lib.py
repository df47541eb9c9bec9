"""ctypes binding of libbmg.so.  Argument marshalling only: every step of the
solver runs in the library's CUDA kernels.  With the environment variable
BMG_LIB=debug at import the binding loads libbmg_debug.so instead (the same
library with device bounds checks, built by build.build(debug=True)).

Tensors passed in must be contiguous CUDA tensors of the documented dtype and
shape; work is enqueued on torch's current CUDA stream, with which the library
orders itself.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libbmg_debug.so" if os.environ.get("BMG_LIB") == "debug" else "libbmg.so")

BMG_OK, BMG_EINVAL, BMG_ENOMEM, BMG_ECUDA, BMG_ESINGULAR, BMG_ENAN, BMG_ENOTCONV, BMG_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7
BMG_EBOUNDS = -8
BMG_FP64, BMG_FP32_IR, BMG_BF16_IR = 0, 1, 2
BMG_PERIODIC_X, BMG_PERIODIC_Y = 1, 2
_PREC = {"fp64": BMG_FP64, "fp32": BMG_FP32_IR, "bf16": BMG_BF16_IR}


class BmgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


if not os.path.exists(library_path):
    raise ImportError(f"{library_path} is missing: build it with paper_2502_05279_gb300.build.build() "
                      "(debug=True for libbmg_debug.so; there is no CPU fallback)")
lib = ctypes.CDLL(library_path)


class Stencil(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("coef", ctypes.c_void_p)]


class ProfRow(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("kernel", ctypes.c_int), ("fp32", ctypes.c_int),
                ("launches", ctypes.c_int), ("ms", ctypes.c_double)]


KERNEL_NAMES = ("relax", "resid_restrict", "interp_correct", "coarse_solve", "residual_norm", "norm_finalize",
                "ir_update", "ir_residual", "fcg", "tail", "relax_pair", "pair_restrict")
_KRYLOV = {"none": 0, "fcg": 1}
# the two pre-smoothing sweeps with the residual and restriction in one pass (BMG_FUSE_*)
_FUSE = {"auto": 0, "off": 1, "on": 2}
# right-hand sides per warp in the one-pass sweeps of a batch of right-hand sides (BMG_RHS_BLOCK_*)
_RHS_BLOCK = {"auto": 0, "off": 1, 2: 2, 4: 4}
# Gauss-Seidel kernel of the FP32 cycle's 9-point levels (all compute the same bits)
_SMOOTHER = {"auto": 0, "rows": 1, "tile": 2, **{f"tile{k}": 2 + k for k in range(6)},
             "pair": 8, **{f"pair{k}": 8 + k for k in range(4)}, "line": 12, "yline": 13,
             "xyline": 14}
TILE_SWEEP = 16   # bmg_tuned_cluster value of tile shape 0 (shape s: 16 + s)
# cycle arithmetic: one rounding per operation, or fused multiply-adds
_ARITH = {"rounded": 0, "fused": 1}


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("interp", ctypes.c_int), ("coarsest", ctypes.c_int),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("inner_cycles", ctypes.c_int),
                ("bf16_levels", ctypes.c_int), ("use_graph", ctypes.c_int), ("krylov", ctypes.c_int),
                ("mlp", ctypes.c_void_p), ("stream", ctypes.c_void_p), ("smoother", ctypes.c_int),
                ("arith", ctypes.c_int), ("fuse_restrict", ctypes.c_int), ("rhs_block", ctypes.c_int),
                ("periodic", ctypes.c_int)]


P, I, D, L = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
_sig = {
    "bmg_setup": (I, [ctypes.POINTER(Stencil), I, I, ctypes.POINTER(Opts), ctypes.POINTER(P)]),
    "bmg_solve": (I, [P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D)]),
    "bmg_history": (I, [P, ctypes.POINTER(D), I]),
    "bmg_num_levels": (I, [P]),
    "bmg_level_size": (I, [P, I]),
    "bmg_level_shape": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
    "bmg_get_stencil": (I, [P, I, P]),
    "bmg_get_interp": (I, [P, I, P]),
    "bmg_launch_count": (L, [P]),
    "bmg_free": (None, [P]),
    "bmg_strerror": (ctypes.c_char_p, [I]),
    "bmg_last_error": (ctypes.c_char_p, []),
    "bmg_dendy_interp": (I, [I, P, P, P]),
    "bmg_rap": (I, [I, P, P, P, P]),
    "bmg_relax": (I, [I, I, P, P, P, I, P]),
    "bmg_relax_line": (I, [I, I, P, P, P, P, I, P]),
    "bmg_relax_line_y": (I, [I, I, P, P, P, P, I, P]),
    "bmg_debug_build": (I, []),
    "bmg_debug_take": (I, [ctypes.POINTER(I), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "bmg_debug_site_name": (ctypes.c_char_p, [I]),
    "bmg_debug_shrink": (I, [ctypes.c_longlong]),
    "bmg_resid_restrict": (I, [I, I, P, P, P, P, P, P]),
    "bmg_interp_correct": (I, [I, P, P, P, P]),
    "bmg_residual": (I, [I, I, P, P, P, P, ctypes.POINTER(D), P]),
    "bmg_coarse_factor": (I, [I, P, P, P]),
    "bmg_coarse_solve": (I, [I, P, P, P, P]),
    "bmg_inner_cycle": (I, [P, P, P]),
    "bmg_measure_fp64_rate": (I, [ctypes.POINTER(D), P]),
    "bmg_wait_selftest": (I, []),
    "bmg_batch_rhs": (I, [P, I, ctypes.POINTER(Opts), ctypes.POINTER(P)]),
    "bmg_tuned_pair": (I, [P, I]),
    "bmg_time_cycles": (I, [P, P, P, I, ctypes.POINTER(D)]),
    "bmg_setup_batched": (I, [I, P, P, ctypes.POINTER(Opts), ctypes.POINTER(P)]),
    "bmg_solve_batched": (I, [P, P, P, D, I, P, P]),
    "bmg_batched_history": (I, [P, I, ctypes.POINTER(D), I]),
    "bmg_time_cycles_batched": (I, [P, P, P, I, ctypes.POINTER(D)]),
    "bmg_batched_launch_count": (L, [P]),
    "bmg_batched_tuned_cluster": (I, [P, I]),
    "bmg_free_batched": (None, [P]),
    "bmg_residual_noalloc": (I, [I, I, P, P, P, P, ctypes.POINTER(D), P]),
    "bmg_mlp_create": (I, [ctypes.POINTER(P)]),
    "bmg_mlp_set_params": (I, [P, P, I]),
    "bmg_mlp_get_params": (I, [P, P, I]),
    "bmg_mlp_get_adam": (I, [P, P, P, ctypes.POINTER(I), I]),
    "bmg_mlp_set_adam": (I, [P, P, P, I, I]),
    "bmg_mlp_loss_grad": (I, [P, I, P, I, P, P, ctypes.POINTER(D), P, P, P]),
    "bmg_mlp_twogrid": (I, [P, I, I, P, I, P, P, P, ctypes.POINTER(D), P, P]),
    "bmg_mlp_adam": (I, [P, ctypes.c_float, P]),
    "bmg_mlp_infer": (I, [P, I, P, P, P]),
    "bmg_learned_interp": (I, [I, P, P, P, P]),
    "bmg_mlp_features": (I, [I, P, P, P]),
    "bmg_interp_info": (I, [P, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(D)]),
    "bmg_tuned_cluster": (I, [P, I]),
    "bmg_fill_uniform": (I, [I, ctypes.c_ulonglong, P, P]),
    "bmg_mlp_free": (None, [P]),
    "bmg_profile": (I, [P, P, P, I, P, I]),
}
for _name, (_res, _args) in _sig.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def _check(rc: int, allow=()):
    if rc != BMG_OK and rc not in allow:
        raise BmgError(rc, f"{lib.bmg_strerror(rc).decode()}: {lib.bmg_last_error().decode()}")
    return rc


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor, dtype=torch.float64, name="tensor"):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


def _n_of(t: torch.Tensor) -> int:
    return t.shape[-1] - 2


def _need(t: torch.Tensor, count: int, name: str) -> torch.Tensor:
    """Refuse a tensor holding fewer values than the library reads or writes
    through its pointer: the C ABI takes bare pointers, so the sizes are
    checked here."""
    if t is not None and t.numel() < count:
        raise ValueError(f"{name} holds {t.numel()} values; {count} are needed")
    return t


def _planes(kind: int) -> int:
    """Stencil planes a kernel of this kind reads: O, W, S (5-point) or also SW, NW."""
    return 5 if kind == 9 else 3


def _grid(n: int) -> int:
    return (n + 2) * (n + 2)


class Hierarchy:
    """A BoxMG hierarchy built on the GPU (bmg_setup) and its solver (bmg_solve)."""

    def __init__(self, kind: int, coef: torch.Tensor, precision: str = "fp64", coarsest: int = 3,
                 nu1: int = 2, nu2: int = 1, inner_cycles: int = 1, bf16_levels: int = 2,
                 use_graph: bool = True, krylov: str = "none", mlp: "Mlp | None" = None, smoother: str = "auto",
                 arith: str = "rounded", fuse_restrict: str = "auto", periodic: str = ""):
        """periodic: "" (Dirichlet sides), "x", "y" or "xy" (those axes wrap
        around; a periodic axis has 2^m points, a Dirichlet one 2^m - 1)."""
        nx, ny = coef.shape[-1] - 2, coef.shape[-2] - 2     # any size; 2^m - 1 squares natively
        self.nx, self.ny, self.kind, self.precision, self.arith = nx, ny, kind, precision, arith
        if kind in (5, 9):
            _need(coef, _planes(kind) * (nx + 2) * (ny + 2), "coef")
        st = Stencil(kind, _ptr(coef, name="coef"))
        o = Opts(_PREC[precision], 1 if mlp is not None else 0, coarsest, nu1, nu2, inner_cycles, bf16_levels,
                 int(use_graph), _KRYLOV[krylov], mlp._h if mlp is not None else None, _stream(),
                 _SMOOTHER[smoother], _ARITH[arith], _FUSE[fuse_restrict])
        if set(periodic) - set("xy"):
            raise ValueError(f"periodic must be a combination of 'x' and 'y', not {periodic!r}")
        o.periodic = (BMG_PERIODIC_X if "x" in periodic else 0) | (BMG_PERIODIC_Y if "y" in periodic else 0)
        self.periodic = periodic
        h = ctypes.c_void_p()
        _check(lib.bmg_setup(ctypes.byref(st), nx, ny, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.n = self.level_shape(0)[0]   # level 0: nx = ny = n, the embedding square, or the periodic nx

    def solve(self, rhs: torch.Tensor, x: torch.Tensor | None = None, tol: float = 1e-10, maxit: int = 100):
        """Returns (x, iterations, relative residual, converged)."""
        if x is None:
            x = torch.zeros_like(rhs)
        self._need_grid(rhs, x)
        it, rr = ctypes.c_int(0), ctypes.c_double(0.0)
        rc = _check(lib.bmg_solve(self._h, _ptr(rhs, name="rhs"), _ptr(x, name="x"), tol, maxit,
                                  ctypes.byref(it), ctypes.byref(rr)), allow=(BMG_ENOTCONV,))
        return x, it.value, rr.value, rc == BMG_OK

    def time_cycles(self, rhs: torch.Tensor, x: torch.Tensor, cycles: int) -> float:
        """Device milliseconds of `cycles` solve iterations (no convergence test)."""
        self._need_grid(rhs, x)
        ms = ctypes.c_double(0.0)
        _check(lib.bmg_time_cycles(self._h, _ptr(rhs, name="rhs"), _ptr(x, name="x"), cycles, ctypes.byref(ms)))
        return ms.value

    def profile(self, rhs: torch.Tensor, x: torch.Tensor, cycles: int):
        """Per (level, kernel, fp32) device time of `cycles` iterations: a list of
        dicts with keys level, kernel, fp32, launches, ms."""
        self._need_grid(rhs, x)
        rows = (ProfRow * 256)()
        cnt = _check_size(lib.bmg_profile(self._h, _ptr(rhs, name="rhs"), _ptr(x, name="x"), cycles, rows, 256))
        return [dict(level=r.level, kernel=KERNEL_NAMES[r.kernel], fp32=bool(r.fp32), launches=r.launches, ms=r.ms)
                for r in rows[:cnt]]

    def _need_grid(self, rhs, x):
        """rhs and x in the caller's (ny+2) x (nx+2) layout."""
        _need(rhs, (self.nx + 2) * (self.ny + 2), "rhs")
        _need(x, (self.nx + 2) * (self.ny + 2), "x")

    def history(self):
        cnt = lib.bmg_history(self._h, None, 0)
        buf = (ctypes.c_double * max(cnt, 1))()
        lib.bmg_history(self._h, buf, cnt)
        return list(buf[:cnt])

    @property
    def num_levels(self) -> int:
        return lib.bmg_num_levels(self._h)

    def level_size(self, level: int) -> int:
        return _check_size(lib.bmg_level_size(self._h, level))

    def level_shape(self, level: int) -> tuple[int, int]:
        """(nx, ny) of a level: (n, n) for Dirichlet hierarchies."""
        nx, ny = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib.bmg_level_shape(self._h, level, ctypes.byref(nx), ctypes.byref(ny)))
        return nx.value, ny.value

    def stencil(self, level: int) -> torch.Tensor:
        nx, ny = self.level_shape(level)
        out = torch.empty((5, ny + 2, nx + 2), dtype=torch.float64, device="cuda")
        _check(lib.bmg_get_stencil(self._h, level, _ptr(out)))
        return out

    def interp(self, level: int) -> torch.Tensor:
        nx, ny = self.level_shape(level + 1)
        out = torch.empty((8, ny + 2, nx + 2), dtype=torch.float64, device="cuda")
        _check(lib.bmg_get_interp(self._h, level, _ptr(out)))
        return out

    def inner_cycle(self, r32: torch.Tensor) -> torch.Tensor:
        _need(r32, _grid(self.n), "r32")
        e = torch.empty_like(r32)
        _check(lib.bmg_inner_cycle(self._h, _ptr(r32, torch.float32, "r32"), _ptr(e, torch.float32, "e32")))
        return e

    def tuned_cluster(self, level: int) -> int:
        return _check_size(lib.bmg_tuned_cluster(self._h, level))

    def tuned_pair(self, level: int) -> int:
        """Two-sweep pass shape used on `level` (-1: sweeps one at a time)."""
        return lib.bmg_tuned_pair(self._h, level)

    def interp_info(self):
        """(kept interpolation: "learned" or "dendy", learned factor, Dendy factor)."""
        used, fl, fd = ctypes.c_int(0), ctypes.c_double(0), ctypes.c_double(0)
        _check(lib.bmg_interp_info(self._h, ctypes.byref(used), ctypes.byref(fl), ctypes.byref(fd)))
        return ("learned" if used.value == 1 else "dendy"), fl.value, fd.value

    @property
    def launch_count(self) -> int:
        return lib.bmg_launch_count(self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib.bmg_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent problems solved together (bmg_setup_batched): one
    launch per cycle stage over all problems, one CUDA graph per iteration."""

    def __init__(self, kind: int, coefs, precision: str = "fp64", nu1: int = 2, nu2: int = 1,
                 inner_cycles: int = 1, bf16_levels: int = 2, use_graph: bool = True, smoother: str = "auto",
                 arith: str = "rounded"):
        self.kind, self.precision = kind, precision
        self.ns = [_n_of(c) for c in coefs]
        self._coefs = list(coefs)
        nprob = len(coefs)
        if kind in (5, 9):
            for c, n in zip(coefs, self.ns):
                _need(c, _planes(kind) * _grid(n), "coef")
        sts = (Stencil * nprob)(*[Stencil(kind, _ptr(c, name="coef")) for c in coefs])
        ns = (ctypes.c_int * nprob)(*self.ns)
        o = Opts(_PREC[precision], 0, 0, nu1, nu2, inner_cycles, bf16_levels, int(use_graph), 0, None, _stream(),
                 _SMOOTHER[smoother], _ARITH[arith])
        h = ctypes.c_void_p()
        _check(lib.bmg_setup_batched(nprob, sts, ns, ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_hierarchy(cls, h: "Hierarchy", k: int, nu1: int = 2, nu2: int = 1, inner_cycles: int = 1,
                       use_graph: bool = True, smoother: str = "auto", rhs_block="auto") -> "Batch":
        """k right-hand sides of h's operator solved together (bmg_batch_rhs);
        h must stay open while the batch is used.  rhs_block: "auto", "off",
        2 or 4 members per warp in the one-pass sweeps (each stencil value read
        once for them)."""
        self = cls.__new__(cls)
        self.kind, self.precision = h.kind, h.precision
        self.ns = [h.n] * k
        self._coefs = [h]   # keeps the hierarchy alive
        o = Opts(_PREC[h.precision], 0, 0, nu1, nu2, inner_cycles, 0, int(use_graph), 0, None, _stream(),
                 _SMOOTHER[smoother], _ARITH[h.arith], 0, _RHS_BLOCK[rhs_block])
        b = ctypes.c_void_p()
        _check(lib.bmg_batch_rhs(h._h, k, ctypes.byref(o), ctypes.byref(b)))
        self._h = b
        return self

    def _ptrs(self, ts, name):
        """One pointer per problem; each tensor must hold its problem's grid."""
        if len(ts) != len(self.ns):
            raise ValueError(f"{len(ts)} {name} tensors for {len(self.ns)} problems")
        for t, n in zip(ts, self.ns):
            _need(t, _grid(n), name)
        return (ctypes.c_void_p * len(ts))(*[_ptr(t, name=name).value for t in ts])

    def solve(self, rhs, xs=None, tol: float = 1e-10, maxit: int = 100):
        """Returns (xs, iterations per problem, relative residual per problem, all converged)."""
        if xs is None:
            xs = [torch.zeros_like(r) for r in rhs]
        prhs, pxs = self._ptrs(rhs, "rhs"), self._ptrs(xs, "x")
        nprob = len(rhs)
        it = (ctypes.c_int * nprob)()
        rr = (ctypes.c_double * nprob)()
        rc = _check(lib.bmg_solve_batched(self._h, prhs, pxs, tol, maxit, it, rr), allow=(BMG_ENOTCONV,))
        return xs, list(it), list(rr), rc == BMG_OK

    def history(self, p: int):
        cnt = lib.bmg_batched_history(self._h, p, None, 0)
        buf = (ctypes.c_double * max(cnt, 1))()
        lib.bmg_batched_history(self._h, p, buf, cnt)
        return list(buf[:cnt])

    def time_cycles(self, rhs, xs, cycles: int) -> float:
        ms = ctypes.c_double(0.0)
        _check(lib.bmg_time_cycles_batched(self._h, self._ptrs(rhs, "rhs"), self._ptrs(xs, "x"), cycles,
                                           ctypes.byref(ms)))
        return ms.value

    def tuned_cluster(self, stage: int) -> int:
        return _check_size(lib.bmg_batched_tuned_cluster(self._h, stage))

    @property
    def launch_count(self) -> int:
        return lib.bmg_batched_launch_count(self._h)

    def close(self):
        if getattr(self, "_h", None):
            lib.bmg_free_batched(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_PARAMS = 18 * 64 + 64 + 64 * 64 + 64 + 64 * 4 + 4


class Mlp:
    """The learned-interpolation network on the device (bmg_mlp_*)."""

    def __init__(self, params=None):
        h = ctypes.c_void_p()
        _check(lib.bmg_mlp_create(ctypes.byref(h)))
        self._h = h
        if params is not None:
            self.set_params(params)

    def set_params(self, params):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert a.size == MLP_PARAMS
        _check(lib.bmg_mlp_set_params(self._h, a.ctypes.data_as(ctypes.c_void_p), MLP_PARAMS))

    def params(self):
        import numpy as np
        a = np.empty(MLP_PARAMS, dtype=np.float32)
        _check(lib.bmg_mlp_get_params(self._h, a.ctypes.data_as(ctypes.c_void_p), MLP_PARAMS))
        return a

    def adam_state(self):
        """(first moments, second moments, step) of the optimizer (numpy float32)."""
        import numpy as np
        m1, m2, st = np.empty(MLP_PARAMS, np.float32), np.empty(MLP_PARAMS, np.float32), ctypes.c_int(0)
        _check(lib.bmg_mlp_get_adam(self._h, m1.ctypes.data_as(ctypes.c_void_p), m2.ctypes.data_as(ctypes.c_void_p),
                                    ctypes.byref(st), MLP_PARAMS))
        return m1, m2, st.value

    def set_adam_state(self, m1, m2, step: int):
        import numpy as np
        a = np.ascontiguousarray(m1, dtype=np.float32)
        b = np.ascontiguousarray(m2, dtype=np.float32)
        assert a.size == MLP_PARAMS and b.size == MLP_PARAMS
        _check(lib.bmg_mlp_set_adam(self._h, a.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p),
                                    int(step), MLP_PARAMS))

    def loss_grad(self, coef, vecs, eref=None, want_grad=True):
        """(loss, gradient (numpy float32) or None, eref) on one problem; vecs: (K, n+2, n+2) CUDA float64."""
        import numpy as np
        n = _n_of(coef)
        K = vecs.shape[0]
        loss = ctypes.c_double(0.0)
        g = np.empty(MLP_PARAMS, dtype=np.float32) if want_grad else None
        er_in = None if eref is None else np.ascontiguousarray(eref, dtype=np.float64)
        er_out = np.empty(K, dtype=np.float64)
        _check(lib.bmg_mlp_loss_grad(self._h, n, _ptr(coef, name="coef"), K, _ptr(vecs, name="vecs"),
                                     None if er_in is None else er_in.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.byref(loss), None if g is None else g.ctypes.data_as(ctypes.c_void_p),
                                     er_out.ctypes.data_as(ctypes.c_void_p), _stream()))
        return loss.value, g, (er_in if er_in is not None else er_out)

    def twogrid(self, coefs, vecs, eref=None, want_grad=True):
        """The two-grid loss over a batch of crops: coefs (C, 5, n+2, n+2) and
        vecs (C, K, n+2, n+2) CUDA float64, n = 7, 15 or 31; eref (C, K) CUDA
        float64 or None.  With eref: (loss, gradient (numpy float32) or None,
        energies (C, K) tensor); without: (None, None, Dendy's energies)."""
        import numpy as np
        if coefs.dim() != 4 or vecs.dim() != 4 or coefs.shape[0] != vecs.shape[0] or coefs.shape[1] != 5:
            raise ValueError("coefs must be (C, 5, n+2, n+2) and vecs (C, K, n+2, n+2)")
        C, K, m = vecs.shape[0], vecs.shape[1], vecs.shape[-1]
        if coefs.shape[-1] != m or coefs.shape[-2] != m or vecs.shape[-2] != m:
            raise ValueError("coefs and vecs must share the crop grid")
        energies = torch.empty((C, K), dtype=torch.float64, device=vecs.device)
        if eref is not None and tuple(eref.shape) != (C, K):
            raise ValueError("eref must be (C, K)")
        loss = ctypes.c_double(0.0)
        g = np.empty(MLP_PARAMS, dtype=np.float32) if (want_grad and eref is not None) else None
        _check(lib.bmg_mlp_twogrid(self._h, C, m - 2, _ptr(coefs, name="coefs"), K, _ptr(vecs, name="vecs"),
                                   None if eref is None else _ptr(eref, name="eref"), _ptr(energies, name="energies"),
                                   ctypes.byref(loss), None if g is None else g.ctypes.data_as(ctypes.c_void_p),
                                   _stream()))
        return (loss.value if eref is not None else None), g, energies

    def adam(self, lr: float):
        _check(lib.bmg_mlp_adam(self._h, ctypes.c_float(lr), _stream()))

    def infer(self, coef):
        n = _n_of(coef)
        nc = (n - 1) // 2
        _need(coef, 5 * _grid(n), "coef")
        out = torch.empty((nc * nc, 4), dtype=torch.float32, device=coef.device)
        _check(lib.bmg_mlp_infer(self._h, n, _ptr(coef, name="coef"), _ptr(out, torch.float32, "delta"), _stream()))
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib.bmg_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_features(coef):
    """(n_c^2, 18) FP32 features of every interior coarse point (bmg_mlp_features)."""
    n = _n_of(coef)
    nc = (n - 1) // 2
    _need(coef, 5 * _grid(n), "coef")
    X = torch.empty((nc * nc, 18), dtype=torch.float32, device=coef.device)
    _check(lib.bmg_mlp_features(n, _ptr(coef, name="coef"), _ptr(X, torch.float32, "X"), _stream()))
    return X


def learned_interp(coef, delta):
    n = _n_of(coef)
    nc = (n - 1) // 2
    _need(coef, 5 * _grid(n), "coef")
    _need(delta, nc * nc * 4, "delta")
    ci = torch.empty((8, nc + 2, nc + 2), dtype=torch.float64, device=coef.device)
    _check(lib.bmg_learned_interp(n, _ptr(coef), _ptr(delta, torch.float32, "delta"), _ptr(ci), _stream()))
    return ci


def fill_uniform(n: int, seed: int, device="cuda"):
    x = torch.zeros((n + 2, n + 2), dtype=torch.float64, device=device)
    _check(lib.bmg_fill_uniform(n, seed, _ptr(x), _stream()))
    return x


def _need_level(kind: int, coef, f, x):
    """One level's stencil (the planes its kind reads), right-hand side and iterate."""
    n = _n_of(coef)
    _need(coef, _planes(kind) * _grid(n), "coef")
    _need(f, _grid(n), "f")
    _need(x, _grid(n), "x")


def _check_size(v: int) -> int:
    if v < 0:
        _check(v)
    return v


def dendy_interp(coef: torch.Tensor) -> torch.Tensor:
    n = _n_of(coef)
    nc = (n - 1) // 2
    _need(coef, 5 * _grid(n), "coef")
    ci = torch.empty((8, nc + 2, nc + 2), dtype=torch.float64, device=coef.device)
    _check(lib.bmg_dendy_interp(n, _ptr(coef), _ptr(ci), _stream()))
    return ci


def rap(coef: torch.Tensor, ci: torch.Tensor) -> torch.Tensor:
    n = _n_of(coef)
    nc = (n - 1) // 2
    _need(coef, 5 * _grid(n), "coef")
    _need(ci, 8 * _grid(nc), "ci")
    out = torch.empty((5, nc + 2, nc + 2), dtype=torch.float64, device=coef.device)
    _check(lib.bmg_rap(n, _ptr(coef), _ptr(ci), _ptr(out), _stream()))
    return out


def relax(kind: int, coef: torch.Tensor, f: torch.Tensor, x: torch.Tensor, sweeps: int = 1) -> torch.Tensor:
    _need_level(kind, coef, f, x)
    _check(lib.bmg_relax(_n_of(coef), kind, _ptr(coef), _ptr(f), _ptr(x), sweeps, _stream()))
    return x


def relax_line(kind: int, coef: torch.Tensor, f: torch.Tensor, x: torch.Tensor, sweeps: int = 1,
               axis: str = "x") -> torch.Tensor:
    """Zebra line Gauss-Seidel sweeps in place on x: x-lines (bmg_relax_line)
    or y-lines (axis="y", bmg_relax_line_y)."""
    _need_level(kind, coef, f, x)
    work = torch.empty_like(x)
    fn = {"x": lib.bmg_relax_line, "y": lib.bmg_relax_line_y}[axis]
    _check(fn(_n_of(coef), kind, _ptr(coef), _ptr(f), _ptr(x), _ptr(work), sweeps, _stream()))
    return x


def resid_restrict(kind: int, coef, ci, x, f) -> torch.Tensor:
    n = _n_of(coef)
    nc = (n - 1) // 2
    _need_level(kind, coef, f, x)
    _need(ci, 8 * _grid(nc), "ci")
    fc = torch.empty((nc + 2, nc + 2), dtype=torch.float64, device=coef.device)
    _check(lib.bmg_resid_restrict(n, kind, _ptr(coef), _ptr(ci), _ptr(x), _ptr(f), _ptr(fc), _stream()))
    return fc


def interp_correct(ci, ec, x) -> torch.Tensor:
    nc = (_n_of(x) - 1) // 2
    _need(x, _grid(_n_of(x)), "x")
    _need(ci, 8 * _grid(nc), "ci")
    _need(ec, _grid(nc), "ec")
    _check(lib.bmg_interp_correct(_n_of(x), _ptr(ci), _ptr(ec), _ptr(x), _stream()))
    return x


def residual(kind: int, coef, x, f, want_r: bool = True):
    """Returns (r or None, ||r||)."""
    n = _n_of(coef)
    _need_level(kind, coef, f, x)
    r = torch.empty_like(f) if want_r else None
    nrm = ctypes.c_double(0.0)
    _check(lib.bmg_residual(n, kind, _ptr(coef), _ptr(x), _ptr(f), _ptr(r) if want_r else None,
                            ctypes.byref(nrm), _stream()))
    return r, nrm.value


def coarse_factor(coef: torch.Tensor) -> torch.Tensor:
    n = _n_of(coef)
    _need(coef, 5 * _grid(n), "coef")
    L = torch.empty((n * n, n * n), dtype=torch.float64, device=coef.device)
    _check(lib.bmg_coarse_factor(n, _ptr(coef), _ptr(L), _stream()))
    return L


def coarse_solve(L: torch.Tensor, f: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    n = _n_of(f)
    _need(f, _grid(n), "f")
    _need(x, _grid(n), "x")
    _need(L, n * n * n * n, "L")
    _check(lib.bmg_coarse_solve(_n_of(f), _ptr(L), _ptr(f), _ptr(x), _stream()))
    return x


def measure_fp64_rate() -> float:
    v = ctypes.c_double(0.0)
    _check(lib.bmg_measure_fp64_rate(ctypes.byref(v), _stream()))
    return v.value


def debug_build() -> bool:
    """True when the loaded library is libbmg_debug.so (bmg_debug_build)."""
    return bool(lib.bmg_debug_build())


def debug_take():
    """The first device bounds-check failure recorded since the last call, as
    (site name, index, extent), or None; clears the records (bmg_debug_take)."""
    site, index, extent = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
    rc = _check_size(lib.bmg_debug_take(ctypes.byref(site), ctypes.byref(index), ctypes.byref(extent)))
    if rc == 0:
        return None
    return lib.bmg_debug_site_name(site.value).decode(), index.value, extent.value


def debug_shrink(k: int) -> None:
    """Test hook of debug builds: checks use extent - k (bmg_debug_shrink)."""
    _check(lib.bmg_debug_shrink(k))
