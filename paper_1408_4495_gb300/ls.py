"""Thin ctypes binding of libls (``include/ls.h``): argument marshalling only.

Every step of the solve runs inside the CUDA library; this module only turns numpy arrays
(host) or torch CUDA tensors (device) into pointers and sizes.  If the library has not
been built, or cannot be loaded, every call raises: there is no CPU path.

Complex arrays cross the boundary as interleaved (re, im) float64, C order, right-hand
sides outermost, i.e. numpy ``complex128`` of shape ``(nrhs,) + (n,) * d`` or a torch
``complex128`` CUDA tensor of that shape.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libls.so")

LS_OK, LS_EINVAL, LS_ENOMEM, LS_ECUDA, LS_ENOCONV, LS_ESTATE, LS_ETIMEOUT, LS_EBUFFER = range(8)
LS_PREC_FP64, LS_PREC_MIXED, LS_PREC_FF = 0, 1, 2
LS_K0_BALL, LS_K0_CORRECTED = 0, 1
LS_FRONT_3XTF32, LS_FRONT_FP32, LS_FRONT_TF32, LS_FRONT_BF16 = 0, 1, 2, 3
STATUS_NAMES = ["LS_OK", "LS_EINVAL", "LS_ENOMEM", "LS_ECUDA", "LS_ENOCONV", "LS_ESTATE", "LS_ETIMEOUT", "LS_EBUFFER"]

# every entry point declared in include/ls.h
EXPORTS = ["ls_setup", "ls_setup_laplace", "ls_factor", "ls_rhs_plane_wave", "ls_rhs_point_source", "ls_solve",
           "ls_far_field", "ls_k0_weight", "ls_general_support", "ls_general_boundary_stencils",
           "ls_general_sketch", "ls_general_setup", "ls_general_rows", "ls_set_medium", "ls_fault_alloc",
           "ls_export_factors", "ls_import_factors",
           "ls_last_error", "ls_free",
           "ls_kernel_table", "ls_stencils", "ls_apply", "ls_stencil_apply", "ls_precond", "ls_get_nd_stats",
           "ls_profile_start", "ls_profile_stop", "ls_autotune", "ls_tune_info", "ls_set_tune", "ls_apply_noalloc", "ls_set_precond_refine"]


class LsGrid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("buffer_b", ctypes.c_int),
                ("restart", ctypes.c_int), ("max_iter", ctypes.c_int), ("prec", ctypes.c_int),
                ("k0_rule", ctypes.c_int), ("front_fmt", ctypes.c_int)]


class LsInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("refinements", ctypes.c_int), ("rel_resid", ctypes.c_double),
                ("converged", ctypes.c_int)]


class LsNdStats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("fronts", ctypes.c_int), ("max_front", ctypes.c_int),
                ("factor_entries", ctypes.c_int64), ("factor_flops", ctypes.c_double),
                ("solve_bytes", ctypes.c_double), ("fwd_factor_bytes", ctypes.c_double),
                ("fwd_bytes_per_rhs", ctypes.c_double), ("bwd_factor_bytes", ctypes.c_double),
                ("bwd_bytes_per_rhs", ctypes.c_double)]


class LsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libls (raises if it is missing: build it with paper_1408_4495_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libls not built ({path} missing); run python -m paper_1408_4495_gb300.build")
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.ls_setup.argtypes = [ctypes.POINTER(LsGrid), dp, vp, vp, ctypes.POINTER(vp)]
    lib.ls_factor.argtypes = [vp]
    lib.ls_set_medium.argtypes = [vp, vp]
    lib.ls_export_factors.argtypes = [vp, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    lib.ls_import_factors.argtypes = [vp, vp, ctypes.c_size_t]
    lib.ls_fault_alloc.argtypes = [ctypes.c_long]
    lib.ls_rhs_plane_wave.argtypes = [vp, ip, vp, vp]
    lib.ls_setup_laplace.argtypes = [ctypes.POINTER(LsGrid), vp, vp, ctypes.POINTER(vp)]
    lib.ls_rhs_point_source.argtypes = [vp, ip, vp, vp, vp]
    lib.ls_far_field.argtypes = [vp, ip, vp, vp, ip, vp, vp]
    lib.ls_k0_weight.argtypes = [ip, dp, dp, ip, vp]
    lib.ls_general_support.argtypes = [ip, ip, vp, ip, vp]
    lib.ls_general_boundary_stencils.argtypes = [ip, ip, vp, vp, ip, vp, vp]
    lib.ls_general_sketch.argtypes = [vp, vp, ip, vp, vp]
    lib.ls_general_setup.argtypes = [vp, vp, vp, vp]
    lib.ls_general_rows.argtypes = [ip, ip, vp, vp, vp, vp, vp, vp]
    lib.ls_solve.argtypes = [vp, ip, vp, dp, vp, ctypes.POINTER(LsInfo)]
    lib.ls_last_error.argtypes = [vp]
    lib.ls_last_error.restype = ctypes.c_char_p
    lib.ls_free.argtypes = [vp]
    lib.ls_free.restype = None
    lib.ls_kernel_table.argtypes = [vp, vp]
    lib.ls_stencils.argtypes = [vp, vp, vp]
    lib.ls_apply.argtypes = [vp, ip, vp, vp, ip]
    lib.ls_stencil_apply.argtypes = [vp, ip, vp, vp, ip]
    lib.ls_precond.argtypes = [vp, ip, vp, vp]
    lib.ls_get_nd_stats.argtypes = [vp, ctypes.POINTER(LsNdStats)]
    lib.ls_apply_noalloc.argtypes = [vp, ip, vp, vp]
    lib.ls_autotune.argtypes = [vp, ip, ctypes.c_char_p, ip]
    lib.ls_tune_info.argtypes = [vp, ctypes.c_char_p, ip]
    lib.ls_set_tune.argtypes = [vp, ctypes.c_char_p]
    lib.ls_set_precond_refine.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.ls_profile_start.argtypes = [ctypes.c_char_p]
    lib.ls_profile_stop.argtypes = [ctypes.c_char_p, ip]
    for name in EXPORTS:
        if name not in ("ls_last_error", "ls_free"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a):
    """Pointer of a numpy array (host) or a torch tensor (device or host)."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def profile_start(timed_class: str | None = None) -> None:
    """Reset the library's per-kernel-class launch counters; time one class with CUDA events."""
    load().ls_profile_start(timed_class.encode() if timed_class else None)


def profile_stop() -> dict:
    """Counters and timed-class device time since profile_start (see include/ls.h)."""
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    load().ls_profile_stop(buf, len(buf))
    return json.loads(buf.value.decode())


def k0_weight(dim: int, omega: float, h: float, rule: int = LS_K0_BALL) -> complex:
    """ls_k0_weight: the weight of the singular point (host computation, no device)."""
    lib = load()
    out = (ctypes.c_double * 2)()
    st = lib.ls_k0_weight(int(dim), float(omega), float(h), int(rule), out)
    if st != LS_OK:
        raise LsError(st, "ls_k0_weight: bad arguments")
    return complex(out[0], out[1])


def general_support(m: np.ndarray, b: int = 2) -> np.ndarray:
    """ls_general_support: boolean mask of the general-domain unknowns (Sec. 4)."""
    m = np.ascontiguousarray(m, dtype=np.float64)
    mask = np.empty(m.shape, dtype=np.uint8)
    st = load().ls_general_support(m.ndim, m.shape[0], _ptr(m), int(b), _ptr(mask))
    if st != LS_OK:
        raise LsError(st, "ls_general_support: bad arguments")
    return mask.astype(bool)


def general_boundary_stencils(mask: np.ndarray, T: np.ndarray):
    """ls_general_boundary_stencils: (alpha (unknowns x 3^d), boundary flags) from the sketch T
    (unknowns x r, rows in increasing flat index of the unknowns)."""
    mk = np.ascontiguousarray(mask, dtype=np.uint8)
    T = np.ascontiguousarray(T, dtype=np.complex128)
    no, r = T.shape
    d = mk.ndim
    alpha = np.empty((no, 3**d), dtype=np.complex128)
    bnd = np.empty(no, dtype=np.int32)
    st = load().ls_general_boundary_stencils(d, mk.shape[0], _ptr(mk), _ptr(T), int(r), _ptr(alpha), _ptr(bnd))
    if st != LS_OK:
        raise LsError(st, "ls_general_boundary_stencils: bad arguments or an undetermined stencil")
    return alpha, bnd.astype(bool)


def fault_alloc(k: int):
    """ls_fault_alloc: the k-th device allocation from now fails with LS_ENOMEM (0 disarms)."""
    st = load().ls_fault_alloc(int(k))
    if st != LS_OK:
        raise LsError(st, "ls_fault_alloc: k must be >= 0")


def general_rows(mask: np.ndarray, alpha: np.ndarray, boundary: np.ndarray, alpha_interior: np.ndarray):
    """ls_general_rows: (rows (n^d x 3^d), interior flags (n^d,)) of the box embedding of the
    general-domain preconditioner (Sec. 4), on the host."""
    mk = np.ascontiguousarray(mask, dtype=np.uint8)
    d = mk.ndim
    al = np.ascontiguousarray(alpha, dtype=np.complex128)
    bd = np.ascontiguousarray(boundary, dtype=np.int32)
    ai = np.ascontiguousarray(alpha_interior, dtype=np.complex128)
    nu = int(np.count_nonzero(mk))
    if al.shape != (nu, 3**d) or bd.shape != (nu,) or ai.shape != (3**d,):
        raise ValueError("alpha (unknowns x 3^d), boundary (unknowns,), alpha_interior (3^d,)")
    rows = np.empty((mk.size, 3**d), dtype=np.complex128)
    inter = np.empty(mk.size, dtype=np.uint8)
    st = load().ls_general_rows(d, mk.shape[0], _ptr(mk), _ptr(al), _ptr(bd), _ptr(ai), _ptr(rows), _ptr(inter))
    if st != LS_OK:
        raise LsError(st, "ls_general_rows: bad arguments or inconsistent stencils")
    return rows, inter.astype(bool)


@dataclass
class SolveInfo:
    iters: int
    refinements: int
    rel_resid: float
    converged: bool


class Solver:
    """One medium on one grid: ``ls_setup`` at construction, ``ls_free`` on close.

    ``laplace=True`` selects the Laplace variant (``ls_setup_laplace``, Sec. 5): ``m`` is then
    the potential V and ``omega`` is ignored.  ``k0_rule`` picks the weight of the singular
    point (``LS_K0_BALL`` or ``LS_K0_CORRECTED``, Sec. 2.1); ``front_fmt`` the arithmetic of the
    fronts' Schur products on the mixed path (``LS_FRONT_3XTF32`` or ``LS_FRONT_FP32``)."""

    def __init__(self, m, omega: float = 0.0, dim: int | None = None, buffer_b: int = 2, restart: int = 50,
                 max_iter: int = 500, mixed: bool = True, stream=None, laplace: bool = False,
                 k0_rule: int = LS_K0_BALL, front_fmt: int = LS_FRONT_3XTF32):
        self.lib = load()
        if isinstance(m, np.ndarray):
            m = np.ascontiguousarray(m, dtype=np.float64)
        self.d = dim if dim is not None else m.ndim
        self.n = int(m.shape[0])
        self.N = self.n ** self.d
        self.omega = 0.0 if laplace else float(omega)
        self.laplace = laplace
        self.mixed = mixed
        self.k0_rule = k0_rule
        g = LsGrid(self.d, self.n, buffer_b, restart, max_iter, LS_PREC_MIXED if mixed else LS_PREC_FP64,
                   k0_rule, front_fmt)
        h = ctypes.c_void_p()
        if laplace:
            st = self.lib.ls_setup_laplace(ctypes.byref(g), _ptr(m), _stream_ptr(stream), ctypes.byref(h))
        else:
            st = self.lib.ls_setup(ctypes.byref(g), self.omega, _ptr(m), _stream_ptr(stream), ctypes.byref(h))
        if st != LS_OK:
            raise LsError(st, self.lib.ls_last_error(None).decode())
        self.h = h

    def _check(self, st, allow=()):
        if st != LS_OK and st not in allow:
            raise LsError(st, self.lib.ls_last_error(self.h).decode())
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.ls_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- the path
    def factor(self):
        self._check(self.lib.ls_factor(self.h))

    def export_factors(self) -> np.ndarray:
        """ls_export_factors: the factorization as a host byte array (header + fronts)."""
        size = ctypes.c_size_t(0)
        self._check(self.lib.ls_export_factors(self.h, None, 0, ctypes.byref(size)))
        blob = np.empty(size.value, dtype=np.uint8)
        self._check(self.lib.ls_export_factors(self.h, _ptr(blob), blob.size, ctypes.byref(size)))
        return blob

    def import_factors(self, blob: np.ndarray):
        """ls_import_factors: a factorization exported by a context of the same grid and medium."""
        blob = np.ascontiguousarray(blob, dtype=np.uint8)
        self._check(self.lib.ls_import_factors(self.h, _ptr(blob), blob.size))

    def set_medium(self, m):
        """ls_set_medium: a new medium on this grid (drops the factorization)."""
        if isinstance(m, np.ndarray):
            m = np.ascontiguousarray(m, dtype=np.float64)
        self._check(self.lib.ls_set_medium(self.h, _ptr(m)))

    def rhs_plane_wave(self, dirs, out=None):
        dirs_np = dirs if not isinstance(dirs, np.ndarray) else np.ascontiguousarray(dirs, dtype=np.float64)
        nrhs = int(dirs_np.shape[0])
        if out is None:
            shape = (nrhs,) + (self.n,) * self.d
            if isinstance(dirs_np, np.ndarray):
                out = np.empty(shape, dtype=np.complex128)
            else:  # a torch tensor: output on the same device
                import torch
                out = torch.empty(shape, dtype=torch.complex128, device=dirs_np.device)
        self._check(self.lib.ls_rhs_plane_wave(self.h, nrhs, _ptr(dirs_np), _ptr(out)))
        return out

    def rhs_point_source(self, points, strengths=None, out=None):
        """g = K f for delta sources at the (nrhs, d) 0-based grid indices ``points``."""
        pts = points if not isinstance(points, np.ndarray) else np.ascontiguousarray(points, dtype=np.int32)
        nrhs = int(pts.shape[0])
        q = strengths
        if isinstance(q, np.ndarray):
            q = np.ascontiguousarray(q, dtype=np.complex128)
        if out is None:
            shape = (nrhs,) + (self.n,) * self.d
            if isinstance(pts, np.ndarray):
                out = np.empty(shape, dtype=np.complex128)
            else:
                import torch
                out = torch.empty(shape, dtype=torch.complex128, device=pts.device)
        self._check(self.lib.ls_rhs_point_source(self.h, nrhs, _ptr(pts), _ptr(q) if q is not None else None,
                                                 _ptr(out)))
        return out

    def far_field(self, dirs, us, obs, out=None):
        """Far-field pattern u_inf(obs_k) of the scattered fields ``us`` of the plane waves
        ``dirs``: an (nrhs, nobs) complex array (see ls_far_field in include/ls.h)."""
        d = dirs if not isinstance(dirs, np.ndarray) else np.ascontiguousarray(dirs, dtype=np.float64)
        o = obs if not isinstance(obs, np.ndarray) else np.ascontiguousarray(obs, dtype=np.float64)
        if isinstance(us, np.ndarray):
            us = np.ascontiguousarray(us, dtype=np.complex128)
        nrhs, nobs = int(d.shape[0]), int(o.shape[0])
        if out is None:
            if isinstance(us, np.ndarray):
                out = np.empty((nrhs, nobs), dtype=np.complex128)
            else:
                import torch
                out = torch.empty((nrhs, nobs), dtype=torch.complex128, device=us.device)
        self._check(self.lib.ls_far_field(self.h, nrhs, _ptr(d), _ptr(us), nobs, _ptr(o), _ptr(out)))
        return out

    def solve(self, rhs, tol: float = 1e-6, out=None, raise_on_noconv: bool = True):
        nrhs = int(rhs.shape[0])
        if out is None:
            out = np.empty_like(rhs) if isinstance(rhs, np.ndarray) else rhs.new_empty(rhs.shape)
        infos = (LsInfo * nrhs)()
        st = self.lib.ls_solve(self.h, nrhs, _ptr(rhs), float(tol), _ptr(out), infos)
        self._check(st, allow=() if raise_on_noconv else (LS_ENOCONV,))
        return out, [SolveInfo(i.iters, i.refinements, i.rel_resid, bool(i.converged)) for i in infos]

    # ---- inspection entry points
    def general_sketch(self, mask: np.ndarray, R: np.ndarray) -> np.ndarray:
        """ls_general_sketch: T = (K omega^2 m) R on the unknowns of ``mask`` (Sec. 4.1); R is
        (unknowns x r), rows in increasing flat index of the unknowns."""
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        R = np.ascontiguousarray(R, dtype=np.complex128)
        if R.ndim != 2 or R.shape[0] != int(np.count_nonzero(mk)):
            raise ValueError("R must be (number of unknowns) x r")
        T = np.empty_like(R)
        self._check(self.lib.ls_general_sketch(self.h, _ptr(mk), int(R.shape[1]), _ptr(R), _ptr(T)))
        return T

    def general_setup(self, mask: np.ndarray, alpha: np.ndarray, boundary: np.ndarray):
        """ls_general_setup: the general-domain preconditioner of Sec. 4 from the unknowns
        ``mask`` and the boundary stencils (outputs of general_boundary_stencils)."""
        mk = np.ascontiguousarray(mask, dtype=np.uint8)
        al = np.ascontiguousarray(alpha, dtype=np.complex128)
        bd = np.ascontiguousarray(boundary, dtype=np.int32)
        nu = int(np.count_nonzero(mk))
        if al.shape != (nu, 3 ** self.d) or bd.shape != (nu,):
            raise ValueError("alpha must be (unknowns) x 3^d and boundary (unknowns,)")
        self._check(self.lib.ls_general_setup(self.h, _ptr(mk), _ptr(al), _ptr(bd)))

    def general_domain(self, m: np.ndarray, R: np.ndarray, buffer_b: int = 2):
        """The Sec. 4 pipeline through the C-ABI: unknowns (ls_general_support), device sketch
        (ls_general_sketch), boundary stencils (ls_general_boundary_stencils) and the
        preconditioner switch (ls_general_setup).  Returns the mask of the unknowns."""
        mask = general_support(m, buffer_b)
        T = self.general_sketch(mask, R)
        alpha, bnd = general_boundary_stencils(mask, T)
        self.general_setup(mask, alpha, bnd)
        return mask

    def kernel_table(self):
        out = np.empty((self.n + 1,) * self.d, dtype=np.complex128)
        self._check(self.lib.ls_kernel_table(self.h, _ptr(out)))
        return out

    def stencils(self):
        p3 = 3 ** self.d
        a = np.empty((p3, p3), dtype=np.complex128)
        c = np.empty(p3, dtype=np.complex128)
        self._check(self.lib.ls_stencils(self.h, _ptr(a), _ptr(c)))
        return a, c

    def _unary(self, fn, x, *extra):
        nrhs = int(x.shape[0])
        out = np.empty_like(x) if isinstance(x, np.ndarray) else x.new_empty(x.shape)
        self._check(fn(self.h, nrhs, _ptr(x), _ptr(out), *extra))
        return out

    def apply(self, x, mixed: bool | None = None, prec: int | None = None):
        """(I + K omega^2 m) x; prec overrides mixed (LS_PREC_FF: float-float operator)."""
        if prec is None:
            mixed = self.mixed if mixed is None else mixed
            prec = LS_PREC_MIXED if mixed else LS_PREC_FP64
        return self._unary(self.lib.ls_apply, x, prec)

    def stencil_apply(self, x, mixed: bool | None = None):
        mixed = self.mixed if mixed is None else mixed
        return self._unary(self.lib.ls_stencil_apply, x, LS_PREC_MIXED if mixed else LS_PREC_FP64)

    def precond(self, x):
        return self._unary(self.lib.ls_precond, x)

    def apply_noalloc(self, x, out):
        """FP64 operator apply into a caller-provided device tensor, without any device
        allocation inside the library (see ls_apply_noalloc in include/ls.h).  x and out must
        be complex128 tensors of shape (nrhs,) + (n,) * d on one CUDA device; anything else is
        refused here, before the library would read or write past the end of a buffer."""
        for name, t in (("x", x), ("out", out)):
            if not hasattr(t, "data_ptr") or not getattr(t, "is_cuda", False):
                raise ValueError(f"{name} must be a CUDA tensor")
            if str(t.dtype) != "torch.complex128":
                raise ValueError(f"{name} must be complex128, got {t.dtype}")
            if t.dim() != self.d + 1 or tuple(t.shape[1:]) != (self.n,) * self.d:
                raise ValueError(f"{name} must have shape (nrhs,) + {(self.n,) * self.d}, got {tuple(t.shape)}")
        if tuple(x.shape) != tuple(out.shape):
            raise ValueError(f"x {tuple(x.shape)} and out {tuple(out.shape)} differ in shape")
        if x.device != out.device:
            raise ValueError(f"x ({x.device}) and out ({out.device}) are on different devices")
        self._check(self.lib.ls_apply_noalloc(self.h, int(x.shape[0]), _ptr(x), _ptr(out)))
        return out

    def autotune(self, nrhs: int) -> dict:
        """ls_autotune: time the launch-shape alternatives on this context (factorization and
        solves of nrhs right-hand sides), apply and keep the fastest; returns the report."""
        import json
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(self.lib.ls_autotune(self.h, int(nrhs), buf, len(buf)))
        return json.loads(buf.value.decode())

    def tune(self) -> dict:
        """ls_tune_info: the context's launch-shape choices."""
        import json
        buf = ctypes.create_string_buffer(1024)
        self._check(self.lib.ls_tune_info(self.h, buf, len(buf)))
        return json.loads(buf.value.decode())

    def set_tune(self, choices: dict) -> None:
        """ls_set_tune: apply launch-shape choices (any keys of tune()) to this context."""
        import json
        self._check(self.lib.ls_set_tune(self.h, json.dumps(choices).encode()))

    def precond_refine(self, mode: int = -2) -> float:
        """ls_set_precond_refine: the FP32 preconditioner's refinement step (1 on, 0 off,
        -1 automatic, -2 unchanged); returns the current factorization's estimate E (-1:
        none yet)."""
        err = ctypes.c_double(-1.0)
        self._check(self.lib.ls_set_precond_refine(self.h, int(mode), ctypes.byref(err)))
        return err.value

    def nd_stats(self) -> dict:
        s = LsNdStats()
        self._check(self.lib.ls_get_nd_stats(self.h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in LsNdStats._fields_}
