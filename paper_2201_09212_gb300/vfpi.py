"""Thin ctypes binding of ``libvfpi`` (the C ABI in ``include/vfpi.h``).

Argument marshalling only: arrays may be numpy arrays (host memory) or torch
tensors (host or CUDA); the library itself detects which and every step of the
solve runs in its CUDA kernels.  There is no fallback: if the library is not
built, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from . import build as _build

VFPI_OK = 0
VFPI_NOT_CONVERGED = 1
STATUS_NAMES = {0: "VFPI_OK", 1: "VFPI_NOT_CONVERGED", -1: "VFPI_ERR_INVALID_ARG",
                -2: "VFPI_ERR_NONFINITE", -3: "VFPI_ERR_CUDA", -4: "VFPI_ERR_OOM",
                -5: "VFPI_ERR_TIMEOUT", -6: "VFPI_ERR_CONTACT_OVERLAP",
                -7: "VFPI_ERR_UNSUPPORTED"}
STATUS_CODES = {name: code for code, name in STATUS_NAMES.items()}
DTYPES = {"f32": (0, np.float32), "f64": (1, np.float64)}
W_MODES = {"frobenius": 0, "scalar": 1, "user": 2}
NORMS = {"abs": 0, "rms": 1}
OPERATORS = {"strict": 0, "proximal": 1}

EXPORTED = ("vfpi_default_opts", "vfpi_create", "vfpi_update", "vfpi_set_rhs",
            "vfpi_set_velocity", "vfpi_get_velocity", "vfpi_get_lambda", "vfpi_get_w",
            "vfpi_step", "vfpi_solve", "vfpi_solve_async", "vfpi_get_status",
            "vfpi_get_scene_status",
            "vfpi_get_lambda_star", "vfpi_set_friction", "vfpi_adjoint",
            "vfpi_integrate", "vfpi_advance", "vfpi_matvec", "vfpi_last_kernel_ms", "vfpi_get_layout",
            "vfpi_get_storage",
            "vfpi_configure_launch", "vfpi_set_tolerance", "vfpi_set_chebyshev",
            "vfpi_set_adjoint_chebyshev", "vfpi_set_adjoint_tolerance",
            "vfpi_set_regularization", "vfpi_set_anisotropic_friction",
            "vfpi_set_barzilai_borwein",
            "vfpi_last_error", "vfpi_status_string", "vfpi_destroy", "vfpi_solve_noalloc",
            "vfpi_noalloc_last_error", "vfpi_shard_sweep", "vfpi_get_nodes", "vfpi_set_halo",
            "vfpi_get_shard_info", "vfpi_get_split_stats", "vfpi_set_split_stats",
            "vfpi_get_split_vstar", "vfpi_finish_split", "vfpi_shard_set_theta")


class VfpiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class _Bsr(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("nnzb", C.c_int32), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("vals", C.c_void_p)]


class _Contacts(C.Structure):
    _fields_ = [("n_c", C.c_int32), ("node_i", C.c_void_p), ("node_j", C.c_void_p),
                ("R", C.c_void_p), ("mu", C.c_void_p), ("phi", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("w_mode", C.c_int32), ("alpha", C.c_double),
                ("w_user", C.c_void_p), ("theta_th", C.c_double), ("l_max", C.c_int32),
                ("operator_", C.c_int32), ("residual_norm", C.c_int32), ("n_scenes", C.c_int32),
                ("scene_ptr", C.c_void_p), ("block_threads", C.c_int32),
                ("force_path", C.c_int32), ("kernel_variant", C.c_int32),
                ("grid_ctas", C.c_int32), ("chebyshev_ls", C.c_int32),
                ("chebyshev_u", C.c_double), ("n_halo", C.c_int32), ("reserved", C.c_int32)]


_LIB = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load ``libvfpi.so`` (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2201_09212_gb300.build.build()")
    L = C.CDLL(path)
    vp, i32, st = C.c_void_p, C.c_int32, C.c_int
    sig = {
        "vfpi_default_opts": (None, [vp]),
        "vfpi_create": (st, [vp, vp, vp, C.c_double, vp, vp, vp]),
        "vfpi_update": (st, [vp, vp, vp, vp]),
        "vfpi_set_rhs": (st, [vp, vp, vp]),
        "vfpi_set_velocity": (st, [vp, vp]),
        "vfpi_get_velocity": (st, [vp, vp]),
        "vfpi_get_lambda": (st, [vp, vp]),
        "vfpi_get_w": (st, [vp, vp]),
        "vfpi_get_lambda_star": (st, [vp, vp]),
        "vfpi_set_friction": (st, [vp, vp]),
        "vfpi_adjoint": (st, [vp, vp, vp, vp, vp, vp, vp, vp]),
        "vfpi_step": (st, [vp, vp]),
        "vfpi_solve": (st, [vp, vp, vp, vp, vp]),
        "vfpi_solve_async": (st, [vp]),
        "vfpi_get_status": (st, [vp, vp, vp]),
        "vfpi_get_scene_status": (st, [vp, vp]),
        "vfpi_integrate": (st, [vp, vp]),
        "vfpi_advance": (st, [vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "vfpi_matvec": (st, [vp, vp, vp]),
        "vfpi_last_kernel_ms": (st, [vp, vp]),
        "vfpi_configure_launch": (st, [vp, i32, i32, i32]),
        "vfpi_set_tolerance": (st, [vp, C.c_double, i32]),
        "vfpi_set_chebyshev": (st, [vp, i32, C.c_double]),
        "vfpi_set_adjoint_chebyshev": (st, [vp, i32, C.c_double]),
        "vfpi_set_adjoint_tolerance": (st, [vp, C.c_double, i32, i32]),
        "vfpi_set_regularization": (st, [vp, vp]),
        "vfpi_set_anisotropic_friction": (st, [vp, vp]),
        "vfpi_set_barzilai_borwein": (st, [vp, i32, C.c_double]),
        "vfpi_get_layout": (st, [vp, vp]),
        "vfpi_get_storage": (st, [vp, vp]),
        "vfpi_last_error": (C.c_char_p, [vp]),
        "vfpi_status_string": (C.c_char_p, [st]),
        "vfpi_destroy": (None, [vp]),
        "vfpi_solve_noalloc": (st, [vp, vp, vp, C.c_double, i32, i32, vp, vp, vp, vp, vp, vp]),
        "vfpi_noalloc_last_error": (C.c_char_p, []),
        "vfpi_shard_sweep": (st, [vp, vp]),
        "vfpi_get_nodes": (st, [vp, vp, i32, vp]),
        "vfpi_set_halo": (st, [vp, i32, i32, vp]),
        "vfpi_get_shard_info": (st, [vp, vp]),
        "vfpi_get_split_stats": (st, [vp, vp]),
        "vfpi_set_split_stats": (st, [vp, vp]),
        "vfpi_get_split_vstar": (st, [vp, vp]),
        "vfpi_finish_split": (st, [vp, vp, vp]),
        "vfpi_shard_set_theta": (st, [vp, C.c_double]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


class _Keep:
    """Holds converted arrays alive for the duration of a call."""

    def __init__(self):
        self.refs = []

    def ptr(self, a, dtype=None):
        if a is None:
            return None
        if _is_torch(a):
            if not a.is_contiguous():
                raise ValueError("tensors passed to libvfpi must be contiguous")
            if dtype is not None and a.dtype != _torch_dtype(dtype):
                raise TypeError(f"expected {np.dtype(dtype)} tensor, got {a.dtype}")
            self.refs.append(a)
            return a.data_ptr()
        arr = np.ascontiguousarray(a, dtype=dtype)
        self.refs.append(arr)
        return arr.ctypes.data


def _torch_dtype(dt):
    import torch
    return {np.dtype(np.float32): torch.float32, np.dtype(np.float64): torch.float64,
            np.dtype(np.int32): torch.int32}[np.dtype(dt)]


@dataclasses.dataclass
class SolveResult:
    v: object
    lam: object
    iters: object
    theta: object
    status: int

    @property
    def converged(self) -> bool:
        return self.status == VFPI_OK


class Solver:
    """One V-FPI problem (or a batch of independent scenes) resident on the GPU."""

    def __init__(self, row_ptr, col_idx, vals, b, node_i, node_j, R, mu, phi, *, h=1e-3,
                 dtype="f32", w_mode="frobenius", alpha=0.0, w_user=None, theta_th=1e-5,
                 l_max=200, norm="abs", scene_ptr=None, block_threads=0, force_path=0,
                 kernel_variant=0, grid_ctas=0, chebyshev_ls=0, chebyshev_u=1.0,
                 operator="strict", n_halo=0, stream=None):
        self._L = lib()
        self.dtype_code, self.np_dtype = DTYPES[dtype]
        self.n_nodes = int(len(row_ptr) - 1)
        self.n = 3 * self.n_nodes
        self.n_c = int(len(node_i))
        self.n_scenes = 1 if scene_ptr is None else int(len(scene_ptr) - 1)
        k = _Keep()
        fd = self.np_dtype
        bsr = _Bsr(self.n_nodes, int(len(col_idx)), k.ptr(row_ptr, np.int32),
                   k.ptr(col_idx, np.int32), k.ptr(vals, fd))
        con = _Contacts(self.n_c, k.ptr(node_i, np.int32),
                        k.ptr(node_j, np.int32) if node_j is not None else None,
                        k.ptr(R, fd), k.ptr(mu, fd), k.ptr(phi, fd))
        o = _Opts()
        self._L.vfpi_default_opts(C.byref(o))
        o.dtype = self.dtype_code
        o.w_mode = W_MODES[w_mode]
        o.alpha = float(alpha)
        o.w_user = k.ptr(w_user, fd)
        o.theta_th = float(theta_th)
        o.l_max = int(l_max)
        o.residual_norm = NORMS[norm]
        o.operator_ = OPERATORS[operator]
        o.n_scenes = self.n_scenes
        o.scene_ptr = k.ptr(scene_ptr, np.int32)
        o.block_threads = int(block_threads)
        o.force_path = int(force_path)
        o.kernel_variant = int(kernel_variant)
        o.grid_ctas = int(grid_ctas)
        o.chebyshev_ls = int(chebyshev_ls)
        o.chebyshev_u = float(chebyshev_u)
        o.n_halo = int(n_halo)
        self.n_halo = int(n_halo)
        self.h = float(h)
        self._theta_th, self._l_max = float(theta_th), int(l_max)
        self.stream = stream
        sptr = None
        if stream is not None:
            sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        handle = C.c_void_p()
        st = self._L.vfpi_create(C.byref(bsr), k.ptr(b, fd), C.byref(con), C.c_double(h),
                                 C.byref(o), sptr, C.byref(handle))
        if st != VFPI_OK:
            raise VfpiError(st, self._L.vfpi_last_error(None).decode())
        self._h = handle

    @classmethod
    def from_scene(cls, scene, **kw):
        dtype = kw.pop("dtype", "f64" if scene.vals.dtype == np.float64 else "f32")
        return cls(scene.row_ptr, scene.col_idx, scene.vals, scene.b, scene.node_i, scene.node_j,
                   scene.R, scene.mu, scene.phi, h=scene.h, dtype=dtype,
                   scene_ptr=kw.pop("scene_ptr", scene.scene_ptr), **kw)

    # ------------------------------------------------------------------ utils
    def _check(self, st, allow_nc=False):
        if st == VFPI_OK or (allow_nc and st == VFPI_NOT_CONVERGED):
            return st
        raise VfpiError(st, self._L.vfpi_last_error(self._h).decode())

    def _out(self, shape, out, dtype=None):
        if out is not None:
            return out
        return np.empty(shape, dtype=dtype or self.np_dtype)

    def close(self):
        if getattr(self, "_h", None):
            self._L.vfpi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------ calls
    def solve(self, v=None, want_lambda=True, out_v=None, out_lam=None) -> SolveResult:
        """Alg. 1 to theta < theta_th or l_max from warm start ``v`` (or the current
        iterate).  Returns host arrays unless ``out_*`` tensors are given."""
        k = _Keep()
        vv = None
        if v is not None:
            if out_v is not None:
                out_v.copy_(v) if _is_torch(out_v) else np.copyto(out_v, v)
                vv = out_v
            elif _is_torch(v):
                vv = v.clone()
            else:
                vv = np.array(v, dtype=self.np_dtype, copy=True)
        lam = self._out(3 * self.n_c, out_lam) if want_lambda else None
        iters = np.zeros(self.n_scenes, dtype=np.int32)
        theta = np.zeros(self.n_scenes, dtype=np.float64)
        st = self._L.vfpi_solve(self._h, k.ptr(vv, self.np_dtype), k.ptr(lam, self.np_dtype),
                                iters.ctypes.data, theta.ctypes.data)
        self._check(st, allow_nc=True)
        if vv is None:
            vv = self.get_velocity()
        if self.n_scenes == 1:
            return SolveResult(vv, lam, int(iters[0]), float(theta[0]), st)
        return SolveResult(vv, lam, iters, theta, st)

    def solve_async(self):
        self._check(self._L.vfpi_solve_async(self._h))

    def status(self):
        iters = np.zeros(self.n_scenes, dtype=np.int32)
        theta = np.zeros(self.n_scenes, dtype=np.float64)
        st = self._check(self._L.vfpi_get_status(self._h, iters.ctypes.data, theta.ctypes.data),
                         allow_nc=True)
        return iters, theta, st

    # ---------------------------------------------------------- sharded scene
    def shard_sweep(self, sumsq=True):
        """One sweep of this shard's rows (halo values as last set); returns the
        shard's FP64 sum of squares of the update over its rows (without the
        own endpoints of split contacts), or None, without waiting for the
        GPU, when ``sumsq`` is false."""
        if not sumsq:
            self._check(self._L.vfpi_shard_sweep(self._h, None))
            return None
        s2 = C.c_double()
        self._check(self._L.vfpi_shard_sweep(self._h, C.byref(s2)))
        return float(s2.value)

    def shard_set_theta(self, theta):
        """The whole scene's theta of the sweep just taken (the solve goes on):
        the shard's next sweep follows it, with Alg. 3 at the weight these
        thetas give."""
        self._check(self._L.vfpi_shard_set_theta(self._h, float(theta)))

    def shard_info(self):
        """(n_halo, n_split): halo nodes and split contacts (D-contacts with one
        node in the halo) of this shard."""
        info = np.zeros(2, dtype=np.int32)
        self._check(self._L.vfpi_get_shard_info(self._h, info.ctypes.data))
        return int(info[0]), int(info[1])

    def split_stats(self, out=None):
        """[6 n_split] FP64 row statistics (a_rr, ||A_r*||^2 of the three DOFs) of
        each split contact's own endpoint."""
        out = self._out(6 * self.shard_info()[1], out, np.float64)
        k = _Keep()
        self._check(self._L.vfpi_get_split_stats(self._h, k.ptr(out, np.float64)))
        return out

    def set_split_stats(self, partner):
        """The other endpoints' statistics, [6 n_split] FP64 (W is formed again)."""
        k = _Keep()
        self._check(self._L.vfpi_set_split_stats(self._h, k.ptr(partner, np.float64)))

    def split_vstar(self, out=None):
        """[3 n_split] v* of each split contact's own endpoint, from the last sweep."""
        out = self._out(3 * self.shard_info()[1], out)
        k = _Keep()
        self._check(self._L.vfpi_get_split_vstar(self._h, k.ptr(out, self.np_dtype)))
        return out

    def finish_split(self, partner_vstar) -> float:
        """Second half of the sweep from the other endpoints' v* [3 n_split];
        returns the shard's whole FP64 sum of squares of the sweep."""
        s2 = C.c_double()
        k = _Keep()
        self._check(self._L.vfpi_finish_split(self._h, k.ptr(partner_vstar, self.np_dtype),
                                              C.byref(s2)))
        return float(s2.value)

    def get_nodes(self, nodes, out=None):
        """v of own nodes ``nodes`` (indices < n_nodes), [3 * len(nodes)]."""
        out = self._out(3 * len(nodes), out)
        k = _Keep()
        self._check(self._L.vfpi_get_nodes(self._h, k.ptr(nodes, np.int32), int(len(nodes)),
                                           k.ptr(out, self.np_dtype)))
        return out

    def set_halo(self, first, vals):
        """v of halo nodes [first, first + len(vals) / 3)."""
        k = _Keep()
        self._check(self._L.vfpi_set_halo(self._h, int(first), int(len(vals) // 3),
                                          k.ptr(vals, self.np_dtype)))

    def scene_status(self):
        """Per-scene outcome of the last solve or adjoint solve (status codes)."""
        out = np.zeros(self.n_scenes, dtype=np.int32)
        self._check(self._L.vfpi_get_scene_status(self._h, out.ctypes.data))
        return out

    def step(self) -> float:
        theta = np.zeros(max(self.n_scenes, 1), dtype=np.float64)
        self._check(self._L.vfpi_step(self._h, theta.ctypes.data))
        return float(theta[0]) if self.n_scenes == 1 else theta

    def set_velocity(self, v):
        k = _Keep()
        self._check(self._L.vfpi_set_velocity(self._h, k.ptr(v, self.np_dtype)))

    def get_velocity(self, out=None):
        out = self._out(self.n, out)
        k = _Keep()
        self._check(self._L.vfpi_get_velocity(self._h, k.ptr(out, self.np_dtype)))
        return out

    def get_lambda(self, out=None):
        out = self._out(3 * self.n_c, out)
        k = _Keep()
        self._check(self._L.vfpi_get_lambda(self._h, k.ptr(out, self.np_dtype)))
        return out

    def get_lambda_star(self, out=None):
        out = self._out(3 * self.n_c, out)
        k = _Keep()
        self._check(self._L.vfpi_get_lambda_star(self._h, k.ptr(out, self.np_dtype)))
        return out

    def set_friction(self, mu):
        k = _Keep()
        self._check(self._L.vfpi_set_friction(self._h, k.ptr(mu, self.np_dtype)))

    def adjoint(self, g_v, lambda_star=None, out_b=None, out_phi=None, out_mu=None):
        """Implicit adjoint of the converged solve: returns (dL/db, dL/dphi, dL/dmu,
        iters, theta) for dL/dv = g_v at the active set frozen by ``lambda_star``."""
        k = _Keep()
        g_b = self._out(self.n, out_b)
        g_phi = self._out(self.n_c, out_phi)
        g_mu = self._out(self.n_c, out_mu)
        iters = np.zeros(self.n_scenes, dtype=np.int32)
        theta = np.zeros(self.n_scenes, dtype=np.float64)
        st = self._L.vfpi_adjoint(self._h, k.ptr(lambda_star, self.np_dtype),
                                  k.ptr(g_v, self.np_dtype), k.ptr(g_b, self.np_dtype),
                                  k.ptr(g_phi, self.np_dtype), k.ptr(g_mu, self.np_dtype),
                                  iters.ctypes.data, theta.ctypes.data)
        self._check(st, allow_nc=True)
        if self.n_scenes == 1:
            return g_b, g_phi, g_mu, int(iters[0]), float(theta[0])
        return g_b, g_phi, g_mu, iters, theta

    def get_w(self, out=None):
        out = self._out(self.n, out)
        k = _Keep()
        self._check(self._L.vfpi_get_w(self._h, k.ptr(out, self.np_dtype)))
        return out

    def set_rhs(self, b=None, phi=None):
        k = _Keep()
        self._check(self._L.vfpi_set_rhs(self._h, k.ptr(b, self.np_dtype), k.ptr(phi, self.np_dtype)))

    def update(self, vals=None, b=None, contacts=None):
        k = _Keep()
        con = None
        if contacts is not None:
            node_i, node_j, R, mu, phi = contacts
            con = _Contacts(int(len(node_i)), k.ptr(node_i, np.int32),
                            k.ptr(node_j, np.int32) if node_j is not None else None,
                            k.ptr(R, self.np_dtype), k.ptr(mu, self.np_dtype),
                            k.ptr(phi, self.np_dtype))
            self.n_c = int(len(node_i))
        self._check(self._L.vfpi_update(self._h, k.ptr(vals, self.np_dtype), k.ptr(b, self.np_dtype),
                                        C.byref(con) if con is not None else None))

    def integrate(self, x):
        """x += h * v_hat in FP64; numpy arrays are updated in place."""
        k = _Keep()
        if _is_torch(x):
            self._check(self._L.vfpi_integrate(self._h, k.ptr(x, np.float64)))
            return x
        if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
            raise TypeError("x must be a contiguous float64 array")
        self._check(self._L.vfpi_integrate(self._h, x.ctypes.data))
        return x

    def advance(self, b=None, phi=None, v=None, out_v=None, out_lam=None, x=None) -> SolveResult:
        """One time step in one call (vfpi_advance): right-hand side ``b``/``phi``,
        warm start ``v``, Alg. 1, ``out_v``/``out_lam`` written, ``x`` (FP64,
        updated in place) integrated; one wait for the whole step.  Outputs
        are allocated as host arrays when not given."""
        k = _Keep()
        if x is not None and not _is_torch(x) and not (
                isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
            raise TypeError("x must be a contiguous float64 array")
        vo = self._out(self.n, out_v)
        lam = self._out(3 * self.n_c, out_lam)
        iters = np.zeros(self.n_scenes, dtype=np.int32)
        theta = np.zeros(self.n_scenes, dtype=np.float64)
        st = self._L.vfpi_advance(self._h, k.ptr(b, self.np_dtype), k.ptr(phi, self.np_dtype),
                                  k.ptr(v, self.np_dtype), k.ptr(vo, self.np_dtype),
                                  k.ptr(lam, self.np_dtype),
                                  None if x is None else k.ptr(x, np.float64),
                                  iters.ctypes.data, theta.ctypes.data)
        self._check(st, allow_nc=True)
        if self.n_scenes == 1:
            return SolveResult(vo, lam, int(iters[0]), float(theta[0]), st)
        return SolveResult(vo, lam, iters, theta, st)

    def matvec(self, x, out=None):
        out = self._out(self.n, out)
        k = _Keep()
        self._check(self._L.vfpi_matvec(self._h, k.ptr(x, self.np_dtype), k.ptr(out, self.np_dtype)))
        return out

    def configure_launch(self, kernel_variant=0, block_threads=0, grid_ctas=0):
        self._check(self._L.vfpi_configure_launch(self._h, int(kernel_variant), int(block_threads),
                                                  int(grid_ctas)))

    def last_kernel_ms(self) -> float:
        ms = C.c_float()
        self._check(self._L.vfpi_last_kernel_ms(self._h, C.byref(ms)))
        return float(ms.value)

    def set_tolerance(self, theta_th, l_max):
        self._check(self._L.vfpi_set_tolerance(self._h, float(theta_th), int(l_max)))
        self._theta_th, self._l_max = float(theta_th), int(l_max)

    def set_regularization(self, omega=None):
        k = _Keep()
        self._check(self._L.vfpi_set_regularization(self._h, k.ptr(omega, self.np_dtype)))

    def set_anisotropic_friction(self, mu2=None):
        k = _Keep()
        self._check(self._L.vfpi_set_anisotropic_friction(self._h, k.ptr(mu2, self.np_dtype)))

    def set_barzilai_borwein(self, rule, alpha0=0.0):
        """rule: 0 off, "bb1"/1, "bb2"/2, "alt"/3."""
        rule = {"bb1": 1, "bb2": 2, "alt": 3, None: 0}.get(rule, rule)
        self._check(self._L.vfpi_set_barzilai_borwein(self._h, int(rule), float(alpha0)))

    def set_chebyshev(self, l_s, u=1.0):
        self._check(self._L.vfpi_set_chebyshev(self._h, int(l_s), float(u)))

    def set_adjoint_chebyshev(self, l_s, u=1.0):
        """Alg. 3 for the adjoint solves only (l_s = 0: off)."""
        self._check(self._L.vfpi_set_adjoint_chebyshev(self._h, int(l_s), float(u)))

    def set_adjoint_tolerance(self, theta_th, l_max, relative=True):
        """Stop test of the adjoint solves: theta < theta_th (* ||g_v|| if relative)."""
        self._check(self._L.vfpi_set_adjoint_tolerance(self._h, float(theta_th), int(l_max),
                                                       1 if relative else 0))

    def layout(self) -> dict:
        info = (C.c_int64 * 8)()
        self._check(self._L.vfpi_get_layout(self._h, info))
        keys = ("n_pad", "n_slices", "slots", "path", "grid", "threads", "max_grid", "sms")
        return dict(zip(keys, (int(x) for x in info)))

    STORAGE_NAMES = ("full", "symmetric", "blocks6")

    def storage(self) -> dict:
        """How the solve kernels read A: the forward Alg. 1 sweep's storage in
        the current launch shape (``full``, ``symmetric`` or ``blocks6``;
        Barzilai-Borwein sweeps read ``full``) and the flags that allow the
        others."""
        info = (C.c_int32 * 4)()
        self._check(self._L.vfpi_get_storage(self._h, info))
        return {"storage": self.STORAGE_NAMES[int(info[0])], "blocks_symmetric": bool(info[1]),
                "a_symmetric": bool(info[2])}
