"""GB300 steady-state memristor-crossbar solver: Python binding of libmca.so.

Argument marshalling only; every step of the solve runs in the library's CUDA kernels.
The binding takes NumPy arrays (host) or torch CUDA tensors (device) and passes their
pointers through the C ABI declared in include/mca.h.  It fails loudly when the library
is missing or no GPU is present; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

PREC_FP64 = 0
PREC_BF16 = 1
PREC_BF16_SPLIT = 2
PREC_MHAT = 3
PREC_JACOBI = 4
PREC_NONE = 5

FLAG_GRAPHS = 1
FLAG_AUTOTUNE = 2
FLAG_PAIR_GEMM = 4

DEVICE_SINH = 0
DEVICE_YAKOPCIC = 1

APPLY_PAIR = 0
APPLY_F64 = 1
APPLY_F32 = 2

OK = 0
ERR_INVALID_ARG = -1
ERR_CUDA = -2
ERR_NONFINITE = -3
ERR_NOT_CONVERGED = -4
ERR_TIMEOUT = -5
ERR_OOM = -6
ERR_UNSUPPORTED = -7

EXPORTED = (
    "mca_default_params", "mca_create", "mca_solve", "mca_destroy", "mca_strerror",
    "mca_last_error_message", "mca_residual", "mca_residual_pair", "mca_jacobian_apply",
    "mca_jacobian_apply_f32",
    "mca_precond_apply",
    "mca_eigenpairs", "mca_gmres_solve", "mca_profile", "mca_profile_read",
    "mca_kernel_launches", "mca_residual_noalloc", "mca_create_multi", "mca_solve_multi",
    "mca_solve_many", "mca_solve_from", "mca_cnn_conv", "mca_cnn_wgrad_scratch",
    "mca_cnn_conv_wgrad", "mca_cnn_prep_weights", "mca_cnn_features", "mca_cnn_target",
    "mca_cnn_guess", "mca_cnn_loss", "mca_cnn_adam", "mca_cnn_check", "mca_set_conductances",
    "mca_wait_selftest", "mca_tile_config", "mca_batch_create", "mca_batch_solve",
    "mca_batch_precond", "mca_batch_destroy", "mca_batch_profile", "mca_batch_profile_read",
)

BATCH_PHASES = ("residual", "transform_1", "transform_2_modes", "transform_3", "transform_4",
                "spmv_dots", "update", "reorth", "update_x", "other")

FAMILIES = ("residual", "spmv_dots", "reorth", "update_norm", "normalize", "small",
            "update_x", "precond_1", "precond_2", "precond_3", "precond_4")


class Params(ctypes.Structure):
    _fields_ = [
        ("rows", ctypes.c_int32), ("cols", ctypes.c_int32),
        ("g_wire_top", ctypes.c_double), ("g_wire_bot", ctypes.c_double),
        ("g_src", ctypes.c_double), ("g_term_top_right", ctypes.c_double),
        ("g_term_bot_top", ctypes.c_double), ("g_sense", ctypes.c_double),
        ("b", ctypes.c_double),
        ("precision", ctypes.c_int32), ("gmres_restart", ctypes.c_int32),
        ("max_newton", ctypes.c_int32), ("max_batch", ctypes.c_int32),
        ("newton_rtol", ctypes.c_double), ("eta0", ctypes.c_double),
        ("eta_max", ctypes.c_double),
        ("flags", ctypes.c_int32), ("device_model", ctypes.c_int32),
        ("neg_ratio", ctypes.c_double),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("newton_iters", ctypes.c_int32),
        ("gmres_iters", ctypes.c_int32), ("fallback", ctypes.c_int32),
        ("rel_residual", ctypes.c_double), ("kcl_rel_error", ctypes.c_double),
    ]


class Item(ctypes.Structure):
    """One work item of a persistent batched solve (mca_item)."""
    _fields_ = [("handle", ctypes.c_int32), ("map", ctypes.c_int32),
                ("v_in", ctypes.c_void_p), ("v_top", ctypes.c_void_p),
                ("v_bot", ctypes.c_void_p), ("i_out", ctypes.c_void_p)]


class MCAError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


_LIB = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libmca.so (building it first if it is missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_missing:
        _build.build()
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libmca.so not built ({path})")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    lib.mca_default_params.argtypes = [ctypes.POINTER(Params)]
    lib.mca_default_params.restype = None
    lib.mca_create.argtypes = [ctypes.POINTER(Params), P, ctypes.POINTER(P)]
    lib.mca_create_multi.argtypes = [ctypes.POINTER(Params), P, ctypes.c_int32, ctypes.POINTER(P)]
    lib.mca_solve_multi.argtypes = [P, P, P, ctypes.c_int32, P, P, P, P, P]
    lib.mca_solve_many.argtypes = [P, ctypes.c_int32, P, P, P, P, P, P, P, ctypes.c_int32]
    lib.mca_solve.argtypes = [P, P, ctypes.c_int32, P, P, P, P, P]
    lib.mca_destroy.argtypes = [P]
    lib.mca_destroy.restype = None
    lib.mca_strerror.argtypes = [ctypes.c_int]
    lib.mca_strerror.restype = ctypes.c_char_p
    lib.mca_last_error_message.argtypes = []
    lib.mca_last_error_message.restype = ctypes.c_char_p
    lib.mca_residual.argtypes = [P, P, P, ctypes.c_int32, P, P, P, P, P]
    lib.mca_jacobian_apply.argtypes = [P, P, P, P, ctypes.c_int32, P]
    lib.mca_jacobian_apply_f32.argtypes = [P, P, P, P, ctypes.c_int32, ctypes.c_int32, P]
    lib.mca_residual_pair.argtypes = [P, P, P, ctypes.c_int32, P, P, P, P, P, P]
    lib.mca_precond_apply.argtypes = [P, P, P, P, ctypes.c_int32, ctypes.c_int32, P]
    lib.mca_eigenpairs.argtypes = [P, P, P, P, P]
    lib.mca_gmres_solve.argtypes = [P, P, P, P, P, ctypes.c_int32, ctypes.c_double,
                                    ctypes.c_int32, P, P, P]
    lib.mca_profile.argtypes = [P, ctypes.c_int32]
    lib.mca_profile_read.argtypes = [P, ctypes.c_int32, P, P, P, P]
    lib.mca_residual_noalloc.argtypes = [ctypes.POINTER(Params), P, P, P, ctypes.c_int32, P, P,
                                         P, P, P]
    lib.mca_residual_noalloc.restype = ctypes.c_int
    lib.mca_solve_from.argtypes = [P, P, P, P, P, ctypes.c_int32, P, P, P, P, P]
    lib.mca_set_conductances.argtypes = [P, P]
    lib.mca_tile_config.argtypes = [P, P]
    lib.mca_tile_config.restype = ctypes.c_int
    lib.mca_wait_selftest.argtypes = [P, ctypes.c_int64]
    lib.mca_wait_selftest.restype = ctypes.c_int
    lib.mca_set_conductances.restype = ctypes.c_int
    I, F = ctypes.c_int32, ctypes.c_float
    lib.mca_cnn_conv.argtypes = [P, I, I, I, P, I, I, I, I, P, I, I, P, P, P, P]
    lib.mca_cnn_wgrad_scratch.argtypes = [I, I, I, I]
    lib.mca_cnn_wgrad_scratch.restype = ctypes.c_int64
    lib.mca_cnn_conv_wgrad.argtypes = [P, P, I, I, I, I, I, I, I, P, P, P, P]
    lib.mca_cnn_prep_weights.argtypes = [P, I, I, I, I, P, P, P]
    lib.mca_cnn_features.argtypes = [P, P, P, P, P, I, I, I, F, F, P, P]
    lib.mca_cnn_target.argtypes = [P, P, P, P, I, I, I, F, F, P, P]
    lib.mca_cnn_guess.argtypes = [P, P, P, I, I, I, F, F, P, P]
    lib.mca_cnn_loss.argtypes = [P, P, ctypes.c_int64, P, P, P, P]
    lib.mca_cnn_adam.argtypes = [P, P, P, P, ctypes.c_int64, F, F, F, F, I, P]
    lib.mca_cnn_check.argtypes = [P]
    for name in ("mca_solve_from", "mca_cnn_conv", "mca_cnn_conv_wgrad", "mca_cnn_prep_weights",
                 "mca_cnn_features", "mca_cnn_target", "mca_cnn_guess", "mca_cnn_loss",
                 "mca_cnn_adam", "mca_cnn_check"):
        getattr(lib, name).restype = ctypes.c_int
    lib.mca_batch_create.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(P)]
    lib.mca_batch_solve.argtypes = [P, P, ctypes.c_int32, P, P]
    lib.mca_batch_precond.argtypes = [P, P, P, ctypes.c_int32, P]
    lib.mca_batch_profile.argtypes = [P, ctypes.c_int32]
    lib.mca_batch_profile_read.argtypes = [P, P]
    lib.mca_batch_destroy.argtypes = [P]
    lib.mca_batch_destroy.restype = None
    for name in ("mca_batch_create", "mca_batch_solve", "mca_batch_precond",
                 "mca_batch_profile", "mca_batch_profile_read"):
        getattr(lib, name).restype = ctypes.c_int
    lib.mca_kernel_launches.argtypes = []
    lib.mca_kernel_launches.restype = ctypes.c_int64
    for name in ("mca_create", "mca_create_multi", "mca_solve_multi", "mca_solve_many",
                 "mca_solve", "mca_residual", "mca_residual_pair", "mca_jacobian_apply",
                 "mca_jacobian_apply_f32",
                 "mca_precond_apply", "mca_eigenpairs", "mca_gmres_solve", "mca_profile",
                 "mca_profile_read"):
        getattr(lib, name).restype = ctypes.c_int
    _LIB = lib
    return lib


def _check(rc, allow=()):
    if rc != OK and rc not in allow:
        lib = load(False)
        detail = lib.mca_last_error_message().decode()
        raise MCAError(rc, f"{lib.mca_strerror(rc).decode()}: {detail}")
    return rc


def _ptr(a):
    """Device pointer of a torch tensor or host pointer of a NumPy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def kernel_launches():
    """Kernel launches made by the library in this process."""
    return int(load().mca_kernel_launches())


def solve_many(solvers, vins, map_indices=None, n_threads=4, outs=None):
    """Solve several Solver objects concurrently (host threads, one stream each).  vins[k]
    is a host array or device tensor (nvec_k, m_k); outs[k] = (v_top, v_bot, i_out)
    buffers (host or device, default host NumPy).  Returns per solver (v_top, v_bot,
    i_out, stats)."""
    lib = load()
    nh = len(solvers)
    H = (ctypes.c_void_p * nh)(*[s.h.value for s in solvers])
    vins = [np.ascontiguousarray(v, np.float64) if isinstance(v, np.ndarray) else v
            for v in vins]
    if outs is None:
        outs = [(np.empty((v.shape[0], s.m, s.n)), np.empty((v.shape[0], s.m, s.n)),
                 np.empty((v.shape[0], s.n))) for s, v in zip(solvers, vins)]
    outs = [tuple(o) + ((Stats * v.shape[0])(),) for o, v in zip(outs, vins)]
    PA = ctypes.c_void_p * nh
    VIN = PA(*[_ptr(v) for v in vins])
    mis = None
    if map_indices is not None:
        keep = [np.ascontiguousarray(x, np.int32) for x in map_indices]
        mis = PA(*[x.ctypes.data for x in keep])
    NV = (ctypes.c_int32 * nh)(*[v.shape[0] for v in vins])
    VT = PA(*[_ptr(o[0]) for o in outs])
    VB = PA(*[_ptr(o[1]) for o in outs])
    IO = PA(*[_ptr(o[2]) for o in outs])
    ST = PA(*[ctypes.cast(o[3], ctypes.c_void_p).value for o in outs])
    _check(lib.mca_solve_many(H, nh, VIN, mis, NV, VT, VB, IO, ST, n_threads))
    res = []
    for o in outs:
        stats = [dict(status=x.status, newton_iters=x.newton_iters, gmres_iters=x.gmres_iters,
                      rel_residual=x.rel_residual, kcl_rel_error=x.kcl_rel_error,
                      fallback=x.fallback) for x in o[3]]
        res.append((o[0], o[1], o[2], stats))
    return res


class Batch:
    """Persistent batched solve over several Solver objects (shapes): one kernel launch
    solves every (solver, map, input vector) item, one item per CTA at a time."""

    def __init__(self, solvers, max_ctas=0):
        self.lib = load()
        self.solvers = list(solvers)
        H = (ctypes.c_void_p * len(self.solvers))(*[x.h.value for x in self.solvers])
        b = ctypes.c_void_p()
        _check(self.lib.mca_batch_create(H, len(self.solvers), max_ctas, ctypes.byref(b)))
        self.b = b

    def close(self):
        if getattr(self, "b", None):
            self.lib.mca_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @staticmethod
    def items(handles, maps, vins, v_tops=None, v_bots=None, i_outs=None):
        """An Item array from per-item handle and map indices and device tensors (rows of
        2-D tensors or separate tensors; None entries give NULL)."""
        n = len(handles)
        arr = (Item * n)()
        for k in range(n):
            arr[k].handle = int(handles[k])
            arr[k].map = int(maps[k])
            arr[k].v_in = _ptr(vins[k])
            arr[k].v_top = _ptr(v_tops[k]) if v_tops is not None else None
            arr[k].v_bot = _ptr(v_bots[k]) if v_bots is not None else None
            arr[k].i_out = _ptr(i_outs[k]) if i_outs is not None else None
        return arr

    def solve_items(self, items, stream=None, allow_not_converged=False):
        """Solve an Item array; returns the per-item stats dicts."""
        n = len(items)
        st = (Stats * n)()
        rc = self.lib.mca_batch_solve(self.b, ctypes.cast(items, ctypes.c_void_p), n,
                                      ctypes.cast(st, ctypes.c_void_p), _stream_ptr(stream))
        _check(rc, (ERR_NOT_CONVERGED, ERR_NONFINITE) if allow_not_converged else ())
        return [dict(status=x.status, newton_iters=x.newton_iters, gmres_iters=x.gmres_iters,
                     rel_residual=x.rel_residual, kcl_rel_error=x.kcl_rel_error,
                     fallback=x.fallback) for x in st]

    def profile(self, enable=True):
        _check(self.lib.mca_batch_profile(self.b, 1 if enable else 0))

    def profile_read(self):
        """CTA-milliseconds per phase (BATCH_PHASES order) since profiling was enabled."""
        ms = np.zeros(len(BATCH_PHASES))
        _check(self.lib.mca_batch_profile_read(self.b, ms.ctypes.data))
        return dict(zip(BATCH_PHASES, ms.tolist()))

    def precond(self, items, a, stream=None):
        """z = P^-1 r in place on each item's (v_top, v_bot) with a1 = a2 = a[k]."""
        n = len(items)
        av = np.ascontiguousarray(a, np.float64)
        _check(self.lib.mca_batch_precond(self.b, ctypes.cast(items, ctypes.c_void_p),
                                          av.ctypes.data, n, _stream_ptr(stream)))


def residual_noalloc(params, gmap, x, vin, F, D, fnorm=None, dmean=None, stream=None):
    """mca_residual_noalloc on device tensors (no handle, no device allocation)."""
    rc = load().mca_residual_noalloc(ctypes.byref(params), _ptr(gmap), _ptr(x), _ptr(vin),
                                     x.shape[0], _ptr(F), _ptr(D), _ptr(fnorm), _ptr(dmean),
                                     _stream_ptr(stream))
    return _check(rc)


def default_params(rows, cols, **kw):
    lib = load()
    p = Params()
    lib.mca_default_params(ctypes.byref(p))
    p.rows = rows
    p.cols = cols
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Solver:
    """One crossbar: ``Solver(params, gmap)`` then ``solve(vin)``."""

    def __init__(self, params: Params, gmap):
        """gmap: (m, n) for one crossbar, or (k, m, n) for k crossbars of this shape."""
        self.lib = load()
        self.params = params
        self.m, self.n = params.rows, params.cols
        g = gmap if not isinstance(gmap, np.ndarray) else np.ascontiguousarray(gmap, np.float64)
        self.n_maps = int(g.shape[0]) if g.ndim == 3 else 1
        h = ctypes.c_void_p()
        _check(self.lib.mca_create_multi(ctypes.byref(params), _ptr(g), self.n_maps,
                                         ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.mca_destroy(self.h)
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

    def solve(self, vin, v_top=None, v_bot=None, i_out=None, stream=None,
              allow_not_converged=False, map_index=None):
        """Solve for ``nvec`` input vectors.  ``vin`` is (nvec, m) host or device; the
        output buffers default to host NumPy arrays; ``map_index`` (nvec ints) picks each
        vector's crossbar in a multi-map solver.  Returns (v_top, v_bot, i_out, stats)."""
        nvec = vin.shape[0] if vin.ndim == 2 else 1
        mi = None if map_index is None else np.ascontiguousarray(map_index, np.int32)
        if isinstance(vin, np.ndarray):
            vin = np.ascontiguousarray(vin, np.float64)
        if v_top is None:
            v_top = np.empty((nvec, self.m, self.n))
        if v_bot is None:
            v_bot = np.empty((nvec, self.m, self.n))
        if i_out is None:
            i_out = np.empty((nvec, self.n))
        st = (Stats * nvec)()
        rc = self.lib.mca_solve_multi(self.h, _ptr(vin), _ptr(mi), nvec, _ptr(v_top),
                                      _ptr(v_bot), _ptr(i_out), ctypes.cast(st, ctypes.c_void_p),
                                      _stream_ptr(stream))
        allow = (ERR_NOT_CONVERGED, ERR_NONFINITE) if allow_not_converged else ()
        _check(rc, allow)
        stats = [dict(status=s.status, newton_iters=s.newton_iters, gmres_iters=s.gmres_iters,
                      rel_residual=s.rel_residual, kcl_rel_error=s.kcl_rel_error,
                      fallback=s.fallback) for s in st]
        return v_top, v_bot, i_out, stats

    def set_conductances(self, gmaps):
        """Replace the crossbars' conductance maps (same count and shape)."""
        g = gmaps if not isinstance(gmaps, np.ndarray) else np.ascontiguousarray(gmaps, np.float64)
        _check(self.lib.mca_set_conductances(self.h, _ptr(g)))

    def solve_from(self, vin, guess, v_top=None, v_bot=None, i_out=None, stream=None,
                   map_index=None, allow_not_converged=False, fallback=None):
        """Newton from a device guess (nvec, 2*m*n) FP64 with the fallback rule of
        mca_solve_from (fallback: device states of the same shape, or None for V = 0);
        returns (v_top, v_bot, i_out, stats)."""
        nvec = vin.shape[0]
        mi = None if map_index is None else np.ascontiguousarray(map_index, np.int32)
        if isinstance(vin, np.ndarray):
            vin = np.ascontiguousarray(vin, np.float64)
        if v_top is None:
            v_top = np.empty((nvec, self.m, self.n))
        if v_bot is None:
            v_bot = np.empty((nvec, self.m, self.n))
        if i_out is None:
            i_out = np.empty((nvec, self.n))
        st = (Stats * nvec)()
        rc = self.lib.mca_solve_from(self.h, _ptr(vin), _ptr(guess), _ptr(fallback), _ptr(mi),
                                     nvec, _ptr(v_top),
                                     _ptr(v_bot), _ptr(i_out), ctypes.cast(st, ctypes.c_void_p),
                                     _stream_ptr(stream))
        _check(rc, (ERR_NOT_CONVERGED, ERR_NONFINITE) if allow_not_converged else ())
        stats = [dict(status=s.status, newton_iters=s.newton_iters, gmres_iters=s.gmres_iters,
                      rel_residual=s.rel_residual, kcl_rel_error=s.kcl_rel_error,
                      fallback=s.fallback) for s in st]
        return v_top, v_bot, i_out, stats

    def solve_raw(self, vin_ptr, nvec, vt_ptr, vb_ptr, io_ptr, stats_ptr=None, stream=None):
        """Pointer-level call of mca_solve (no allocation, no checks); returns the status."""
        return self.lib.mca_solve(self.h, vin_ptr, nvec, vt_ptr, vb_ptr, io_ptr, stats_ptr,
                                  _stream_ptr(stream))

    def solve_multi_raw(self, vin_ptr, map_ptr, nvec, vt_ptr, vb_ptr, io_ptr, stats_ptr=None,
                        stream=None):
        """Pointer-level call of mca_solve_multi (map_ptr: host int32 map indices or None);
        returns the status."""
        return self.lib.mca_solve_multi(self.h, vin_ptr, map_ptr, nvec, vt_ptr, vb_ptr, io_ptr,
                                        stats_ptr, _stream_ptr(stream))

    def tile_config(self):
        """[(persistent, tile columns, layers per tile)] of the four tensor-core transforms."""
        cfg = (ctypes.c_int32 * 12)()
        _check(self.lib.mca_tile_config(self.h, ctypes.addressof(cfg)))
        return [tuple(cfg[3 * s:3 * s + 3]) for s in range(4)]

    def profile(self, enable=True):
        _check(self.lib.mca_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """{family: dict(launches, ms, bytes, flops)} since profiling was enabled."""
        out = {}
        for f, name in enumerate(FAMILIES):
            n = ctypes.c_int64()
            ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            _check(self.lib.mca_profile_read(self.h, f, ctypes.addressof(n), ctypes.addressof(ms),
                                             ctypes.addressof(by), ctypes.addressof(fl)))
            out[name] = dict(launches=n.value, ms=ms.value, bytes=by.value, flops=fl.value)
        return out

    # ---- single operations (device tensors) ---------------------------------------
    def residual(self, x, vin, F, D, stream=None):
        nvec = x.shape[0]
        fn = np.zeros(nvec)
        dm = np.zeros(nvec)
        _check(self.lib.mca_residual(self.h, _ptr(x), _ptr(vin), nvec, _ptr(F), _ptr(D),
                                     _ptr(fn), _ptr(dm), _stream_ptr(stream)))
        return fn, dm

    def residual_pair(self, x, vin, F, D, stream=None):
        """The FP32-pair residual; returns (||F||, mean(D), error bound on ||F||)."""
        nvec = x.shape[0]
        fn = np.zeros(nvec)
        dm = np.zeros(nvec)
        fe = np.zeros(nvec)
        _check(self.lib.mca_residual_pair(self.h, _ptr(x), _ptr(vin), nvec, _ptr(F), _ptr(D),
                                          _ptr(fn), _ptr(dm), _ptr(fe), _stream_ptr(stream)))
        return fn, dm, fe

    def jacobian_apply(self, D, z, w, stream=None):
        _check(self.lib.mca_jacobian_apply(self.h, _ptr(D), _ptr(z), _ptr(w), z.shape[0],
                                           _stream_ptr(stream)))

    def jacobian_apply_f32(self, D, z, w, mode=None, stream=None):
        """w = J z with FP32 z; mode APPLY_PAIR (the solver's form), APPLY_F64 or APPLY_F32."""
        _check(self.lib.mca_jacobian_apply_f32(self.h, _ptr(D), _ptr(z), _ptr(w), z.shape[0],
                                               APPLY_PAIR if mode is None else mode,
                                               _stream_ptr(stream)))

    def precond_apply(self, a, r, z, precision=None, stream=None):
        a = np.ascontiguousarray(a, np.float64)
        prec = self.params.precision if precision is None else precision
        _check(self.lib.mca_precond_apply(self.h, _ptr(a), _ptr(r), _ptr(z), r.shape[0], prec,
                                          _stream_ptr(stream)))

    def eigenpairs(self):
        mu = np.empty(self.n)
        qr = np.empty((self.n, self.n))
        nu = np.empty(self.m)
        qc = np.empty((self.m, self.m))
        _check(self.lib.mca_eigenpairs(self.h, _ptr(mu), _ptr(qr), _ptr(nu), _ptr(qc)))
        return mu, qr, nu, qc

    def gmres_solve(self, D, a, rhs, dx, rtol, max_iters=0, stream=None):
        """Restarted FGMRES on J dx = rhs from dx = 0 (max_iters <= 0: one cycle)."""
        a = np.ascontiguousarray(a, np.float64)
        nvec = rhs.shape[0]
        its = np.zeros(nvec, np.int32)
        res = np.zeros(nvec)
        _check(self.lib.mca_gmres_solve(self.h, _ptr(D), _ptr(a), _ptr(rhs), _ptr(dx), nvec,
                                        rtol, int(max_iters), _ptr(its), _ptr(res),
                                        _stream_ptr(stream)))
        return its, res
