"""GB300-native (sm_103a) FWIME operators: thin Python binding of libfwime.

Barnier et al., "Full waveform inversion by model extension: practical
applications" (arXiv 2206.02362).  The operators of the Theory section --
f (Eq. 1), B and B* (Eq. 8), the subsurface-offset extended Born operator B~
and its adjoint B~* (Eqs. 1-5), the tomographic operator T and T* (Eq. 9) and
the FWIME gradient B* r + T* r (Eqs. 7-9) -- run entirely in the CUDA kernels
of ``libfwime.so`` (C ABI in ``include/fwime.h``).  This module only marshals
arguments: torch tensors provide device memory and streams.

There is no CPU fallback.  Importing this package loads ``libfwime.so`` (and
builds it with nvcc if it is missing); if that fails the import raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None

FWIME_OK, FWIME_EINVAL, FWIME_ENOMEM, FWIME_ECFL, FWIME_ECUDA, FWIME_ETIMEOUT, FWIME_EBUSY = 0, -1, -2, -3, -4, -5, -6
OPT_SHOTS_PER_BATCH, OPT_SEGMENT, OPT_PLAIN, OPT_GRAPH, OPT_HOST_IO, OPT_ZCHUNK, OPT_LAUNCHES, OPT_WORKSPACE = \
    1, 2, 3, 4, 5, 6, 7, 8
OPT_PROFILE = 9
OPT_REUSE_BACKGROUND = 10
OPT_BACKGROUND_REUSED = 11
OPT_TIME_LAG = 12
OPT_FREE_SURFACE = 13
OPT_BATCH_USED = 15
K_PROP, K_SCATTER, K_IMAGE, K_POINTS, K_OTHER = range(5)
KERNEL_NAMES = ("prop", "scatter", "image", "points", "other")
(OP_FORWARD, OP_BORN, OP_BORN_ADJ, OP_BORN_EXT, OP_BORN_EXT_ADJ, OP_TOMO, OP_TOMO_ADJ,
 OP_GRADIENT, OP_OBJECTIVE) = range(9)

ABI_FUNCTIONS = ("fwime_create", "fwime_workspace_bytes", "fwime_set_option", "fwime_get_option",
                 "fwime_forward", "fwime_born", "fwime_born_adj", "fwime_born_ext", "fwime_born_ext_adj",
                 "fwime_tomo", "fwime_tomo_adj", "fwime_gradient", "fwime_gradient_forward", "fwime_gradient_backward",
                 "fwime_objective", "fwime_vp_solve", "fwime_spline", "fwime_spline_refine",
                 "fwime_autotune", "fwime_autotune_schedule", "fwime_forward_group", "fwime_sync", "fwime_profile_read",
                 "fwime_last_error_detail", "fwime_strerror", "fwime_destroy",
                 "fwime_server_create", "fwime_request_bytes", "fwime_submit", "fwime_poll", "fwime_wait",
                 "fwime_server_last_error")
REQ_FORWARD, REQ_GRADIENT = 0, 1
SERVE_PLAIN = 1


class FwimeError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        msg = f"{where}: {strerror(code)} ({code})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


class GridC(ctypes.Structure):
    _fields_ = [("nz", ctypes.c_int), ("nx", ctypes.c_int), ("sponge", ctypes.c_int), ("nt", ctypes.c_int),
                ("nh", ctypes.c_int), ("dz", ctypes.c_float), ("dx", ctypes.c_float), ("dt", ctypes.c_float)]


class GeomC(ctypes.Structure):
    _fields_ = [("nshot", ctypes.c_int), ("src_iz", ctypes.POINTER(ctypes.c_int)),
                ("src_ix", ctypes.POINTER(ctypes.c_int)), ("nrec", ctypes.c_int),
                ("rec_iz", ctypes.POINTER(ctypes.c_int)), ("rec_ix", ctypes.POINTER(ctypes.c_int))]


class ScheduleC(ctypes.Structure):
    _fields_ = [("segment", ctypes.c_int), ("shots_per_batch", ctypes.c_int), ("zchunk", ctypes.c_int),
                ("us_stencil", ctypes.c_float), ("us_scatter", ctypes.c_float), ("us_image", ctypes.c_float),
                ("us_per_shot", ctypes.c_double)]


class RequestC(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("grid", GridC), ("geom", GeomC), ("host_io", ctypes.c_int),
                ("v", ctypes.c_void_p), ("w", ctypes.c_void_p), ("pt", ctypes.c_void_p), ("dobs", ctypes.c_void_p),
                ("d", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("eps", ctypes.c_float)]


class ResultC(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int), ("status", ctypes.c_int), ("objective", ctypes.c_double),
                ("queued_s", ctypes.c_double), ("latency_s", ctypes.c_double), ("enqueue_s", ctypes.c_double)]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libfwime.so (building it first if absent); raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"libfwime.so not built at {path}")
        path = _build.build()
    lib = ctypes.CDLL(path)
    vp, fp, ip = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int
    lib.fwime_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(GridC), ctypes.POINTER(GeomC), ctypes.c_size_t, vp]
    lib.fwime_workspace_bytes.argtypes = [ctypes.POINTER(GridC), ctypes.POINTER(GeomC), ip, ip, ip,
                                          ctypes.POINTER(ctypes.c_size_t)]
    lib.fwime_set_option.argtypes = [vp, ip, ctypes.c_longlong]
    lib.fwime_get_option.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_longlong)]
    lib.fwime_forward.argtypes = [vp, fp, fp, fp]
    lib.fwime_born.argtypes = [vp, fp, fp, fp, fp]
    lib.fwime_born_adj.argtypes = [vp, fp, fp, fp, fp, ip]
    lib.fwime_born_ext.argtypes = [vp, fp, fp, fp, fp]
    lib.fwime_born_ext_adj.argtypes = [vp, fp, fp, fp, fp, ip]
    lib.fwime_tomo.argtypes = [vp, fp, fp, fp, fp, fp]
    lib.fwime_tomo_adj.argtypes = [vp, fp, fp, fp, fp, fp, ip]
    lib.fwime_gradient.argtypes = [vp, fp, fp, fp, fp, ctypes.c_float, fp, ctypes.POINTER(ctypes.c_double)]
    lib.fwime_objective.argtypes = [vp, fp, fp, fp, fp, ctypes.c_float, ctypes.POINTER(ctypes.c_double)]
    lib.fwime_gradient_forward.argtypes = [vp, fp, fp, fp, fp, ctypes.c_float, ctypes.POINTER(ctypes.c_double)]
    lib.fwime_gradient_backward.argtypes = [vp, fp, fp, fp, fp, ctypes.c_float, fp, ip]
    lib.fwime_vp_solve.argtypes = [vp, fp, fp, fp, ctypes.c_float, ip, fp, ctypes.POINTER(ctypes.c_double)]
    lib.fwime_spline.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_float), ip, ctypes.POINTER(ctypes.c_float), fp, fp,
                                 ip, ip]
    fl = ctypes.POINTER(ctypes.c_float)
    lib.fwime_spline_refine.argtypes = [vp, ip, fl, ip, fl, fp, ip, fl, ip, fl, fp]
    lib.fwime_autotune.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]
    lib.fwime_autotune_schedule.argtypes = [vp, ip, ctypes.POINTER(ScheduleC)]
    lib.fwime_forward_group.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                        ctypes.POINTER(vp)]
    lib.fwime_sync.argtypes = [vp]
    lib.fwime_profile_read.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_double), ip]
    lib.fwime_last_error_detail.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.fwime_strerror.argtypes = [ip]
    lib.fwime_strerror.restype = ctypes.c_char_p
    lib.fwime_destroy.argtypes = [vp]
    lib.fwime_destroy.restype = None
    lib.fwime_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t, ip, ip]
    lib.fwime_request_bytes.argtypes = [ctypes.POINTER(RequestC), ctypes.POINTER(ctypes.c_size_t)]
    lib.fwime_submit.argtypes = [vp, ctypes.POINTER(RequestC), ctypes.POINTER(ctypes.c_uint64)]
    lib.fwime_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ResultC)]
    lib.fwime_wait.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ResultC)]
    lib.fwime_server_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    for name in ABI_FUNCTIONS:
        if name not in ("fwime_strerror", "fwime_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().fwime_strerror(int(code)).decode()


@dataclass(frozen=True)
class Grid:
    """Physical grid nz x nx at dz, dx; `sponge` absorbing points per side; nt samples at dt; nh offsets."""
    nz: int
    nx: int
    sponge: int
    nt: int
    dt: float
    dx: float
    dz: float | None = None
    nh: int = 1

    def c(self) -> GridC:
        dz = self.dx if self.dz is None else self.dz
        return GridC(self.nz, self.nx, self.sponge, self.nt, self.nh, float(dz), float(self.dx), float(self.dt))


@dataclass
class Geometry:
    """One point source per shot and a fixed receiver spread (physical-grid indices)."""
    src_iz: np.ndarray
    src_ix: np.ndarray
    rec_iz: np.ndarray
    rec_ix: np.ndarray

    @property
    def nshot(self) -> int:
        return int(len(self.src_iz))

    @property
    def nrec(self) -> int:
        return int(len(self.rec_iz))

    def c(self):
        arrs = [np.ascontiguousarray(a, dtype=np.int32) for a in (self.src_iz, self.src_ix, self.rec_iz, self.rec_ix)]
        P = ctypes.POINTER(ctypes.c_int)
        g = GeomC(self.nshot, arrs[0].ctypes.data_as(P), arrs[1].ctypes.data_as(P), self.nrec,
                  arrs[2].ctypes.data_as(P), arrs[3].ctypes.data_as(P))
        return g, arrs


def workspace_bytes(grid: Grid, geom: Geometry, op: int, shots_per_batch: int = 0, segment: int = 0) -> int:
    gc = grid.c()
    gm, keep = geom.c()
    out = ctypes.c_size_t(0)
    rc = load().fwime_workspace_bytes(ctypes.byref(gc), ctypes.byref(gm), op, shots_per_batch, segment,
                                      ctypes.byref(out))
    if rc != FWIME_OK:
        raise FwimeError(rc, "fwime_workspace_bytes")
    return int(out.value)


def _ptr(t) -> int:
    """Device (or, in host-I/O mode, host) address of a contiguous float32 tensor/array."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if t.dtype != np.float32 or not t.flags.c_contiguous:
            raise TypeError("arrays must be contiguous float32")
        return t.ctypes.data
    if t.dtype.__str__() != "torch.float32" or not t.is_contiguous():
        raise TypeError("tensors must be contiguous float32")
    return t.data_ptr()


def forward_group(contexts, vs, ws, ds, sync: bool = True):
    """f(m) for several contexts (different grids, nt, shots) with one launch per time step for all
    of them (fwime_forward_group).  vs/ws/ds: per-context device tensors as for Context.forward."""
    n = len(contexts)
    arr = lambda xs: (ctypes.c_void_p * n)(*xs)  # noqa: E731
    rc = load().fwime_forward_group(arr([c._h.value for c in contexts]), n, arr([_ptr(t) for t in vs]),
                                    arr([_ptr(t) for t in ws]), arr([_ptr(t) for t in ds]))
    if rc != FWIME_OK:
        raise FwimeError(rc, "fwime_forward_group", contexts[0].detail())
    if sync:
        for c in contexts:
            c.sync()
    return ds


class Context:
    """One fwime_ctx: a grid, an acquisition geometry, a CUDA stream and a workspace.

    Methods mirror the C ABI (``fwime_forward`` -> ``forward`` ...).  Arguments are
    contiguous float32 CUDA tensors (host arrays with ``host_io=True``); outputs are
    written into the given tensors.  Each call is asynchronous on the stream unless
    ``sync=True`` (the default), which waits and raises on device-side errors.
    """

    def __init__(self, grid: Grid, geom: Geometry, max_workspace_bytes: int = 0, stream=None, **options):
        self.grid, self.geom = grid, geom
        lib = load()
        self._lib = lib
        self._h = ctypes.c_void_p()
        gc = grid.c()
        gm, keep = geom.c()
        s = None
        if stream is not None:
            s = ctypes.c_void_p(int(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream))
        self.stream = stream
        rc = lib.fwime_create(ctypes.byref(self._h), ctypes.byref(gc), ctypes.byref(gm),
                              ctypes.c_size_t(max_workspace_bytes), s)
        if rc != FWIME_OK:
            raise FwimeError(rc, "fwime_create")
        for k, v in options.items():
            self.set_option(k, v)

    _OPTS = {"shots_per_batch": OPT_SHOTS_PER_BATCH, "segment": OPT_SEGMENT, "plain": OPT_PLAIN,
             "graph": OPT_GRAPH, "host_io": OPT_HOST_IO, "zchunk": OPT_ZCHUNK, "profile": OPT_PROFILE,
             "reuse_background": OPT_REUSE_BACKGROUND, "time_lag": OPT_TIME_LAG, "free_surface": OPT_FREE_SURFACE}

    def set_option(self, name, value):
        opt = self._OPTS[name] if isinstance(name, str) else int(name)
        self._check(self._lib.fwime_set_option(self._h, opt, int(value)), "fwime_set_option")

    def get_option(self, name) -> int:
        opt = {**self._OPTS, "launches": OPT_LAUNCHES, "workspace": OPT_WORKSPACE,
               "background_reused": OPT_BACKGROUND_REUSED, "batch_used": OPT_BATCH_USED}[name] \
            if isinstance(name, str) else int(name)
        v = ctypes.c_longlong(0)
        self._check(self._lib.fwime_get_option(self._h, opt, ctypes.byref(v)), "fwime_get_option")
        return int(v.value)

    @property
    def launches(self) -> int:
        """Kernels launched by the last operator call."""
        return self.get_option("launches")

    def detail(self) -> str:
        buf = ctypes.create_string_buffer(512)
        self._lib.fwime_last_error_detail(self._h, buf, 512)
        return buf.value.decode(errors="replace")

    def _check(self, rc, where):
        if rc != FWIME_OK:
            raise FwimeError(rc, where, self.detail())

    def sync(self):
        self._check(self._lib.fwime_sync(self._h), "fwime_sync")

    def profile_read(self, reset: bool = False) -> dict:
        """Per kernel family: summed CUDA-event ms, launches and algorithmic bytes (profile mode)."""
        out = {}
        for k, name in enumerate(KERNEL_NAMES):
            ms, n, b = ctypes.c_double(0), ctypes.c_longlong(0), ctypes.c_double(0)
            self._check(self._lib.fwime_profile_read(self._h, k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b),
                                                     0), "fwime_profile_read")
            out[name] = {"ms": ms.value, "launches": n.value, "bytes": b.value}
        if reset:
            self._check(self._lib.fwime_profile_read(self._h, 0, None, None, None, 1), "fwime_profile_read")
        return out

    def _done(self, rc, where, sync):
        self._check(rc, where)
        if sync:
            self.sync()

    def forward(self, v, w, d, sync=True):
        self._done(self._lib.fwime_forward(self._h, _ptr(v), _ptr(w), _ptr(d)), "fwime_forward", sync)
        return d

    def born(self, v, w, dv, d, sync=True):
        self._done(self._lib.fwime_born(self._h, _ptr(v), _ptr(w), _ptr(dv), _ptr(d)), "fwime_born", sync)
        return d

    def born_adj(self, v, w, d, dv, accumulate=False, sync=True):
        self._done(self._lib.fwime_born_adj(self._h, _ptr(v), _ptr(w), _ptr(d), _ptr(dv), int(accumulate)),
                   "fwime_born_adj", sync)
        return dv

    def born_ext(self, v, w, pt, d, sync=True):
        self._done(self._lib.fwime_born_ext(self._h, _ptr(v), _ptr(w), _ptr(pt), _ptr(d)), "fwime_born_ext", sync)
        return d

    def born_ext_adj(self, v, w, d, pt, accumulate=False, sync=True):
        self._done(self._lib.fwime_born_ext_adj(self._h, _ptr(v), _ptr(w), _ptr(d), _ptr(pt), int(accumulate)),
                   "fwime_born_ext_adj", sync)
        return pt

    def tomo(self, v, w, pt, dv, d, sync=True):
        self._done(self._lib.fwime_tomo(self._h, _ptr(v), _ptr(w), _ptr(pt), _ptr(dv), _ptr(d)), "fwime_tomo", sync)
        return d

    def tomo_adj(self, v, w, pt, d, dv, accumulate=False, sync=True):
        self._done(self._lib.fwime_tomo_adj(self._h, _ptr(v), _ptr(w), _ptr(pt), _ptr(d), _ptr(dv),
                                            int(accumulate)), "fwime_tomo_adj", sync)
        return dv

    def gradient(self, v, w, pt, dobs, grad, eps=0.0, sync=True):
        """Returns Phi (host float, valid once synced) and fills grad = B* r + T* r."""
        self._J = ctypes.c_double(0.0)
        self._done(self._lib.fwime_gradient(self._h, _ptr(v), _ptr(w), _ptr(pt), _ptr(dobs), ctypes.c_float(eps),
                                            _ptr(grad), ctypes.byref(self._J)), "fwime_gradient", sync)
        return float(self._J.value)

    def gradient_forward(self, v, w, pt, dobs, eps=0.0, sync=True):
        """Forward half of the gradient: Phi (valid once synced), with the adjoint sweep's state kept in the
        context (fwime_gradient_forward); no adjoint kernel runs."""
        self._J = ctypes.c_double(0.0)
        self._done(self._lib.fwime_gradient_forward(self._h, _ptr(v), _ptr(w), _ptr(pt), _ptr(dobs),
                                                    ctypes.c_float(eps), ctypes.byref(self._J)),
                   "fwime_gradient_forward", sync)
        return float(self._J.value)

    def gradient_backward(self, v, w, pt, dobs, grad, eps=0.0, accumulate=False, sync=True):
        """Adjoint half: grad (=, or +=) B* r + T* r from the state gradient_forward kept for the same v, w, pt
        (else the whole gradient) (fwime_gradient_backward)."""
        self._done(self._lib.fwime_gradient_backward(self._h, _ptr(v), _ptr(w), _ptr(pt), _ptr(dobs),
                                                     ctypes.c_float(eps), _ptr(grad), int(bool(accumulate))),
                   "fwime_gradient_backward", sync)
        return grad

    def vp_solve(self, v, w, dres, pt, eps=0.0, niter=10, sync=True):
        """Variable projection (Eqs. 2-5): niter CG iterations on (B~*B~ + eps^2 D*D) p~ = B~* dres, in place on
        pt.  Returns the objective Phi_eps,m at every iterate (niter + 1 values): a list when sync, else the
        ctypes array that the next sync() fills."""
        hist = (ctypes.c_double * (niter + 1))()
        self._vp_hist = hist
        self._done(self._lib.fwime_vp_solve(self._h, _ptr(v), _ptr(w), _ptr(dres), ctypes.c_float(eps), int(niter),
                                            _ptr(pt), hist), "fwime_vp_solve", sync)
        return list(hist) if sync else hist

    def spline(self, zs, xs, inp, out, adjoint=False, accumulate=False, sync=True):
        """Linear spline re-parametrisation (Eq. 1): out = S inp (model on the nodes zs x xs, metres, to the
        physical grid) or, with adjoint, out = S* inp (grid to nodes)."""
        z = np.ascontiguousarray(zs, dtype=np.float32)
        x = np.ascontiguousarray(xs, dtype=np.float32)
        P = ctypes.POINTER(ctypes.c_float)
        self._done(self._lib.fwime_spline(self._h, len(z), z.ctypes.data_as(P), len(x), x.ctypes.data_as(P),
                                          _ptr(inp), _ptr(out), int(bool(adjoint)), int(bool(accumulate))),
                   "fwime_spline", sync)
        return out

    def spline_refine(self, zc, xc, mc, zf, xf, mf, sync=True):
        """Model-space multiscale step: mf on the fine nodes zf x xf = the coarse spline of mc (nodes zc x xc)
        evaluated there (fwime_spline_refine)."""
        P = ctypes.POINTER(ctypes.c_float)
        a = [np.ascontiguousarray(n, dtype=np.float32) for n in (zc, xc, zf, xf)]
        self._done(self._lib.fwime_spline_refine(self._h, len(a[0]), a[0].ctypes.data_as(P), len(a[1]),
                                                 a[1].ctypes.data_as(P), _ptr(mc), len(a[2]), a[2].ctypes.data_as(P),
                                                 len(a[3]), a[3].ctypes.data_as(P), _ptr(mf)),
                   "fwime_spline_refine", sync)
        return mf

    def autotune(self, op: int) -> tuple[int, float]:
        """Times the stencil kernel on this operator's batch for candidate chunkings; keeps the fastest.
        Returns (rows per warp chosen, microseconds per launch)."""
        zc, us = ctypes.c_int(0), ctypes.c_float(0)
        self._check(self._lib.fwime_autotune(self._h, int(op), ctypes.byref(zc), ctypes.byref(us)), "fwime_autotune")
        return int(zc.value), float(us.value)

    def autotune_schedule(self, op: int) -> dict:
        """Times segment length x shots per launch x stencil chunking for operator `op` and keeps the fastest
        (fwime_autotune_schedule); returns the schedule and its timings."""
        r = ScheduleC()
        self._check(self._lib.fwime_autotune_schedule(self._h, int(op), ctypes.byref(r)), "fwime_autotune_schedule")
        return {k: getattr(r, k) for k, _ in ScheduleC._fields_}

    def objective(self, v, w, pt, dobs, eps=0.0, sync=True):
        """Phi = 1/2||f + B~p~ - dobs||^2 + eps^2/2||D p~||^2 alone (no adjoint sweep); valid once synced."""
        self._J = ctypes.c_double(0.0)
        self._done(self._lib.fwime_objective(self._h, _ptr(v), _ptr(w), _ptr(pt), _ptr(dobs), ctypes.c_float(eps),
                                             ctypes.byref(self._J)), "fwime_objective", sync)
        return float(self._J.value)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.fwime_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
