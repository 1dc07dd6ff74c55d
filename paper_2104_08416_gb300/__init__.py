"""Python binding of the GB300 spectral-element wave stepper (libsem.so).

Argument marshalling only: every step of the time loop runs in the CUDA
kernels behind the C ABI declared in include/sem.h, and the functions here
carry the same names as the C calls. PyTorch provides the device memory
(through its caching allocator, installed with ``sem_set_allocator``) and the
CUDA stream the library enqueues on.

The library is built in-tree (``paper_2104_08416_gb300/libsem.so``) by
``paper_2104_08416_gb300.build.build()``. If it is missing, ``load()`` raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsem.so")

SEM_OK, SEM_ERR_INVALID_ARG, SEM_ERR_STATE, SEM_ERR_CUDA, SEM_ERR_OOM, SEM_ERR_TIMEOUT, SEM_ERR_UNSUPPORTED = range(7)
SEM_FP64, SEM_FP32_KAHAN, SEM_FP32 = 0, 1, 2
SEM_ORDER_NONE, SEM_ORDER_ROWMAJOR, SEM_ORDER_RANDOM, SEM_ORDER_HILBERT = 0, 1, 2, 3
SEM_ORDER_CONNECTIVITY, SEM_ORDER_DISTANCE, SEM_ORDER_HILBERT_WIDE = 4, 5, 6
SEM_SRC_RICKER = 0
SEM_SCHEME_LEAPFROG, SEM_SCHEME_HEUN = 0, 1
SCHEMES = {"leapfrog": SEM_SCHEME_LEAPFROG, "heun": SEM_SCHEME_HEUN}
SEM_METRIC_BILINEAR, SEM_METRIC_STORED = 0, 1
METRICS = {"bilinear": SEM_METRIC_BILINEAR, "stored": SEM_METRIC_STORED}
PRECISIONS = {"fp64": SEM_FP64, "fp32_kahan": SEM_FP32_KAHAN, "fp32": SEM_FP32}
ORDERINGS = {"none": SEM_ORDER_NONE, "rowmajor": SEM_ORDER_ROWMAJOR, "random": SEM_ORDER_RANDOM,
             "hilbert": SEM_ORDER_HILBERT, "connectivity": SEM_ORDER_CONNECTIVITY, "distance": SEM_ORDER_DISTANCE,
             "hilbert_wide": SEM_ORDER_HILBERT_WIDE}
DEFAULT_SEED = 2104084160

# every symbol include/sem.h declares
EXPORTS = (
    "sem_set_allocator", "sem_mesh_create", "sem_reorder", "sem_set_model", "sem_set_source",
    "sem_set_receivers", "sem_cfl_dt", "sem_set_scheme", "sem_set_metric", "sem_read_metric", "sem_set_dt", "sem_step", "sem_get_step", "sem_read_traces",
    "sem_read_wavefield", "sem_set_state", "sem_get_state", "sem_apply_stiffness", "sem_read_mass",
    "sem_get_permutation", "sem_get_sizes", "sem_node_coordinates", "sem_get_snapped",
    "sem_compute_ordering", "sem_count_nodes", "sem_hilbert_cells", "sem_plan_check", "sem_launch_info", "sem_set_stream", "sem_set_stream_tiling",
    "sem_stream_order", "sem_stream_schedule", "sem_stream_withhold",
    "sem_set_tuning",
    "sem_profile_enable", "sem_profile_read", "sem_traffic_model", "sem_transfer_bytes",
    "sem_apply_stiffness_dev_noalloc", "sem_misfit_gradient", "sem_batch_create", "sem_batch_step", "sem_batch_info",
    "sem_batch_set_stream", "sem_batch_mode", "sem_batch_last_error", "sem_batch_destroy", "sem_last_error", "sem_destroy",
)

_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_I32 = C.POINTER(C.c_int32)
_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class SemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"sem status {status}: {msg}")
        self.status = status


def load(path: str | None = None):
    """Load libsem.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"{path} not found: run paper_2104_08416_gb300.build.build() first")
    lib = C.CDLL(path)
    sig = {
        "sem_set_allocator": (_ALLOC, _FREE, _P),
        "sem_mesh_create": (_D, C.c_int64, _I32, C.c_int64, C.c_int, C.c_int, _P, C.POINTER(_P)),
        "sem_reorder": (_P, C.c_int, C.c_uint64),
        "sem_set_model": (_P, _D, _D),
        "sem_set_source": (_P, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double),
        "sem_set_receivers": (_P, _D, C.c_int32, C.c_int64),
        "sem_cfl_dt": (_P, _D),
        "sem_set_dt": (_P, C.c_double),
        "sem_set_scheme": (_P, C.c_int),
        "sem_set_metric": (_P, C.c_int),
        "sem_read_metric": (_P, _D),
        "sem_step": (_P, C.c_int64),
        "sem_get_step": (_P, _I64),
        "sem_read_traces": (_P, _D, C.c_int64),
        "sem_read_wavefield": (_P, _D),
        "sem_set_state": (_P, _D, _D, C.c_int64),
        "sem_get_state": (_P, _D, _D, _I64),
        "sem_apply_stiffness": (_P, _D, _D),
        "sem_read_mass": (_P, _D),
        "sem_get_permutation": (_P, _I64, _I64),
        "sem_get_sizes": (_P, _I64, _I64),
        "sem_node_coordinates": (_P, _D),
        "sem_get_snapped": (_P, _I64, _I64),
        "sem_compute_ordering": (_D, C.c_int64, _I32, C.c_int64, C.c_int, C.c_int, C.c_uint64, _I64, _I64),
        "sem_count_nodes": (_I32, C.c_int64, C.c_int64, C.c_int, _I64),
        "sem_hilbert_cells": (C.c_int32, C.c_int32, _I32),
        "sem_plan_check": (_D, C.c_int64, _I32, C.c_int64, C.c_int, C.c_int, C.c_uint64, C.c_int, C.c_int, _D,
                           C.c_int32, _I64, C.c_char_p, C.c_size_t),
        "sem_launch_info": (_P, _I64, _I64),
        "sem_set_stream": (_P, C.c_int),
        "sem_set_stream_tiling": (_P, C.c_int, C.c_int),
        "sem_stream_order": (_P, _I32, _I32),
        "sem_stream_schedule": (_I32, _I32, C.c_int32, C.c_int, C.c_int, C.POINTER(C.c_uint32), _I32),
        "sem_stream_withhold": (_P, C.c_int64, C.c_int32),
        "sem_set_tuning": (_P, C.c_int, C.c_int),
        "sem_profile_enable": (_P, C.c_int),
        "sem_profile_read": (_P, _D, _I64, _D, _I64),
        "sem_traffic_model": (_P, _D, _D),
        "sem_transfer_bytes": (_P, _I64, _I64),
        "sem_apply_stiffness_dev_noalloc": (_P, _P, _P),
        "sem_misfit_gradient": (_P, _D, C.c_int64, C.c_int64, _D, _D),
        "sem_batch_create": (C.POINTER(_P), C.c_int32, C.c_int32, C.POINTER(_P)),
        "sem_batch_step": (_P, C.c_int64),
        "sem_batch_info": (_P, _I32, _I32, _I32, _I32),
        "sem_batch_mode": (_P, _I32, _I32),
        "sem_batch_set_stream": (_P, C.c_int),
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = list(args)
        f.restype = C.c_int
    lib.sem_last_error.argtypes = [_P]
    lib.sem_last_error.restype = C.c_char_p
    lib.sem_destroy.argtypes = [_P]
    lib.sem_destroy.restype = None
    lib.sem_batch_last_error.argtypes = [_P]
    lib.sem_batch_last_error.restype = C.c_char_p
    lib.sem_batch_destroy.argtypes = [_P]
    lib.sem_batch_destroy.restype = None
    _lib = lib
    return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _check(st: int, handle=None):
    if st != SEM_OK:
        msg = ""
        if handle is not None and _lib is not None:
            msg = (_lib.sem_last_error(handle) or b"").decode()
        raise SemError(st, msg)


# ---------------------------------------------------------------- allocator
_torch_alloc_refs = None


def sem_set_allocator_torch():
    """Route the library's device allocations through torch's caching allocator."""
    global _torch_alloc_refs
    import torch

    lib = load()

    def _alloc(nbytes, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                          stream if stream else 0))
        except Exception:  # out of memory -> NULL, the library reports SEM_ERR_OOM
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _ALLOC(_alloc), _FREE(_free)
    _check(lib.sem_set_allocator(a, f, None))
    _torch_alloc_refs = (a, f)


def sem_set_allocator_default():
    global _torch_alloc_refs
    lib = load()
    _check(lib.sem_set_allocator(_ALLOC(), _FREE(), None))
    _torch_alloc_refs = None


# ------------------------------------------------------------- host-only calls
def sem_count_nodes(quads, nv: int, order: int) -> int:
    lib = load()
    q = np.ascontiguousarray(quads, dtype=np.int32)
    n = C.c_int64()
    _check(lib.sem_count_nodes(_ptr(q, C.c_int32), int(nv), q.shape[0], int(order), C.byref(n)))
    return n.value


def sem_compute_ordering(coords, quads, order: int, kind, seed: int = DEFAULT_SEED):
    """(elem_order, node_order) with order[new] = old id; no device needed."""
    lib = load()
    kind = ORDERINGS[kind] if isinstance(kind, str) else int(kind)
    c = np.ascontiguousarray(coords, dtype=np.float64)
    q = np.ascontiguousarray(quads, dtype=np.int32)
    nn = sem_count_nodes(q, c.shape[0], order)
    eo = np.zeros(q.shape[0], dtype=np.int64)
    no = np.zeros(nn, dtype=np.int64)
    _check(lib.sem_compute_ordering(_ptr(c, C.c_double), c.shape[0], _ptr(q, C.c_int32), q.shape[0], int(order),
                                    kind, C.c_uint64(seed & (2 ** 64 - 1)), _ptr(eo, C.c_int64),
                                    _ptr(no, C.c_int64)))
    return eo, no


def sem_hilbert_cells(W: int, H: int) -> np.ndarray:
    lib = load()
    out = np.zeros((W * H, 2), dtype=np.int32)
    _check(lib.sem_hilbert_cells(int(W), int(H), _ptr(out, C.c_int32)))
    return out


def sem_stream_schedule(dep_ptr, dep, band_steps: int, window_levels: int):
    """Host-only wavefront order of a block graph (see sem.h): returns
    (sched uint32[band_steps * nblocks], levels int32[nblocks])."""
    lib = load()
    dp = np.ascontiguousarray(dep_ptr, dtype=np.int32)
    dd = np.ascontiguousarray(dep, dtype=np.int32)
    nb = dp.shape[0] - 1
    sched = np.zeros(max(0, band_steps * nb), dtype=np.uint32)
    lev = np.zeros(max(0, nb), dtype=np.int32)
    _check(lib.sem_stream_schedule(_ptr(dp, C.c_int32), _ptr(dd, C.c_int32), nb, int(band_steps),
                                   int(window_levels), _ptr(sched, C.c_uint32), _ptr(lev, C.c_int32)))
    return sched, lev


def sem_plan_check(coords, quads, order: int, kind, eb: int, fp64: bool = False, receivers=None,
                   seed: int = DEFAULT_SEED):
    """Host-only replay of the step kernel's block plan (see sem.h).
    Returns (status, info dict, message)."""
    lib = load()
    kind = ORDERINGS[kind] if isinstance(kind, str) else int(kind)
    c = np.ascontiguousarray(coords, dtype=np.float64)
    q = np.ascontiguousarray(quads, dtype=np.int32)
    rec = np.ascontiguousarray(np.zeros((0, 2)) if receivers is None else receivers, dtype=np.float64)
    info = np.zeros(7, dtype=np.int64)
    msg = C.create_string_buffer(512)
    st = lib.sem_plan_check(_ptr(c, C.c_double), c.shape[0], _ptr(q, C.c_int32), q.shape[0], int(order), kind,
                            C.c_uint64(seed & (2 ** 64 - 1)), int(eb), int(bool(fp64)), _ptr(rec, C.c_double),
                            rec.shape[0], _ptr(info, C.c_int64), msg, 512)
    keys = ("nblocks", "dense", "open_nodes", "max_entries", "max_packet", "npartial", "max_colors")
    return st, dict(zip(keys, (int(v) for v in info))), msg.value.decode()


# ------------------------------------------------------------------ handle
class SEM:
    """One mesh handle (sem_mesh*). Methods mirror the C calls."""

    def __init__(self, coords, quads, order: int, precision="fp32_kahan", stream=None):
        lib = load()
        self._lib = lib
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        c = np.ascontiguousarray(coords, dtype=np.float64)
        q = np.ascontiguousarray(quads, dtype=np.int32)
        h = _P()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
        st = lib.sem_mesh_create(_ptr(c, C.c_double), c.shape[0], _ptr(q, C.c_int32), q.shape[0], int(order),
                                 prec, _P(stream or None), C.byref(h))
        _check(st)
        self.h = h
        self.order = order
        self.precision = prec
        nn, ne = C.c_int64(), C.c_int64()
        _check(lib.sem_get_sizes(h, C.byref(nn), C.byref(ne)), h)
        self.n_nodes, self.n_elems = nn.value, ne.value
        self.nrec = 0
        self.max_steps = 0

    def _c(self, st):
        _check(st, self.h)

    def sem_reorder(self, kind, seed: int = DEFAULT_SEED):
        kind = ORDERINGS[kind] if isinstance(kind, str) else int(kind)
        self._c(self._lib.sem_reorder(self.h, kind, C.c_uint64(seed & (2 ** 64 - 1))))

    def sem_set_model(self, vel, rho=None):
        v = np.ascontiguousarray(np.broadcast_to(np.asarray(vel, dtype=np.float64), (self.n_elems,)))
        r = None if rho is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(rho, dtype=np.float64), (self.n_elems,)))
        self._c(self._lib.sem_set_model(self.h, _ptr(v, C.c_double), None if r is None else _ptr(r, C.c_double)))

    def sem_set_source(self, f0, t0, amp, x, y, kind=SEM_SRC_RICKER):
        self._c(self._lib.sem_set_source(self.h, kind, f0, t0, amp, x, y))

    def sem_set_receivers(self, xy, max_steps: int):
        a = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        self._c(self._lib.sem_set_receivers(self.h, _ptr(a, C.c_double), a.shape[0], int(max_steps)))
        self.nrec = a.shape[0]
        self.max_steps = int(max_steps)

    def sem_cfl_dt(self) -> float:
        d = C.c_double()
        self._c(self._lib.sem_cfl_dt(self.h, C.byref(d)))
        return d.value

    def sem_set_scheme(self, scheme):
        scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
        self._c(self._lib.sem_set_scheme(self.h, scheme))

    def sem_set_metric(self, metric):
        """'bilinear' (FP32 metric formed per point from the bilinear map) or
        'stored' (FP64-computed metric rounded once to FP32 and streamed)."""
        metric = METRICS[metric] if isinstance(metric, str) else int(metric)
        self._c(self._lib.sem_set_metric(self.h, metric))

    def sem_read_metric(self) -> np.ndarray:
        """(E, P, 3) array of (gxx, gxy, gyy) per element (original order) and
        GLL point, as the step kernels use them."""
        out = np.zeros((self.n_elems, (self.order + 1) ** 2, 3))
        self._c(self._lib.sem_read_metric(self.h, _ptr(out, C.c_double)))
        return out

    def sem_set_dt(self, dt: float):
        self._c(self._lib.sem_set_dt(self.h, float(dt)))

    def sem_set_tuning(self, elems_per_block: int, threads_per_block: int = 0):
        self._c(self._lib.sem_set_tuning(self.h, int(elems_per_block), int(threads_per_block)))

    def sem_step(self, nsteps: int):
        self._c(self._lib.sem_step(self.h, int(nsteps)))

    def sem_get_step(self) -> int:
        s = C.c_int64()
        self._c(self._lib.sem_get_step(self.h, C.byref(s)))
        return s.value

    def sem_read_traces(self, cap: int | None = None) -> np.ndarray:
        cap = self.max_steps if cap is None else cap
        out = np.zeros((self.nrec, cap), dtype=np.float64)
        self._c(self._lib.sem_read_traces(self.h, _ptr(out, C.c_double), int(cap)))
        return out

    def sem_read_wavefield(self) -> np.ndarray:
        u = np.zeros(self.n_nodes, dtype=np.float64)
        self._c(self._lib.sem_read_wavefield(self.h, _ptr(u, C.c_double)))
        return u

    def sem_set_state(self, u, u_prev, step: int = 0):
        a = np.ascontiguousarray(u, dtype=np.float64)
        b = np.ascontiguousarray(u_prev, dtype=np.float64)
        self._c(self._lib.sem_set_state(self.h, _ptr(a, C.c_double), _ptr(b, C.c_double), int(step)))

    def sem_get_state(self):
        a = np.zeros(self.n_nodes)
        b = np.zeros(self.n_nodes)
        s = C.c_int64()
        self._c(self._lib.sem_get_state(self.h, _ptr(a, C.c_double), _ptr(b, C.c_double), C.byref(s)))
        return a, b, s.value

    def sem_apply_stiffness(self, u) -> np.ndarray:
        a = np.ascontiguousarray(u, dtype=np.float64)
        out = np.zeros(self.n_nodes)
        self._c(self._lib.sem_apply_stiffness(self.h, _ptr(a, C.c_double), _ptr(out, C.c_double)))
        return out

    def sem_read_mass(self) -> np.ndarray:
        out = np.zeros(self.n_nodes)
        self._c(self._lib.sem_read_mass(self.h, _ptr(out, C.c_double)))
        return out

    def sem_get_permutation(self):
        e = np.zeros(self.n_elems, dtype=np.int64)
        n = np.zeros(self.n_nodes, dtype=np.int64)
        self._c(self._lib.sem_get_permutation(self.h, _ptr(e, C.c_int64), _ptr(n, C.c_int64)))
        return e, n

    def sem_node_coordinates(self) -> np.ndarray:
        out = np.zeros((self.n_nodes, 2))
        self._c(self._lib.sem_node_coordinates(self.h, _ptr(out, C.c_double)))
        return out

    def sem_get_snapped(self):
        s = C.c_int64()
        r = np.zeros(max(self.nrec, 1), dtype=np.int64)
        self._c(self._lib.sem_get_snapped(self.h, C.byref(s), _ptr(r, C.c_int64)))
        return s.value, r[: self.nrec]

    def sem_launch_info(self):
        a, b = C.c_int64(), C.c_int64()
        self._c(self._lib.sem_launch_info(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def sem_set_stream(self, steps_per_launch: int):
        self._c(self._lib.sem_set_stream(self.h, int(steps_per_launch)))

    def sem_set_stream_tiling(self, band_steps: int, window_levels: int = 0):
        self._c(self._lib.sem_set_stream_tiling(self.h, int(band_steps), int(window_levels)))

    def sem_stream_order(self):
        """(band_steps, window_levels) of the wavefront order last uploaded."""
        t, w = C.c_int32(), C.c_int32()
        self._c(self._lib.sem_stream_order(self.h, C.byref(t), C.byref(w)))
        return t.value, w.value

    def sem_stream_withhold(self, step: int, block: int):
        self._c(self._lib.sem_stream_withhold(self.h, int(step), int(block)))

    def sem_profile_enable(self, enable: bool = True):
        self._c(self._lib.sem_profile_enable(self.h, 1 if enable else 0))

    def sem_profile_read(self):
        """(block_ms, block_launches, open_ms, open_launches) since the last read."""
        bm, om = C.c_double(), C.c_double()
        bl, ol = C.c_int64(), C.c_int64()
        self._c(self._lib.sem_profile_read(self.h, C.byref(bm), C.byref(bl), C.byref(om), C.byref(ol)))
        return bm.value, bl.value, om.value, ol.value

    def sem_traffic_model(self):
        a, b = C.c_double(), C.c_double()
        self._c(self._lib.sem_traffic_model(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def sem_transfer_bytes(self):
        a, b = C.c_int64(), C.c_int64()
        self._c(self._lib.sem_transfer_bytes(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def sem_apply_stiffness_dev_noalloc(self, dev_u_ptr: int, dev_Ku_ptr: int):
        """K u on device arrays (storage order, handle's storage type) without
        any allocation; enqueued on the handle's stream, not synchronised."""
        self._c(self._lib.sem_apply_stiffness_dev_noalloc(self.h, _P(dev_u_ptr), _P(dev_Ku_ptr)))

    def sem_misfit_gradient(self, d_obs, nsteps: int, checkpoint_every: int = 0, gradient: bool = True):
        """(J, dJ/dvel) of a run from rest against observed traces
        d_obs[nrec][nsteps]; the gradient is None when gradient=False."""
        obs = np.ascontiguousarray(d_obs, dtype=np.float64)
        J = C.c_double()
        g = np.zeros(self.n_elems, dtype=np.float64) if gradient else None
        self._c(self._lib.sem_misfit_gradient(self.h, _ptr(obs, C.c_double), int(nsteps), int(checkpoint_every),
                                              C.byref(J), _ptr(g, C.c_double) if gradient else None))
        return J.value, g

    def sem_destroy(self):
        if getattr(self, "h", None):
            self._lib.sem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.sem_destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.sem_destroy()


def sem_mesh_create(coords, quads, order: int, precision="fp32_kahan", stream=None) -> SEM:
    return SEM(coords, quads, order, precision, stream)


class SEMBatch:
    """Batched shots (sem_batch*): advances several configured SEM handles
    together. Methods mirror the C calls; the handles stay readable through
    their own methods."""

    def __init__(self, shots, autotune_steps: int = 0):
        self._lib = load()
        self.shots = list(shots)
        arr = (_P * len(self.shots))(*[s.h for s in self.shots])
        out = _P()
        st = self._lib.sem_batch_create(arr, len(self.shots), int(autotune_steps), C.byref(out))
        _check(st)
        self.h = out

    def _c(self, st):
        if st != SEM_OK:
            raise SemError(st, (self._lib.sem_batch_last_error(self.h) or b"").decode())

    def sem_batch_step(self, nsteps: int):
        self._c(self._lib.sem_batch_step(self.h, int(nsteps)))

    def sem_batch_set_stream(self, mode: int):
        """-1 automatic (default), 1 stream every order class, 2 none but in
        clock-driven 64-step blocks, 0 none (one launch per class and step)."""
        self._c(self._lib.sem_batch_set_stream(self.h, int(mode)))

    def sem_batch_mode(self):
        st, spl = C.c_int32(), C.c_int32()
        self._c(self._lib.sem_batch_mode(self.h, C.byref(st), C.byref(spl)))
        return {"streamed_classes": st.value, "steps_per_launch": spl.value}

    def sem_batch_info(self):
        n = C.c_int32()
        self._c(self._lib.sem_batch_info(self.h, C.byref(n), None, None, None))
        orders = np.zeros(n.value, dtype=np.int32)
        eb = np.zeros(n.value, dtype=np.int32)
        ctas = np.zeros(n.value, dtype=np.int32)
        self._c(self._lib.sem_batch_info(self.h, C.byref(n), _ptr(orders, C.c_int32), _ptr(eb, C.c_int32),
                                         _ptr(ctas, C.c_int32)))
        return {"orders": orders.tolist(), "elems_per_block": eb.tolist(), "ctas": ctas.tolist()}

    def sem_batch_destroy(self):
        if self.h:
            self._lib.sem_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.sem_batch_destroy()
        except Exception:
            pass

