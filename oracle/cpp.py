"""Multi-core C restatement of the FP64 oracle (``sem_ref.c``, OpenMP).

Test infrastructure only (see the package docstring). ``SEMC`` computes what
``sem.SEM`` computes -- dense element stiffness matrices from the bilinear
geometry at the GLL points (Section 4.2, Eqs. deriv_u, numerical_integ), the
lumped mass (Eq. Abar with the mass 1/K), K u summed per node in ascending
(element, local index) order, the snapped Ricker point source (Algorithm 3)
and the leapfrog -- in plain C loops over elements and nodes, parallel over
OpenMP threads. The per-node sums run in a fixed order, so the result does
not depend on the thread count. It is pinned against ``sem.SEM`` by
``tests/test_oracle_cpp.py`` and timed as the CPU baseline by ``bench.py``.

The numbering, the GLL tables and the snapping come from the NumPy oracle
modules (``mesh``, ``gll``, ``sem.snap``); the arithmetic of the operators and
of the time loop is the C file's.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from . import gll as _gll
from . import mesh as _mesh
from . import sem as _sem

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "sem_ref.c")
LIB = os.path.join(_HERE, "_build", "liboracle_sem.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle_sem.so (gcc, OpenMP, no FMA contraction) if it is
    missing or older than its source; return its path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-Wall", SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"oracle C build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    P, D, I64 = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)
    lib.osem_create.restype = P
    lib.osem_create.argtypes = [D, I64, C.c_int64, I64, C.c_int64, C.c_int, D, D, D, D, D, C.c_int]
    lib.osem_destroy.argtypes = [P]
    lib.osem_apply_K.argtypes = [P, D, D]
    lib.osem_mass.argtypes = [P, D]
    lib.osem_run.argtypes = [P, C.c_int64, C.c_double, C.c_int64, D, I64, C.c_int32, D, D, D]
    lib.osem_max_threads.restype = C.c_int
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def max_threads() -> int:
    """OpenMP's default thread count in this process."""
    return int(_load().osem_max_threads())


class SEMC:
    """The C oracle for one mesh and model, in the original numbering.

    threads: OpenMP threads (0 = OpenMP's default, all cores the process may
    use)."""

    def __init__(self, coords, quads, p: int, vel, rho=None, threads: int = 0, validate: bool = True):
        if not 1 <= int(p) <= 8:
            raise ValueError("order must be in 1..8")
        lib = _load()
        self.coords = np.ascontiguousarray(coords, dtype=np.float64)
        self.quads = np.ascontiguousarray(quads, dtype=np.int64)
        self.p = int(p)
        if validate:
            _mesh.validate(self.coords, self.quads, self.p)
        E = self.quads.shape[0]
        self.vel = np.ascontiguousarray(np.broadcast_to(np.asarray(vel, dtype=np.float64), (E,)))
        self.rho = np.ascontiguousarray(np.ones(E) if rho is None else
                                        np.broadcast_to(np.asarray(rho, dtype=np.float64), (E,)))
        nv = self.coords.shape[0]
        conn, self.n_nodes, edges = _mesh.canonical_numbering(self.quads, nv, self.p)
        self.conn = np.ascontiguousarray(conn, dtype=np.int64)
        self.node_xy = _mesh.node_coordinates(self.coords, self.quads, self.p, conn, edges)
        x = _gll.gll_nodes(self.p)
        w = _gll.gll_weights(self.p, x)
        D = np.ascontiguousarray(_gll.derivative_matrix(x))
        self.threads = int(threads)
        self._h = lib.osem_create(_dp(self.coords), _ip(self.quads), E, _ip(self.conn), self.n_nodes, self.p + 1,
                                  _dp(np.ascontiguousarray(x)), _dp(np.ascontiguousarray(w)), _dp(D),
                                  _dp(self.vel), _dp(self.rho), self.threads)
        if not self._h:
            raise ValueError("oracle C set-up failed (allocation or non-positive Jacobian)")
        self.M = np.empty(self.n_nodes)
        lib.osem_mass(self._h, _dp(self.M))
        self._snapped = {}

    def _snap(self, x, y) -> int:
        """sem.snap, remembered per position (a search over all nodes)."""
        key = (float(x), float(y))
        if key not in self._snapped:
            self._snapped[key] = _sem.snap(self.node_xy, x, y)
        return self._snapped[key]

    def close(self):
        if getattr(self, "_h", None):
            _load().osem_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def apply_K(self, u) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty(self.n_nodes)
        _load().osem_apply_K(self._h, _dp(u), _dp(out))
        return out

    def run(self, nsteps: int, dt: float, src=None, receivers=None, u0=None, u_prev=None, step0: int = 0):
        """Leapfrog for `nsteps` steps from (u0, u_prev) (rest by default) at
        times t_k = (step0 + k) dt; same arguments and results as
        ``sem.SEM.run``: (u^n, u^{n-1}, traces[R, nsteps])."""
        u = np.zeros(self.n_nodes) if u0 is None else np.array(u0, dtype=np.float64)
        up = u.copy() if u_prev is None else np.array(u_prev, dtype=np.float64)
        s_node = -1
        f = np.zeros(max(nsteps, 1))
        if src is not None:
            sx, sy, f0, t0, amp = src
            s_node = self._snap(sx, sy)
            f = np.ascontiguousarray(_sem.ricker((step0 + np.arange(max(nsteps, 1))) * dt, f0, t0, amp),
                                     dtype=np.float64)
        rec = np.zeros(0, dtype=np.int64)
        if receivers is not None and len(receivers):
            rec = np.array([self._snap(x, y) for x, y in np.asarray(receivers)], dtype=np.int64)
        traces = np.zeros((rec.size, max(nsteps, 1)))
        _load().osem_run(self._h, int(nsteps), float(dt), int(s_node), _dp(f), _ip(rec), int(rec.size), _dp(u),
                         _dp(up), _dp(traces))
        return u, up, traces[:, :nsteps]
