"""FP64 spectral-element discretisation of the 2D acoustic wave equation.

Test infrastructure only (see the package docstring).

Physics (Section 4.1, Eqs. def_v_1, def_u_1 with initial condition
initial_cond): (1/K) u_t = div v + f and v_t = grad(u) / rho. Eliminating v
gives the scalar second-order form (1/K) u_tt = div((1/rho) grad u) + f', with
K = rho c^2 and natural (Neumann) boundaries from the weak form (Eq.
def_weak_u).

Discretisation (Section 4.2): nodal basis on GLL points that double as
quadrature points, so the mass is diagonal (Eq. Abar with A = M = 1/K):
    M_nu = sum_{e, q : mu(q, e) = nu} w_q |J_q| / (rho_e c_e^2),
and the stiffness that replaces R_nu of Eq. u_change_r_effic is assembled from
dense element matrices
    K_e[a, b] = sum_q w_q |J_q| / rho_e  grad(phi_a) . grad(phi_b)  at x_q,
with grad(phi) = J^-T grad_ref(phi) (Eq. deriv_u, K^(e) = J^-1).

The point source enters like Algorithm 3: the Ricker wavelet value at t_n is
added at the global node nearest to the source position and scaled by the
inverse mass (Eq. u_change with y_nu). Time stepping is the explicit leapfrog
(central difference) for M u_tt = f e_s - K u:
    u^{n+1} = 2 u^n - u^{n-1} + dt^2 M^-1 (f(t_n) e_s - K u^n),  t_n = n dt,
starting from u^0 = u^{-1} = 0 (Eq. initial_cond). Nodal sums run in the
original (element id, local index) order, so results do not depend on any
memory ordering.
"""
from __future__ import annotations

import math

import numpy as np

from . import gll as _gll
from . import mesh as _mesh


def reference_gradient(p: int):
    """B[q, d, a]: d-th reference derivative of basis function a at GLL point q."""
    x = _gll.gll_nodes(p)
    D = _gll.derivative_matrix(x)
    n = p + 1
    P = n * n
    B = np.zeros((P, 2, P))
    for qj in range(n):
        for qi in range(n):
            q = qj * n + qi
            for aj in range(n):
                for ai in range(n):
                    a = aj * n + ai
                    if aj == qj:
                        B[q, 0, a] = D[qi, ai]      # d/dxi of l_ai(xi) l_aj(eta)
                    if ai == qi:
                        B[q, 1, a] = D[qj, aj]      # d/deta
    return B


def ricker(t, f0: float, t0: float, amp: float = 1.0):
    """Ricker wavelet amp (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2)."""
    a = (math.pi * f0 * (np.asarray(t, dtype=np.float64) - t0)) ** 2
    return amp * (1.0 - 2.0 * a) * np.exp(-a)


def snap(node_xy: np.ndarray, x: float, y: float) -> int:
    """Nearest global node by squared Euclidean distance dx*dx + dy*dy; ties go
    to the lowest (original) node id (Algorithm 3: "global node that x^(s)
    maps to")."""
    dx = node_xy[:, 0] - x
    dy = node_xy[:, 1] - y
    return int(np.argmin(dx * dx + dy * dy))


def cfl_dt(coords, quads, p: int, vel) -> float:
    """dt_CFL = min over elements of (shortest distance between GLL points
    adjacent along a local grid line) / c_e. Section 6.2 only says the step
    meets the CFL condition; this is the reading used throughout."""
    coords = np.asarray(coords, dtype=np.float64)
    quads = np.asarray(quads, dtype=np.int64)
    vel = np.broadcast_to(np.asarray(vel, dtype=np.float64), (quads.shape[0],))
    n = p + 1
    s = _gll.gll_nodes(p)
    corners = coords[quads]
    pts = np.zeros((quads.shape[0], n, n, 2))      # [e, j, i]
    for j in range(n):
        for i in range(n):
            pts[:, j, i] = _mesh.bilinear(corners, s[i], s[j])
    d1 = np.linalg.norm(pts[:, :, 1:] - pts[:, :, :-1], axis=-1).min(axis=(1, 2))
    d2 = np.linalg.norm(pts[:, 1:, :] - pts[:, :-1, :], axis=-1).min(axis=(1, 2))
    return float(np.min(np.minimum(d1, d2) / vel))


class SEM:
    """Discrete operators of one mesh + model, in the original numbering."""

    def __init__(self, coords, quads, p: int, vel, rho=None, validate=True):
        self.coords = np.asarray(coords, dtype=np.float64)
        self.quads = np.asarray(quads, dtype=np.int64)
        self.p = int(p)
        if validate:
            _mesh.validate(self.coords, self.quads, self.p)
        E = self.quads.shape[0]
        self.vel = np.broadcast_to(np.asarray(vel, dtype=np.float64), (E,)).copy()
        self.rho = (np.ones(E) if rho is None else
                    np.broadcast_to(np.asarray(rho, dtype=np.float64), (E,)).copy())
        nv = self.coords.shape[0]
        self.conn, self.n_nodes, self.edges = _mesh.canonical_numbering(self.quads, nv, self.p)
        self.node_xy = _mesh.node_coordinates(self.coords, self.quads, self.p, self.conn, self.edges)
        n = self.p + 1
        x = _gll.gll_nodes(self.p)
        w = _gll.gll_weights(self.p, x)
        self.w2 = np.outer(w, w).ravel()                   # w_q = w_i w_j at q = j*n+i
        J = _mesh.jacobians(self.coords, self.quads, self.p)
        self.detJ = J[..., 0, 0] * J[..., 1, 1] - J[..., 0, 1] * J[..., 1, 0]
        Jinv = np.linalg.inv(J)                             # K^(e) at each point
        self.Jinv = Jinv
        metric = Jinv @ np.swapaxes(Jinv, -1, -2)           # J^-1 J^-T
        self.G = (self.w2[None, :] * self.detJ / self.rho[:, None])[..., None, None] * metric
        B = reference_gradient(self.p)
        self.B = B
        self._Ke = None
        # lumped mass, summed per node in (element, local index) order
        mloc = self.w2[None, :] * self.detJ / (self.rho * self.vel ** 2)[:, None]
        self.M = np.bincount(self.conn.ravel(), weights=mloc.ravel(), minlength=self.n_nodes)

    @property
    def Ke(self):
        """Dense element stiffness matrices K_e[E, P, P]."""
        if self._Ke is None:
            # K_e[a, b] = sum_q B[q,:,a]^T G[e,q] B[q,:,b]
            self._Ke = np.einsum("qda,eqdk,qkb->eab", self.B, self.G, self.B, optimize=True)
        return self._Ke

    def apply_K(self, u: np.ndarray) -> np.ndarray:
        """(K u)_nu assembled in (element id, local index) order."""
        ue = u[self.conn]                                   # gather U_mu(q,e)
        re = np.einsum("eab,eb->ea", self.Ke, ue)
        return np.bincount(self.conn.ravel(), weights=re.ravel(), minlength=self.n_nodes)

    def apply_K_at(self, u: np.ndarray, nodes) -> np.ndarray:
        """(K u) at selected nodes only, from the elements that touch them
        (same per-node order as `apply_K`); for sampled checks on large meshes."""
        nodes = np.asarray(nodes, dtype=np.int64)
        out = np.zeros(nodes.size)
        for k, nu in enumerate(nodes):
            es, ls = np.nonzero(self.conn == nu) if self.conn.size < 5_000_000 else _find(self.conn, nu)
            acc = 0.0
            for e, a in zip(es, ls):
                Ke = np.einsum("qd,qdk,qkb->b", self.B[:, :, a], self.G[e], self.B)
                acc += float(Ke @ u[self.conn[e]])
            out[k] = acc
        return out

    def cfl_dt(self) -> float:
        """dt_CFL of this mesh and model (see the module function cfl_dt)."""
        return cfl_dt(self.coords, self.quads, self.p, self.vel)

    def lambda_max(self, iters: int = 300, seed: int = 7) -> float:
        """Largest eigenvalue of M^-1 K by power iteration (symmetrised form)."""
        rng = np.random.default_rng(seed)
        v = rng.standard_normal(self.n_nodes)
        sq = np.sqrt(self.M)
        lam = 0.0
        for _ in range(iters):
            w = self.apply_K(v / sq) / sq
            lam = float(v @ w / (v @ v))
            v = w / np.linalg.norm(w)
        return lam

    def energy(self, u_next, u_cur, dt) -> float:
        """E^{n+1/2} = 1/2 d^T M d / dt^2 + 1/2 u^{n+1 T} K u^n, d = u^{n+1} - u^n;
        constant under unforced leapfrog."""
        d = u_next - u_cur
        return 0.5 * float(d @ (self.M * d)) / dt ** 2 + 0.5 * float(u_next @ self.apply_K(u_cur))

    def run(self, nsteps: int, dt: float, src=None, receivers=None, u0=None, u_prev=None,
            callback=None):
        """Leapfrog for `nsteps` steps.

        src: (x, y, f0, t0, amp) or None. receivers: (R, 2) positions or None.
        Returns (u^{nsteps}, u^{nsteps-1}, traces[R, nsteps]) where
        traces[r, n-1] = u^n at the receiver's node, n = 1..nsteps.
        """
        u = np.zeros(self.n_nodes) if u0 is None else np.array(u0, dtype=np.float64)
        up = u.copy() if u_prev is None else np.array(u_prev, dtype=np.float64)
        s_node = None
        if src is not None:
            sx, sy, f0, t0, amp = src
            s_node = snap(self.node_xy, sx, sy)
        rec_nodes = np.zeros(0, dtype=np.int64)
        if receivers is not None and len(receivers):
            rec_nodes = np.array([snap(self.node_xy, x, y) for x, y in np.asarray(receivers)],
                                 dtype=np.int64)
        traces = np.zeros((rec_nodes.size, nsteps))
        minv = 1.0 / self.M
        for n in range(nsteps):
            rhs = -self.apply_K(u)
            if s_node is not None:
                rhs[s_node] += float(ricker(n * dt, f0, t0, amp))
            un = 2.0 * u - up + dt * dt * (minv * rhs)
            up, u = u, un
            traces[:, n] = u[rec_nodes]
            if callback is not None:
                callback(n + 1, u, up)
        return u, up, traces

    def misfit_gradient(self, nsteps: int, dt: float, src, receivers, d_obs):
        """L2 trace misfit of a run from rest and its gradient with respect to
        the per-element wave speeds, by the discrete adjoint of the leapfrog.

        The run is the one of `run` (u^0 = u^-1 = 0); with traces d_r^n = u^{n+1}
        at receiver r, J = 1/2 sum_r sum_n (d_r^n - d_obs[r, n])^2 dt. Write step
        n as R^n = M (u^{n+1} - 2 u^n + u^{n-1}) + dt^2 K u^n - dt^2 f_n e_s = 0
        and J's Lagrangian as J + sum_n lambda^{n+1} . R^n. Stationarity in
        u^m (m = 1..N) gives, with lambda^{N+1} = lambda^{N+2} = 0,
            lambda^m = 2 lambda^{m+1} - lambda^{m+2} - dt^2 M^-1 K lambda^{m+1}
                       - M^-1 g^m,   g^m = dt sum_r (u^m_r - d_obs[r, m-1]) e_r,
        and, since the speed c_e enters only the lumped mass (M = 1/K with
        K = rho c^2, Section 4.1), dJ/dc_e = sum_nu dM_nu/dc_e C_nu with
        C_nu = sum_{m=1..N} lambda^m_nu (u^m - 2 u^{m-1} + u^{m-2})_nu and
        dM_nu/dc_e = -2 sum_{q in e, mu(q,e) = nu} w_q |J_q| / (rho_e c_e^3).
        Returns (J, grad[E], traces[R, N]). Keeps every state: small meshes only.
        """
        d_obs = np.asarray(d_obs, dtype=np.float64)
        states = [np.zeros(self.n_nodes), np.zeros(self.n_nodes)]        # u^-1, u^0

        def keep(n, u, up):
            states.append(u.copy())

        _, _, traces = self.run(nsteps, dt, src=src, receivers=receivers, callback=keep)
        J = 0.5 * dt * float(np.sum((traces - d_obs) ** 2))
        rec_nodes = np.array([snap(self.node_xy, x, y) for x, y in np.asarray(receivers)], dtype=np.int64)
        minv = 1.0 / self.M
        lam1 = np.zeros(self.n_nodes)      # lambda^{m+1}
        lam2 = np.zeros(self.n_nodes)      # lambda^{m+2}
        C = np.zeros(self.n_nodes)
        for m in range(nsteps, 0, -1):
            g = np.zeros(self.n_nodes)
            np.add.at(g, rec_nodes, dt * (traces[:, m - 1] - d_obs[:, m - 1]))
            lam = 2.0 * lam1 - lam2 - dt * dt * (minv * self.apply_K(lam1)) - minv * g
            # states[k] = u^{k-1}
            a = states[m + 1] - 2.0 * states[m] + states[m - 1]
            C += lam * a
            lam2, lam1 = lam1, lam
        dM = -2.0 * self.w2[None, :] * self.detJ / (self.rho * self.vel ** 3)[:, None]   # [E, P]
        grad = np.sum(dM * C[self.conn], axis=1)
        return J, grad, traces

    # ---------------------------------------------------------- first-order form
    def first_order_rhs(self, U, V, y_node=None, y=0.0):
        """Rates of the paper's first-order system (Section 4.1 with M = 1/K,
        B_kk = -1, F_kk = 1/rho, D = E = 0), discretised as in Section 4.2:
        V (E, P, 2) holds the discontinuous velocity at every element's local
        nodes (physical x, y components), U the continuous pressure.
            dV/dt at local node q of e   = (1/rho_e) grad u (x_q)   (Eq. v_change)
            dU/dt at global node nu      = (R_nu + y_nu) / M_nu       (Eq. u_change)
            R_nu = - sum_{e, q; p: mu(p,e) = nu} w_q |J_q| V_q . grad phi_p (x_q)
        (Eq. u_change_r_effic with B = -I), grad = J^-T grad_ref."""
        ue = np.asarray(U)[self.conn]                                     # (E, P)
        gref = np.einsum("qda,ea->eqd", self.B, ue)                      # reference gradient
        gphys = np.einsum("eqdj,eqd->eqj", self.Jinv, gref)             # J^-T grad_ref
        Vdot = gphys / self.rho[:, None, None]
        wref = np.einsum("eqdj,eqj->eqd", self.Jinv, V)                  # J^-1 V
        re = -np.einsum("q,eq,eqd,qda->ea", self.w2, self.detJ, wref, self.B)
        R = np.bincount(self.conn.ravel(), weights=re.ravel(), minlength=self.n_nodes)
        if y_node is not None:
            R[y_node] += y
        return R / self.M, Vdot

    def run_heun(self, nsteps: int, h: float, src=None, receivers=None, U0=None, V0=None):
        """Heun's predictor-corrector (Section 4.2, Time Integration) on the
        first-order system from U = V = 0 (Eq. initial_cond) or (U0, V0); the
        source y(t) = Ricker at the node nearest src, added to dU/dt.
        Returns (U^N, V^N, traces[R, N]) with traces[r, n-1] = U^n."""
        U = np.zeros(self.n_nodes) if U0 is None else np.array(U0, dtype=np.float64)
        V = np.zeros((self.conn.shape[0], self.conn.shape[1], 2)) if V0 is None else np.array(V0, dtype=np.float64)
        s_node = None
        if src is not None:
            sx, sy, f0, t0, amp = src
            s_node = snap(self.node_xy, sx, sy)
        rec_nodes = np.zeros(0, dtype=np.int64)
        if receivers is not None and len(receivers):
            rec_nodes = np.array([snap(self.node_xy, x, y) for x, y in np.asarray(receivers)], dtype=np.int64)
        traces = np.zeros((rec_nodes.size, nsteps))
        yt = (lambda t: float(ricker(t, f0, t0, amp))) if s_node is not None else (lambda t: 0.0)
        for n in range(nsteps):
            Ud1, Vd1 = self.first_order_rhs(U, V, s_node, yt(n * h))
            Up, Vp = U + h * Ud1, V + h * Vd1
            Ud2, Vd2 = self.first_order_rhs(Up, Vp, s_node, yt((n + 1) * h))
            U = U + 0.5 * h * (Ud1 + Ud2)
            V = V + 0.5 * h * (Vd1 + Vd2)
            traces[:, n] = U[rec_nodes]
        return U, V, traces


def _find(conn, nu):
    idx = np.flatnonzero(conn.ravel() == nu)
    return idx // conn.shape[1], idx % conn.shape[1]
