"""Canonical SEM node numbering and bilinear quad geometry (FP64).

Test infrastructure only (see the package docstring).

Section 4.2 represents the solution by its values U_mu at global SEM nodes,
with mu(p, e) mapping local node p of element e to its global node. The paper
adds SEM nodes to Gmsh meshes in memory but does not fix their numbering, so
this module states one (it is the "original" numbering that all user-facing
arrays use):

* local point (i, j), i, j in 0..p, has local index j*(p+1) + i; xi runs from
  corner c0 to c1, eta from c0 to c3 (corners given counter-clockwise);
* global ids: (1) the mesh vertices in input order; (2) edge-interior nodes,
  edges taken in order of first appearance while scanning e = 0..E-1 over the
  local edges (c0c1, c1c2, c2c3, c3c0), each edge contributing p-1 ids ordered
  from its lower vertex id to its higher one; (3) element-interior nodes,
  e ascending, (i, j) with i fastest.

Geometry generalises the affine map of Section 4.2 (x = x^(e) + J xhat) to the
bilinear map of a quad, so the Jacobian J, its determinant and its inverse
(the K^(e) of Eq. deriv_u) are evaluated at every GLL point.
"""
from __future__ import annotations

import numpy as np

from . import gll as _gll

LOCAL_EDGES = ((0, 1), (1, 2), (2, 3), (3, 0))


def corner_local_index(p: int):
    n = p + 1
    return (0, p, p * n + p, p * n)


def edge_local_indices(p: int, le: int):
    """Local indices of the p-1 interior points of local edge `le`, listed from
    the edge's first corner towards its second corner."""
    n = p + 1
    t = range(1, p)
    if le == 0:
        return [k for k in t]
    if le == 1:
        return [k * n + p for k in t]
    if le == 2:
        return [p * n + (p - k) for k in t]
    return [(p - k) * n for k in t]


def canonical_numbering(quads: np.ndarray, nv: int, p: int):
    """Return (conn[E, P] int64 global ids, n_nodes, edges).

    `edges` is an int64 array with one row (lower vertex, higher vertex,
    first id) per canonical edge, in order of first appearance.
    """
    quads = np.asarray(quads, dtype=np.int64)
    E = quads.shape[0]
    n = p + 1
    P = n * n
    conn = np.full((E, P), -1, dtype=np.int64)
    cl = corner_local_index(p)
    for c in range(4):
        conn[:, cl[c]] = quads[:, c]
    # local edges scanned e-major, local-edge-minor
    va = np.stack([quads[:, a] for a, _ in LOCAL_EDGES], axis=1).ravel()
    vb = np.stack([quads[:, b] for _, b in LOCAL_EDGES], axis=1).ravel()
    lo, hi = np.minimum(va, vb), np.maximum(va, vb)
    key = lo * np.int64(max(nv, 1)) + hi
    uniq, first, inv = np.unique(key, return_index=True, return_inverse=True)
    rank_of_uniq = np.empty(uniq.size, dtype=np.int64)
    rank_of_uniq[np.argsort(first, kind="stable")] = np.arange(uniq.size)
    base = nv + rank_of_uniq[inv] * (p - 1)            # per (e, le)
    forward = (va < vb)
    for le in range(4):
        b_e = base.reshape(E, 4)[:, le]
        f_e = forward.reshape(E, 4)[:, le]
        for t, li in enumerate(edge_local_indices(p, le), start=1):
            k = np.where(f_e, t, p - t)                 # position from the lower vertex
            conn[:, li] = b_e + (k - 1)
    next_id = nv + uniq.size * (p - 1)
    m = (p - 1) * (p - 1)
    if m:
        interior = next_id + np.arange(E, dtype=np.int64)[:, None] * m + np.arange(m)[None, :]
        jj, ii = np.meshgrid(np.arange(1, p), np.arange(1, p), indexing="ij")
        conn[:, (jj * n + ii).ravel()] = interior
        next_id += E * m
    order = np.argsort(first, kind="stable")
    edges = np.stack([lo[first[order]], hi[first[order]],
                      nv + np.arange(uniq.size, dtype=np.int64) * (p - 1)], axis=1)
    return conn, int(next_id), edges


def bilinear(corners: np.ndarray, xi, eta):
    """X(xi, eta) = 1/4 [(1-xi)(1-eta) X0 + (1+xi)(1-eta) X1 + (1+xi)(1+eta) X2
    + (1-xi)(1+eta) X3], summed left to right. corners: (..., 4, 2)."""
    a = 0.25 * (1 - xi) * (1 - eta)
    b = 0.25 * (1 + xi) * (1 - eta)
    c = 0.25 * (1 + xi) * (1 + eta)
    d = 0.25 * (1 - xi) * (1 + eta)
    return (((a * corners[..., 0, :] + b * corners[..., 1, :]) + c * corners[..., 2, :])
            + d * corners[..., 3, :])


def node_coordinates(coords: np.ndarray, quads: np.ndarray, p: int, conn=None, edges=None):
    """Physical position of every global node (used to snap sources/receivers).

    Vertices: their input coordinates. Edge node k (1..p-1) of edge (lo, hi):
    0.5*((1 - s_k) X_lo + (1 + s_k) X_hi), s_k the k-th GLL node.
    Interior node (i, j) of element e: the bilinear map at (s_i, s_j).
    """
    coords = np.asarray(coords, dtype=np.float64)
    quads = np.asarray(quads, dtype=np.int64)
    nv = coords.shape[0]
    if conn is None or edges is None:
        conn, _, edges = canonical_numbering(quads, nv, p)
    s = _gll.gll_nodes(p)
    n_nodes = int(conn.max()) + 1 if conn.size else nv
    xy = np.zeros((n_nodes, 2))
    xy[:nv] = coords
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 3)
    Xlo, Xhi = coords[edges[:, 0]], coords[edges[:, 1]]
    for k in range(1, p):
        xy[edges[:, 2] + k - 1] = 0.5 * ((1.0 - s[k]) * Xlo + (1.0 + s[k]) * Xhi)
    n = p + 1
    corners = coords[quads]                       # (E, 4, 2)
    for j in range(1, p):
        for i in range(1, p):
            xy[conn[:, j * n + i]] = bilinear(corners, s[i], s[j])
    return xy


def jacobians(coords: np.ndarray, quads: np.ndarray, p: int):
    """J[e, q] (2x2, J[a, b] = d x_a / d xi_b) at every GLL point q = j*(p+1)+i."""
    coords = np.asarray(coords, dtype=np.float64)
    corners = coords[np.asarray(quads, dtype=np.int64)]   # (E, 4, 2)
    s = _gll.gll_nodes(p)
    n = p + 1
    E = corners.shape[0]
    J = np.zeros((E, n * n, 2, 2))
    X0, X1, X2, X3 = (corners[:, c, :] for c in range(4))
    for j in range(n):
        eta = s[j]
        for i in range(n):
            xi = s[i]
            dxi = 0.25 * (-(1 - eta) * X0 + (1 - eta) * X1 + (1 + eta) * X2 - (1 + eta) * X3)
            deta = 0.25 * (-(1 - xi) * X0 - (1 + xi) * X1 + (1 + xi) * X2 + (1 - xi) * X3)
            J[:, j * n + i, :, 0] = dxi
            J[:, j * n + i, :, 1] = deta
    return J


def validate(coords, quads, p: int):
    """Raise ValueError for out-of-range indices, unreferenced vertices, edges
    shared by more than two elements, or a non-positive Jacobian at a GLL point."""
    coords = np.asarray(coords)
    quads = np.asarray(quads)
    nv = coords.shape[0]
    if quads.size and (quads.min() < 0 or quads.max() >= nv):
        raise ValueError("quad index out of range")
    if np.unique(quads).size != nv:
        raise ValueError("unreferenced vertex")
    cnt = {}
    for q in quads:
        for a, b in LOCAL_EDGES:
            key = (min(q[a], q[b]), max(q[a], q[b]))
            cnt[key] = cnt.get(key, 0) + 1
    if any(v > 2 for v in cnt.values()):
        raise ValueError("edge shared by more than two elements")
    J = jacobians(coords, quads, p)
    det = J[..., 0, 0] * J[..., 1, 1] - J[..., 0, 1] * J[..., 1, 0]
    if (det <= 0).any():
        raise ValueError("non-positive Jacobian")
