"""Element and node orderings (integer results, bit-exact).

Test infrastructure only (see the package docstring).

Permutations are returned as `order` arrays: order[new] = old id. The library
exports the inverse maps (new id of each old id); ``inverse`` converts.

* ``hilbert_element_order`` -- Section 4.3, reordering steps 1-4: element
  centroids are mapped to the cells of a W x H grid laid over the mesh's
  bounding box, the cells are walked along the generalized Hilbert curve and
  the elements of each visited cell are appended to the list L. Readings of
  the garbled/open points: the "subrectangle width w_s = w_b / w_m" is a scale
  (cells per unit length), W = ceil(sqrt(n_e)) as an integer, H = max(1,
  ceil(W / r)) with r = w_m / h_m; centroid = ((x0 + x1) + (x2 + x3)) * 0.25;
  cell ix = min(W - 1, floor(((xc - x_min) * W) / w_m)) (iy likewise with H,
  h_m), all in FP64 without fused multiply-add; elements sharing a cell keep
  ascending input id; empty cells are skipped.
* ``renumber_nodes`` -- Section 4.3, node procedure: walk the elements in their
  new order, collect each element's not-yet-seen nodes N^(e) (in local index
  order), sort N^(e) by ascending degree (stable, so ties keep local index
  order) and append. Reading: the degree of a node is the number of distinct
  other nodes that share at least one element with it.
* ``random_order`` -- Fisher-Yates driven by splitmix64: for i = n-1 down to 1,
  j = next() mod (i + 1), swap a[i], a[j]; elements use stream seed+2 and
  nodes stream seed+3 (independently).
* ``orderings(kind)`` -- NONE: identity for both; ROWMAJOR: input element
  order with nodes renumbered as above; RANDOM: random elements and random
  nodes; HILBERT: the curve order with nodes renumbered as above;
  CONNECTIVITY / DISTANCE: Section 6.1's node walks (``node_walk``).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import hilbert as _hilbert

MASK64 = (1 << 64) - 1


def splitmix64(seed: int):
    """Generator of splitmix64 outputs (Steele, Lea & Flood 2014)."""
    s = seed & MASK64
    while True:
        s = (s + 0x9E3779B97F4A7C15) & MASK64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        yield z ^ (z >> 31)


def random_order(n: int, seed: int) -> np.ndarray:
    a = list(range(n))
    g = splitmix64(seed)
    for i in range(n - 1, 0, -1):
        j = next(g) % (i + 1)
        a[i], a[j] = a[j], a[i]
    return np.array(a, dtype=np.int64)


def inverse(order: np.ndarray) -> np.ndarray:
    inv = np.empty_like(order)
    inv[order] = np.arange(order.size, dtype=order.dtype)
    return inv


def isqrt_ceil(n: int) -> int:
    r = math.isqrt(n)
    return r if r * r == n else r + 1


def hilbert_grid(coords: np.ndarray, quads: np.ndarray, wide: bool = False):
    """Return (W, H, ix[E], iy[E]): the curve grid and each element's cell.

    Section 4.3 sizes the bounding box w_b = sqrt(n_e), h_b = sqrt(n_e) / r
    (r = w_m / h_m); read with integer cells: W = ceil(sqrt(E)), H =
    max(1, ceil(W / r)). `wide` takes the alternative the same section offers
    for changing how many elements fall in one step of the curve, w_b =
    sqrt(n_e) r and h_b = sqrt(n_e): H = ceil(sqrt(E)), W = max(1, ceil(H r)).
    """
    coords = np.asarray(coords, dtype=np.float64)
    quads = np.asarray(quads, dtype=np.int64)
    E = quads.shape[0]
    xmin, ymin = coords[:, 0].min(), coords[:, 1].min()
    wm = coords[:, 0].max() - xmin
    hm = coords[:, 1].max() - ymin
    r = wm / hm
    if not wide:
        W = isqrt_ceil(E)
        H = max(1, math.ceil(W / r))
    else:
        H = isqrt_ceil(E)
        W = max(1, math.ceil(H * r))
    c = coords[quads]                                     # (E, 4, 2)
    xc = ((c[:, 0, 0] + c[:, 1, 0]) + (c[:, 2, 0] + c[:, 3, 0])) * 0.25
    yc = ((c[:, 0, 1] + c[:, 1, 1]) + (c[:, 2, 1] + c[:, 3, 1])) * 0.25
    ix = np.minimum(W - 1, np.floor(((xc - xmin) * float(W)) / wm).astype(np.int64))
    iy = np.minimum(H - 1, np.floor(((yc - ymin) * float(H)) / hm).astype(np.int64))
    return W, H, np.maximum(ix, 0), np.maximum(iy, 0)


def hilbert_element_order(coords, quads, wide: bool = False) -> np.ndarray:
    """The list L of Section 4.3 as order[new] = old element id."""
    W, H, ix, iy = hilbert_grid(coords, quads, wide)
    rank = _hilbert.rank_grid(W, H)
    key = rank[ix, iy]
    return np.argsort(key, kind="stable").astype(np.int64)   # ties: ascending input id


def node_degrees(conn: np.ndarray, n_nodes: int) -> np.ndarray:
    """Number of distinct other nodes sharing an element with each node."""
    E, P = conn.shape
    A = sp.csr_matrix((np.ones(E * P, dtype=np.int8), (np.repeat(np.arange(E), P), conn.ravel())),
                      shape=(E, n_nodes))
    C = (A.T.astype(np.int32) @ A.astype(np.int32)).tocsr()
    return np.diff(C.indptr).astype(np.int64) - 1


def renumber_nodes_loop(conn, elem_order, degree) -> np.ndarray:
    """The node procedure of Section 4.3 as a plain loop (small meshes)."""
    seen = np.zeros(int(conn.max()) + 1, dtype=bool)
    out = []
    for e in elem_order:
        group = []
        for v in conn[e]:
            if not seen[v]:
                seen[v] = True
                group.append(int(v))
        group.sort(key=lambda v: degree[v])               # stable
        out.extend(group)
    return np.array(out, dtype=np.int64)


def renumber_nodes(conn, elem_order, degree) -> np.ndarray:
    """Same result as `renumber_nodes_loop`, by sorting on (first-touching
    element position, degree, local index of the first touch)."""
    P = conn.shape[1]
    seq = conn[elem_order].ravel()
    nodes, first = np.unique(seq, return_index=True)
    group = first // P
    local = first % P
    idx = np.lexsort((local, degree[nodes], group))
    return nodes[idx].astype(np.int64)


def node_walk(conn, n_nodes: int, key) -> tuple:
    """Section 6.1's node walks ("Node Connectivity", "Node Distance"): from
    the node of smallest key, always to the connected (element-sharing),
    not yet visited node of smallest key; ties go to the lower node id. The
    paper does not say what happens when no such node exists; reading: back up
    along the walk to the latest node that has one, and when the connected part
    is exhausted restart at the unvisited node of smallest key. Each visited
    node is appended to the node order, and the elements containing it that
    are not yet listed are appended, in ascending id, to the element order.
    key[n_nodes]: number of connections, or squared distance to the reference
    point. Plain loops over an explicit adjacency (small meshes)."""
    E, P = conn.shape
    A = sp.csr_matrix((np.ones(E * P, dtype=np.int8), (np.repeat(np.arange(E), P), conn.ravel())),
                      shape=(E, n_nodes))
    nbr = (A.T.astype(np.int32) @ A.astype(np.int32)).tocsr()
    node_elems = A.T.tocsr()
    rank = sorted(range(n_nodes), key=lambda v: (key[v], v))
    visited = np.zeros(n_nodes, dtype=bool)
    listed = np.zeros(E, dtype=bool)
    eo, no = [], []

    def visit(v):
        visited[v] = True
        no.append(v)
        for e in sorted(node_elems.indices[node_elems.indptr[v]:node_elems.indptr[v + 1]]):
            if not listed[e]:
                listed[e] = True
                eo.append(int(e))

    for start in rank:
        if visited[start]:
            continue
        visit(start)
        path = [start]
        while path:
            top = path[-1]
            cand = [int(w) for w in nbr.indices[nbr.indptr[top]:nbr.indptr[top + 1]] if not visited[w]]
            if not cand:
                path.pop()
                continue
            nxt = min(cand, key=lambda w: (key[w], w))
            visit(nxt)
            path.append(nxt)
    return np.array(eo, dtype=np.int64), np.array(no, dtype=np.int64)


def orderings(kind: str, coords, quads, conn, n_nodes, seed: int = 2104084160, degree=None, node_xy=None):
    """(elem_order, node_order) for kind in none/rowmajor/random/hilbert/
    connectivity/distance/hilbert_wide (node_xy needed for distance)."""
    E = conn.shape[0]
    kind = kind.lower()
    if kind == "connectivity":
        return node_walk(conn, n_nodes, node_degrees(conn, n_nodes) if degree is None else degree)
    if kind == "distance":
        # reference point: the lower-left corner of the bounding box (Section
        # 6.1); reading: squared distances compared in units of 2^-30 of the
        # box diagonal squared (floor), so mirror-equal distances tie exactly
        xy = np.asarray(node_xy, dtype=np.float64)
        c = np.asarray(coords, dtype=np.float64)
        x0, y0 = c[:, 0].min(), c[:, 1].min()
        w, h = c[:, 0].max() - x0, c[:, 1].max() - y0
        dx = xy[:, 0] - x0
        dy = xy[:, 1] - y0
        key = np.floor((dx * dx + dy * dy) / (w * w + h * h) * 2.0 ** 30).astype(np.int64)
        return node_walk(conn, n_nodes, key)
    if kind == "none":
        return np.arange(E, dtype=np.int64), np.arange(n_nodes, dtype=np.int64)
    if kind == "random":
        return random_order(E, seed + 2), random_order(n_nodes, seed + 3)
    if kind == "rowmajor":
        eo = np.arange(E, dtype=np.int64)
    elif kind == "hilbert":
        eo = hilbert_element_order(coords, quads)
    elif kind == "hilbert_wide":
        eo = hilbert_element_order(coords, quads, wide=True)
    else:
        raise ValueError(kind)
    if degree is None:
        degree = node_degrees(conn, n_nodes)
    return eo, renumber_nodes(conn, eo, degree)
