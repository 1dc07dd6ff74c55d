"""Pins of the oracle's memory orderings (Section 4.3 element and node
procedures; Section 6.1 "No Strategy"; random baseline)."""
import os

import numpy as np
import pytest

import gen
from oracle import hilbert, mesh, ordering, sem

GOLD = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")


def test_splitmix64_published_vectors():
    ref = [int(l) for l in open(GOLD) if l.strip() and not l.startswith("#")]
    g = ordering.splitmix64(1234567)
    assert [next(g) for _ in range(5)] == ref
    s = gen.SplitMix64(1234567)
    assert [s.next_u64() for _ in range(5)] == ref
    s1, s2 = gen.SplitMix64(99), gen.SplitMix64(99)
    np.testing.assert_array_equal(s1.uniforms(7), [s2.uniform() for _ in range(7)])


def test_random_order_is_fisher_yates():
    # n = 2: one draw j = next() mod 2 decides the swap
    g = ordering.splitmix64(5)
    j = next(g) % 2
    expect = [1, 0] if j == 0 else [0, 1]
    assert ordering.random_order(2, 5).tolist() == expect
    for n in (1, 7, 1000):
        r = ordering.random_order(n, 42)
        assert sorted(r.tolist()) == list(range(n))


def test_hilbert_grid_sizes_of_the_workloads():
    assert ordering.isqrt_ceil(1024) == 32 and ordering.isqrt_ceil(1025) == 33
    m = gen.unit_square(32)
    W, H, _, _ = ordering.hilbert_grid(m["coords"], m["quads"])
    assert (W, H) == (32, 32)
    m = gen.layered(64, 16)                # aspect ratio 4, like 4096 x 1024
    W, H, ix, iy = ordering.hilbert_grid(m["coords"], m["quads"])
    assert (W, H) == (32, 8)
    assert ix.max() == 31 and iy.max() == 7


def _rectangle(nx, ny, w, h):
    xs, ys = np.linspace(0.0, w, nx + 1), np.linspace(0.0, h, ny + 1)
    coords = np.array([(x, y) for y in ys for x in xs])
    quads = np.array([(j * (nx + 1) + i, j * (nx + 1) + i + 1, (j + 1) * (nx + 1) + i + 1, (j + 1) * (nx + 1) + i)
                      for j in range(ny) for i in range(nx)], dtype=np.int32)
    return coords, quads


def test_hilbert_wide_box_sizes():
    """The alternative box of Section 4.3 (w_b = sqrt(n_e) r, h_b = sqrt(n_e)):
    the same grid as the default on a square domain, r times more columns
    than rows otherwise."""
    m = gen.unit_square(32)
    assert ordering.hilbert_grid(m["coords"], m["quads"], wide=True)[:2] == (32, 32)
    np.testing.assert_array_equal(ordering.hilbert_element_order(m["coords"], m["quads"], wide=True),
                                  ordering.hilbert_element_order(m["coords"], m["quads"]))
    coords, quads = _rectangle(30, 10, 3.0, 1.0)          # E = 300, r = 3
    assert ordering.hilbert_grid(coords, quads)[:2] == (18, 6)          # W = ceil(sqrt 300), H = W / r
    assert ordering.hilbert_grid(coords, quads, wide=True)[:2] == (54, 18)  # H = ceil(sqrt 300), W = H r
    m = gen.layered(64, 16)
    assert ordering.hilbert_grid(m["coords"], m["quads"], wide=True)[:2] == (128, 32)


def test_hilbert_wide_order_brute_force():
    """Cells found by scanning every column and row interval (no floor
    formula); the list L is the elements sorted by the curve rank of their
    cell. With 54 x 18 cells over 30 x 10 elements no centroid lies on a cell
    edge and no cell holds two elements."""
    coords, quads = _rectangle(30, 10, 3.0, 1.0)
    W, H = 54, 18
    cx = coords[quads][:, :, 0].mean(axis=1)
    cy = coords[quads][:, :, 1].mean(axis=1)
    ix = np.array([next(k for k in range(W) if k * 3.0 / W < x < (k + 1) * 3.0 / W) for x in cx])
    iy = np.array([next(k for k in range(H) if k * 1.0 / H < y < (k + 1) * 1.0 / H) for y in cy])
    assert len(set(zip(ix.tolist(), iy.tolist()))) == quads.shape[0]
    rank = hilbert.rank_grid(W, H)
    expect = np.argsort(rank[ix, iy], kind="stable")
    L = ordering.hilbert_element_order(coords, quads, wide=True)
    np.testing.assert_array_equal(L, expect)
    # the default box (18 x 6 cells, several elements per cell) orders differently
    assert not np.array_equal(ordering.hilbert_element_order(coords, quads), L)


def test_homogeneous_32x32_element_order_is_listing1_order5():
    """On the 32 x 32 unit square each curve cell holds exactly one element, so
    the element list L is the standard curve of order 5 (Listing 1)."""
    m = gen.unit_square(32)
    L = ordering.hilbert_element_order(m["coords"], m["quads"])
    cells = hilbert.listing1_cells(5)
    np.testing.assert_array_equal(L, cells[:, 1] * 32 + cells[:, 0])


def test_hilbert_order_follows_geometry_not_labels():
    m = gen.unit_square(16)
    r = gen.relabel(m, seed=9)
    L0 = ordering.hilbert_element_order(m["coords"], m["quads"])
    L1 = ordering.hilbert_element_order(r["coords"], r["quads"])
    c0 = m["coords"][m["quads"][L0]].mean(axis=1)
    c1 = r["coords"][r["quads"][L1]].mean(axis=1)
    np.testing.assert_allclose(c0, c1, atol=1e-15)


def test_many_elements_per_cell_keep_input_order():
    m = gen.graded(24, seed=4)
    W, H, ix, iy = ordering.hilbert_grid(m["coords"], m["quads"])
    L = ordering.hilbert_element_order(m["coords"], m["quads"])
    rank = hilbert.rank_grid(W, H)
    key = rank[ix[L], iy[L]]
    assert np.all(np.diff(key) >= 0)
    same = np.diff(key) == 0
    assert np.all(np.diff(L)[same] > 0)
    assert sorted(L.tolist()) == list(range(L.size))


def test_node_degree_brute_force():
    m = gen.relabel(gen.graded(4, seed=2), seed=1)
    conn, n, _ = mesh.canonical_numbering(m["quads"], m["coords"].shape[0], 3)
    deg = ordering.node_degrees(conn, n)
    nbr = [set() for _ in range(n)]
    for row in conn:
        for a in row:
            nbr[a].update(int(b) for b in row if b != a)
    np.testing.assert_array_equal(deg, [len(s) for s in nbr])
    # order 3 on quads: interior node degree P - 1 = 15
    assert deg.min() == 15


@pytest.mark.parametrize("kind", ["rowmajor", "hilbert"])
def test_node_renumbering_vectorised_equals_loop(kind):
    m = gen.relabel(gen.graded(10, seed=6), seed=2)
    conn, n, _ = mesh.canonical_numbering(m["quads"], m["coords"].shape[0], 4)
    deg = ordering.node_degrees(conn, n)
    eo, no = ordering.orderings(kind, m["coords"], m["quads"], conn, n, degree=deg)
    np.testing.assert_array_equal(no, ordering.renumber_nodes_loop(conn, eo, deg))
    assert sorted(no.tolist()) == list(range(n))
    # first-touch property: new node ids grow with the first element that touches them
    new_of_old = ordering.inverse(no)
    first = np.full(n, -1)
    for k, e in enumerate(eo):
        for v in conn[e]:
            if first[v] < 0:
                first[v] = k
    assert np.all(np.diff(first[no]) >= 0)
    # inside one element's group, degrees ascend
    grp = first[no]
    d = deg[no]
    same = np.diff(grp) == 0
    assert np.all(np.diff(d)[same] >= 0)


@pytest.mark.parametrize("kind", ["none", "rowmajor", "random", "hilbert", "hilbert_wide"])
def test_orderings_are_permutations(kind):
    m = gen.graded(9, seed=3)
    conn, n, _ = mesh.canonical_numbering(m["quads"], m["coords"].shape[0], 2)
    eo, no = ordering.orderings(kind, m["coords"], m["quads"], conn, n, seed=7)
    assert sorted(eo.tolist()) == list(range(conn.shape[0]))
    assert sorted(no.tolist()) == list(range(n))
    if kind == "random":
        np.testing.assert_array_equal(eo, ordering.random_order(conn.shape[0], 9))
        np.testing.assert_array_equal(no, ordering.random_order(n, 10))


def test_wavefield_independent_of_input_labels():
    """The method must not change the result: the same geometry listed in a
    scrambled order gives the same wavefield at the same physical points."""
    m = gen.graded(6, seed=5)
    r = gen.relabel(m, seed=8)
    out = []
    for mm in (m, r):
        S = sem.SEM(mm["coords"], mm["quads"], 4, mm["vel"], mm["rho"])
        dt = 2e-4
        u, _, tr = S.run(120, dt, src=(0.5, 0.5, 10.0, 0.12, 1.0),
                         receivers=np.array([[0.3, 0.9], [0.8, 0.2]]))
        key = np.lexsort((S.node_xy[:, 1].round(12), S.node_xy[:, 0].round(12)))
        out.append((u[key], tr))
    scale = np.abs(out[0][0]).max()
    np.testing.assert_allclose(out[0][0], out[1][0], atol=1e-12 * scale)
    np.testing.assert_allclose(out[0][1], out[1][1], atol=1e-12 * scale)


def test_node_walks_hand_traced_two_quads():
    """Section 6.1's node walks traced by hand on two unit quads side by side
    (order 1, nodes = vertices 0..5: bottom row 0,1,2, top row 3,4,5).
    Connections (sharing a quad): degrees 3,5,3,3,5,3. Connectivity walk:
    0 (fewest) -> 3 (deg 3) -> 1 (deg 5, lower id than 4) -> 2 (deg 3, lower id
    than 5) -> 5 -> 4. Distance walk from (0, 0): 0 -> 1 (d^2 1, ties with 3,
    lower id) -> 3 (d^2 1) -> 4 (d^2 2) -> 2 (d^2 4) -> 5. Elements are listed
    as their nodes are first reached: [0, 1] in both."""
    coords = np.array([[0, 0], [1, 0], [2, 0], [0, 1], [1, 1], [2, 1]], dtype=np.float64)
    quads = np.array([[0, 1, 4, 3], [1, 2, 5, 4]], dtype=np.int64)
    conn, n, edges = mesh.canonical_numbering(quads, 6, 1)
    xy = mesh.node_coordinates(coords, quads, 1, conn, edges)
    eo, no = ordering.orderings("connectivity", coords, quads, conn, n)
    assert no.tolist() == [0, 3, 1, 2, 5, 4] and eo.tolist() == [0, 1]
    eo, no = ordering.orderings("distance", coords, quads, conn, n, node_xy=xy)
    assert no.tolist() == [0, 1, 3, 4, 2, 5] and eo.tolist() == [0, 1]


@pytest.mark.parametrize("kind", ["connectivity", "distance"])
def test_node_walks_are_permutations_and_mostly_adjacent(kind):
    m = gen.graded(12, seed=2)
    conn, n, edges = mesh.canonical_numbering(m["quads"], m["coords"].shape[0], 3)
    xy = mesh.node_coordinates(m["coords"], m["quads"], 3, conn, edges)
    eo, no = ordering.orderings(kind, m["coords"], m["quads"], conn, n, node_xy=xy)
    assert sorted(eo.tolist()) == list(range(conn.shape[0]))
    assert sorted(no.tolist()) == list(range(n))
    # consecutive nodes share an element except right after a back-up
    share = 0
    elems_of = [set() for _ in range(n)]
    for e, row in enumerate(conn):
        for v in row:
            elems_of[v].add(e)
    for a, b in zip(no[:-1], no[1:]):
        share += bool(elems_of[a] & elems_of[b])
    assert share >= 0.9 * (n - 1)
