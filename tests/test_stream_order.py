"""Host-side wavefront order of the streamed time loop (sem_stream_schedule).

The streamed loop runs (step, block) units in ticket order and each unit
waits for the previous step at its block's neighbours; the waits end only if
the order is topological. These tests check the library's order against that
definition directly (every unit after step j-1 of each neighbour), that every
unit of the band appears once, that the levels are breadth-first distances
from their level-0 block (brute force), that the tiles are those of the
stated key floor((level + j) / W), and that a block's next step comes within
about a tile row of units. No GPU is needed.
"""
from collections import deque

import numpy as np
import pytest

import gen

SHIFT = 24


@pytest.fixture(scope="module")
def P():
    import paper_2104_08416_gb300 as P
    from paper_2104_08416_gb300 import build
    build.build()
    P.load()
    return P


def grid_graph(R, C, diag=True):
    """Blocks on an R x C grid, adjacent when they share a node (8-neighbour
    with diag, else 4-neighbour), itself included; CSR."""
    nbrs = []
    for r in range(R):
        for c in range(C):
            lst = []
            for dr in (-1, 0, 1):
                for dc in (-1, 0, 1):
                    if not diag and dr and dc:
                        continue
                    rr, cc = r + dr, c + dc
                    if 0 <= rr < R and 0 <= cc < C:
                        lst.append(rr * C + cc)
            nbrs.append(sorted(lst))
    return to_csr(nbrs)


def to_csr(nbrs):
    ptr = np.zeros(len(nbrs) + 1, dtype=np.int32)
    ptr[1:] = np.cumsum([len(x) for x in nbrs])
    dep = np.array([y for x in nbrs for y in x], dtype=np.int32)
    return ptr, dep


def relabel(ptr, dep, perm):
    """Graph with block b renamed perm[b]."""
    nb = len(ptr) - 1
    nbrs = [None] * nb
    for b in range(nb):
        nbrs[perm[b]] = sorted(int(perm[y]) for y in dep[ptr[b]:ptr[b + 1]])
    return to_csr(nbrs)


def bfs(ptr, dep, root):
    nb = len(ptr) - 1
    d = np.full(nb, -1)
    d[root] = 0
    q = deque([root])
    while q:
        x = q.popleft()
        for y in dep[ptr[x]:ptr[x + 1]]:
            if d[y] < 0:
                d[y] = d[x] + 1
                q.append(y)
    return d


def check_order(ptr, dep, T, W, sched, lev):
    nb = len(ptr) - 1
    j = (sched >> SHIFT).astype(np.int64)
    b = (sched & ((1 << SHIFT) - 1)).astype(np.int64)
    assert len(sched) == T * nb
    pos = np.full((T, nb), -1)
    pos[j, b] = np.arange(len(sched))
    assert (pos >= 0).all(), "a unit is missing"
    # topological: after step j-1 of every neighbour (itself included)
    for bb in range(nb):
        for y in dep[ptr[bb]:ptr[bb + 1]]:
            assert (pos[1:, bb] > pos[:-1, y]).all(), (bb, y)
    # levels: breadth-first distances from the level-0 block of each part
    seen = np.zeros(nb, dtype=bool)
    for root in np.flatnonzero(lev == 0):
        d = bfs(ptr, dep, root)
        part = d >= 0
        assert not seen[part].any()
        seen |= part
        assert np.array_equal(lev[part], d[part])
    assert seen.all()
    # the stated key: tile, then step, then level, then block id
    key = np.stack([(lev[b] + j) // W, j, lev[b], b], axis=1)
    assert (np.diff(key[:, 0]) >= 0).all()
    order = np.lexsort(key.T[::-1])
    assert np.array_equal(order, np.arange(len(sched)))
    return pos


@pytest.mark.parametrize("R,C,diag", [(32, 32, True), (8, 64, True), (17, 5, False), (1, 9, True), (1, 1, True)])
@pytest.mark.parametrize("T,W", [(16, 1), (16, 4), (16, 14), (1, 3), (5, 100), (255, 2)])
def test_grid_graphs(P, R, C, diag, T, W):
    ptr, dep = grid_graph(R, C, diag)
    sched, lev = P.sem_stream_schedule(ptr, dep, T, W)
    pos = check_order(ptr, dep, T, W, sched, lev)
    # the level-0 block is an end of a longest shortest path (a corner here)
    r0, c0 = divmod(int(np.flatnonzero(lev == 0)[0]), C)
    assert r0 in (0, R - 1) and c0 in (0, C - 1)
    # reuse distance: a block's next step comes within one tile row of units
    # unless the block is at its tile's top level
    if T > 1 and R * C > 1:
        nb = R * C
        per_level = np.bincount(lev)
        gap = pos[1:] - pos[:-1]
        top = ((lev[None, :] + np.arange(T - 1)[:, None]) % W) == W - 1
        row = W * per_level.max() + per_level.max()
        assert (gap[~top] <= row).all()
        assert (gap > 0).all()
        del nb


def test_shuffled_and_disconnected_graphs(P):
    rng = np.random.default_rng(3)
    a = grid_graph(12, 20)
    b = grid_graph(7, 7, diag=False)
    nb_a = len(a[0]) - 1
    nbrs = [list(a[1][a[0][i]:a[0][i + 1]]) for i in range(nb_a)]
    nbrs += [[y + nb_a for y in b[1][b[0][i]:b[0][i + 1]]] for i in range(len(b[0]) - 1)]
    nbrs.append([len(nbrs)])                      # an isolated block
    ptr, dep = to_csr(nbrs)
    ptr, dep = relabel(ptr, dep, rng.permutation(len(ptr) - 1))
    for T, W in ((16, 3), (7, 1), (3, 50)):
        sched, lev = P.sem_stream_schedule(ptr, dep, T, W)
        check_order(ptr, dep, T, W, sched, lev)


@pytest.mark.parametrize("kind,eb", [("hilbert", 64), ("hilbert", 256), ("rowmajor", 48), ("random", 100)])
def test_block_graphs_of_element_blocks(P, kind, eb):
    """The graph the streamed loop uses: blocks of eb consecutive elements in
    the chosen memory order, adjacent when they share a global node (built
    here from the oracle's canonical numbering and the library's element
    order)."""
    from oracle import mesh as omesh
    m = gen.graded(40, seed=11)
    p = 4
    conn = omesh.canonical_numbering(m["quads"], m["coords"].shape[0], p)[0]
    eo, _ = P.sem_compute_ordering(m["coords"], m["quads"], p, kind)
    blk = np.empty(len(eo), dtype=np.int64)
    blk[eo] = np.arange(len(eo)) // eb
    nb = int(blk.max()) + 1
    node_blocks = {}
    for e in range(len(eo)):
        for g in conn[e]:
            node_blocks.setdefault(int(g), set()).add(int(blk[e]))
    nbrs = [{b} for b in range(nb)]
    for bs in node_blocks.values():
        for x in bs:
            nbrs[x] |= bs
    ptr, dep = to_csr([sorted(x) for x in nbrs])
    for T, W in ((16, 1), (16, 4), (16, 30)):
        sched, lev = P.sem_stream_schedule(ptr, dep, T, W)
        check_order(ptr, dep, T, W, sched, lev)


@pytest.mark.parametrize("bad", ["no_self", "asym", "range"])
def test_malformed_graphs_rejected(P, bad):
    ptr, dep = grid_graph(3, 3)
    dep = dep.copy()
    if bad == "no_self":
        nbrs = [[y for y in dep[ptr[i]:ptr[i + 1]] if y != i] for i in range(9)]
        ptr, dep = to_csr(nbrs)
    elif bad == "asym":
        nbrs = [list(dep[ptr[i]:ptr[i + 1]]) for i in range(9)]
        nbrs[0] = sorted(set(nbrs[0]) | {8})
        ptr, dep = to_csr(nbrs)
    else:
        dep[3] = 9
    with pytest.raises(P.SemError) as ei:
        P.sem_stream_schedule(ptr, dep, 16, 2)
    assert ei.value.status == P.SEM_ERR_INVALID_ARG


def test_band_and_window_limits(P):
    ptr, dep = grid_graph(4, 4)
    for T, W in ((0, 1), (256, 1), (4, 0)):
        with pytest.raises(P.SemError):
            P.sem_stream_schedule(ptr, dep, T, W)
