"""Host-side parts of the C ABI, checked against the oracle on the CPU:
exported symbols, canonical numbering, Hilbert curve, orderings (bit-exact),
snapping, CFL step and input validation. No device is touched."""
import os
import re

import numpy as np
import pytest

import gen
from oracle import hilbert, mesh, ordering, sem as osem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_08416_gb300 import build
    build.build()
    import paper_2104_08416_gb300 as P
    return P


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "sem.h")).read()
    declared = set(re.findall(r"^\s*(?:sem_status|void|const char\*)\s+(sem_\w+)\(", hdr, re.M))
    assert len(declared) >= 25
    assert declared == set(lib.EXPORTS)
    so = lib.load()
    for name in declared:
        assert hasattr(so, name), name


@pytest.mark.parametrize("W,H", [(1, 1), (2, 2), (4, 4), (32, 32), (3, 5), (5, 4), (7, 7), (64, 16), (2048, 8),
                                 (13, 29), (1, 9), (9, 1), (100, 37)])
def test_hilbert_cells_bit_exact(lib, W, H):
    np.testing.assert_array_equal(lib.sem_hilbert_cells(W, H), hilbert.generalized_cells(W, H))


def test_hilbert_cells_listing1_order5(lib):
    np.testing.assert_array_equal(lib.sem_hilbert_cells(32, 32), hilbert.listing1_cells(5))


def _meshes():
    yield "unit32", gen.unit_square(32)
    yield "graded24", gen.graded(24, seed=7)
    yield "graded_relab", gen.relabel(gen.graded(12, seed=3), seed=5)
    yield "layered", gen.layered(64, 16)
    yield "unit_relab", gen.relabel(gen.unit_square(10), seed=1)


@pytest.mark.parametrize("kind", ["none", "rowmajor", "random", "hilbert", "connectivity", "distance", "hilbert_wide"])
@pytest.mark.parametrize("p", [1, 2, 4])
def test_orderings_bit_exact(lib, kind, p):
    for name, m in _meshes():
        conn, n, edges = mesh.canonical_numbering(m["quads"], m["coords"].shape[0], p)
        xy = mesh.node_coordinates(m["coords"], m["quads"], p, conn, edges)
        eo_ref, no_ref = ordering.orderings(kind, m["coords"], m["quads"], conn, n, seed=12345, node_xy=xy)
        eo, no = lib.sem_compute_ordering(m["coords"], m["quads"], p, kind, seed=12345)
        np.testing.assert_array_equal(eo, eo_ref, err_msg=name)
        np.testing.assert_array_equal(no, no_ref, err_msg=name)


def test_node_count(lib):
    for name, m in _meshes():
        for p in (1, 3, 8):
            _, n, _ = mesh.canonical_numbering(m["quads"], m["coords"].shape[0], p)
            assert lib.sem_count_nodes(m["quads"], m["coords"].shape[0], p) == n


@pytest.mark.parametrize("p", [1, 2, 4, 7])
def test_node_coordinates_and_snapping(lib, p):
    m = gen.relabel(gen.graded(8, seed=2), seed=4)
    h = lib.SEM(m["coords"], m["quads"], p, "fp64", stream=0)
    S = osem.SEM(m["coords"], m["quads"], p, m["vel"], m["rho"])
    assert h.n_nodes == S.n_nodes
    np.testing.assert_allclose(h.sem_node_coordinates(), S.node_xy, rtol=0, atol=1e-15)
    h.sem_set_model(m["vel"], m["rho"])
    assert abs(h.sem_cfl_dt() - S.cfl_dt()) <= 1e-14 * S.cfl_dt()
    h.sem_set_source(10.0, 0.12, 1.0, 0.37, 0.61)
    rec = np.array([[0.0, 0.0], [0.5, 1.0], [0.93, 0.12]])
    h.sem_set_receivers(rec, 10)
    s, r = h.sem_get_snapped()
    assert s == osem.snap(S.node_xy, 0.37, 0.61)
    assert r.tolist() == [osem.snap(S.node_xy, x, y) for x, y in rec]
    h.sem_reorder("hilbert")
    e_new, n_new = h.sem_get_permutation()
    conn, n, _ = mesh.canonical_numbering(m["quads"], m["coords"].shape[0], p)
    eo, no = ordering.orderings("hilbert", m["coords"], m["quads"], conn, n)
    np.testing.assert_array_equal(e_new, ordering.inverse(eo))
    np.testing.assert_array_equal(n_new, ordering.inverse(no))
    h.sem_destroy()


def test_gll_rule_through_cfl(lib):
    """The CFL step of one affine square element of side 1 is the smallest GLL
    spacing / 2 (nodes on [-1, 1] scaled to [0, 1]); p = 4: (1 - sqrt(3/7)) / 2."""
    coords = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    quads = np.array([[0, 1, 2, 3]], dtype=np.int32)
    h = lib.SEM(coords, quads, 4, "fp64", stream=0)
    h.sem_set_model([2.0])
    assert abs(h.sem_cfl_dt() - (1 - np.sqrt(3 / 7)) / 2 / 2.0) < 1e-15


def _expect_invalid(lib, coords, quads, p=2):
    with pytest.raises(lib.SemError) as ei:
        lib.SEM(coords, quads, p, "fp64", stream=0)
    assert ei.value.status == lib.SEM_ERR_INVALID_ARG


def test_invalid_meshes_rejected(lib):
    sq = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    _expect_invalid(lib, sq, np.array([[0, 3, 2, 1]], dtype=np.int32))          # clockwise
    _expect_invalid(lib, sq, np.array([[0, 1, 2, 4]], dtype=np.int32))          # index out of range
    _expect_invalid(lib, np.vstack([sq, [[5.0, 5.0]]]), np.array([[0, 1, 2, 3]], dtype=np.int32))  # unused vertex
    _expect_invalid(lib, sq, np.array([[0, 1, 1, 3]], dtype=np.int32))          # repeated vertex
    bow = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])          # self-intersecting
    _expect_invalid(lib, bow, np.array([[0, 1, 2, 3]], dtype=np.int32))
    _expect_invalid(lib, sq, np.array([[0, 1, 2, 3]], dtype=np.int32), p=9)    # order too high
    _expect_invalid(lib, sq, np.zeros((0, 4), dtype=np.int32))                  # empty


def test_state_errors_before_device(lib):
    m = gen.unit_square(2)
    h = lib.SEM(m["coords"], m["quads"], 2, "fp32_kahan", stream=0)
    with pytest.raises(lib.SemError) as ei:
        h.sem_step(1)                      # no model, no dt
    assert ei.value.status == lib.SEM_ERR_STATE
    with pytest.raises(lib.SemError):
        h.sem_set_model(np.full(4, -1.0))
    with pytest.raises(lib.SemError):
        h.sem_set_dt(0.0)
    with pytest.raises(lib.SemError):
        h.sem_reorder(7)
    with pytest.raises(lib.SemError):
        h.sem_set_source(-1.0, 0.0, 1.0, 0.5, 0.5)
    h.sem_destroy()


@pytest.mark.parametrize("kind", ["none", "rowmajor", "random", "hilbert"])
@pytest.mark.parametrize("p", [1, 3, 4, 8])
@pytest.mark.parametrize("eb", [1, 9, 64, 256])
def test_block_plan_replay(lib, kind, p, eb):
    """The step kernel's block plan, replayed on the host with every index
    bounds-checked: each slot reads its own node, the assembled sum equals the
    direct per-slot sum, and each receiver node is recorded by one block."""
    m = gen.relabel(gen.graded(13, seed=p), seed=eb)
    rec = np.array([[0.5, 0.5], [0.0, 0.0], [1.0, 1.0], [0.31, 0.77], [0.5, 0.5]])
    for fp64 in (False, True):
        st, info, msg = lib.sem_plan_check(m["coords"], m["quads"], p, kind, eb, fp64, rec)
        assert st == lib.SEM_OK, msg
        assert info["nblocks"] == -(-m["quads"].shape[0] // eb)
        # first-touch numberings always give the contiguous (DENSE) layout
        if kind in ("rowmajor", "hilbert"):
            assert info["dense"] == 1
        elif info["nblocks"] > 1:
            assert info["dense"] == 0


def test_block_plan_hilbert_has_fewer_open_nodes(lib):
    m = gen.graded(64, seed=3)
    opened = {k: lib.sem_plan_check(m["coords"], m["quads"], 4, k, 64)[1]["open_nodes"]
              for k in ("hilbert", "rowmajor", "random")}
    assert opened["hilbert"] < opened["rowmajor"] < opened["random"], opened


def test_block_plan_replay_at_bench_size(lib):
    """The plan of the benchmark configuration itself (graded 512 x 512,
    order 4, Hilbert, 256-element blocks, FP32 storage, its 16 receivers),
    replayed on the host with every index bounds-checked, with the streamed
    loop's wavefront orders checked topological; the open-node count matches
    what the bench reports for this workload."""
    m = gen.graded(512)
    st, info, msg = lib.sem_plan_check(m["coords"], m["quads"], 4, "hilbert", 256, False, m["receivers"])
    assert st == lib.SEM_OK, msg
    assert info["nblocks"] == 1024 and info["dense"] == 1
    assert info["open_nodes"] == 195565
    assert info["max_colors"] <= 6


def test_stream_tiling_arguments(lib):
    """sem_set_stream_tiling validates its arguments on the host and nothing
    is uploaded before the first streamed launch."""
    m = gen.unit_square(4)
    h = lib.SEM(m["coords"], m["quads"], 2, "fp32_kahan", stream=0)
    assert h.sem_stream_order() == (0, 0)
    for band, window in ((-2, 0), (256, 0), (16, -1)):
        with pytest.raises(lib.SemError) as ei:
            h.sem_set_stream_tiling(band, window)
        assert ei.value.status == lib.SEM_ERR_INVALID_ARG
    for band, window in ((-1, 0), (0, 0), (1, 1), (255, 1000)):
        h.sem_set_stream_tiling(band, window)
    assert h.sem_stream_order() == (0, 0)
    h.sem_destroy()


def test_metric_source_arguments_before_device(lib):
    """sem_set_metric validates on the host: unknown source, the first-order
    scheme with a stored FP32 metric (either call order), FP64 accepts it as
    a no-op; nothing touches the device."""
    m = gen.unit_square(2)
    h = lib.SEM(m["coords"], m["quads"], 2, "fp32", stream=0)
    with pytest.raises(lib.SemError) as ei:
        h.sem_set_metric(7)
    assert ei.value.status == lib.SEM_ERR_INVALID_ARG
    h.sem_set_metric("stored")
    with pytest.raises(lib.SemError) as ei:
        h.sem_set_scheme("heun")
    assert ei.value.status == lib.SEM_ERR_UNSUPPORTED
    h.sem_set_metric("bilinear")
    h.sem_set_scheme("heun")
    with pytest.raises(lib.SemError) as ei:
        h.sem_set_metric("stored")
    assert ei.value.status == lib.SEM_ERR_UNSUPPORTED
    h.sem_destroy()
    g = lib.SEM(m["coords"], m["quads"], 2, "fp64", stream=0)
    g.sem_set_metric("stored")
    g.sem_destroy()
