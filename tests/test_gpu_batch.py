"""Batched shots (sem_batch_*): several meshes of different sizes and orders
advanced together must give, shot by shot, bit for bit the results of
stepping each handle on its own with the same block size; with the
autotuner on, the results stay within the parity tolerance of the oracle."""
import numpy as np
import pytest

import gen
from oracle import sem as osem
from tests._gpu_common import FP32_TOL, need_gpu, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return need_gpu()


def _shots():
    # (mesh, order, ordering): uneven sizes, orders 3..7, a repeated order,
    # a scrambled input numbering
    return [
        (gen.graded(10, seed=1), 3, "hilbert"),
        (gen.graded(16, seed=2), 4, "hilbert"),
        (gen.unit_square(12), 5, "rowmajor"),
        (gen.graded(7, seed=3), 7, "hilbert"),
        (gen.graded(21, seed=4), 4, "random"),
        (gen.relabel(gen.graded(9, seed=5), seed=6), 6, "none"),
    ]


def _handle(P, m, p, kind, prec, nmax, eb=0):
    h = P.SEM(m["coords"], m["quads"], p, prec)
    h.sem_reorder(kind, 3)
    h.sem_set_model(m["vel"], m["rho"])
    if eb:
        h.sem_set_tuning(eb)
    h.sem_set_source(m["f0"], m["t0"], m["amp"], *m["src_xy"])
    h.sem_set_receivers(m["receivers"], nmax)
    S = osem.SEM(m["coords"], m["quads"], p, m["vel"], m["rho"])
    h.sem_set_dt(0.3 * S.cfl_dt())
    return h


@pytest.mark.parametrize("prec", ["fp32_kahan", "fp64", "fp32"])
def test_batch_equals_individual_runs(P, prec):
    shots = _shots()
    nmax = 60
    chunks = (37, 1, 20)            # graph replays, a single step, a remainder
    batch_h = [_handle(P, m, p, k, prec, nmax, eb=11) for m, p, k in shots]
    solo_h = [_handle(P, m, p, k, prec, nmax, eb=11) for m, p, k in shots]
    b = P.SEMBatch(batch_h)
    for c in chunks:
        b.sem_batch_step(c)
    info = b.sem_batch_info()
    assert sorted(info["orders"]) == [3, 4, 5, 6, 7]
    for h in solo_h:
        for c in chunks:
            h.sem_step(c)
    for hb, hs in zip(batch_h, solo_h):
        assert hb.sem_get_step() == hs.sem_get_step() == sum(chunks)
        ub, us = hb.sem_read_wavefield(), hs.sem_read_wavefield()
        assert np.linalg.norm(us) > 0
        assert np.array_equal(ub, us)
        assert np.array_equal(hb.sem_read_traces(), hs.sem_read_traces())
    b.sem_batch_destroy()
    for h in batch_h + solo_h:
        h.sem_destroy()


def _streamable_shots():
    # DENSE plans only (Hilbert and row-major), orders 3..7, three shots of
    # order 4 of uneven sizes
    return [
        (gen.graded(10, seed=1), 3, "hilbert"),
        (gen.graded(16, seed=2), 4, "hilbert"),
        (gen.unit_square(12), 5, "rowmajor"),
        (gen.graded(7, seed=3), 7, "hilbert"),
        (gen.graded(21, seed=4), 4, "hilbert"),
        (gen.relabel(gen.graded(9, seed=5), seed=6), 6, "hilbert"),
        (gen.graded(5, seed=9), 4, "rowmajor"),
    ]


@pytest.mark.parametrize("prec,mode", [("fp32_kahan", -1), ("fp64", -1), ("fp32_kahan", 2), ("fp64", 1)])
def test_streamed_batch_equals_individual_runs(P, prec, mode):
    """Every shot streamable: in clock-driven 64-step blocks each order runs
    as one streamed launch over the blocks of all its shots (mode -1: the
    automatic choice streams these small classes; 1: every class) or as one
    launch per step (mode 2), across graph replays, a single step, a
    remainder and a second call; shot by shot bitwise the results of
    sem_step on each handle alone."""
    shots = _streamable_shots()
    nmax = 160
    chunks = (70, 1, 64, 5)
    batch_h = [_handle(P, m, p, k, prec, nmax, eb=11) for m, p, k in shots]
    solo_h = [_handle(P, m, p, k, prec, nmax, eb=11) for m, p, k in shots]
    b = P.SEMBatch(batch_h)
    b.sem_batch_set_stream(mode)
    for c in chunks:
        b.sem_batch_step(c)
    assert b.sem_batch_mode() == {"streamed_classes": 0 if mode == 2 else 5, "steps_per_launch": 64}
    with pytest.raises(P.SemError) as ei:
        b.sem_batch_set_stream(0)
    assert ei.value.status == P.SEM_ERR_STATE
    for h in solo_h:
        for c in chunks:
            h.sem_step(c)
    for hb, hs in zip(batch_h, solo_h):
        assert hb.sem_get_step() == hs.sem_get_step() == sum(chunks)
        ub, us = hb.sem_read_wavefield(), hs.sem_read_wavefield()
        assert np.linalg.norm(us) > 0
        assert np.array_equal(ub, us)
        assert np.array_equal(hb.sem_read_traces(), hs.sem_read_traces())
    # the shots stay usable on their own after the batch
    for hb, hs in zip(batch_h, solo_h):
        hb.sem_step(9)
        hs.sem_step(9)
        assert np.array_equal(hb.sem_read_wavefield(), hs.sem_read_wavefield())
    b.sem_batch_destroy()
    for h in batch_h + solo_h:
        h.sem_destroy()


def test_batch_with_a_gather_plan_runs_one_launch_per_step(P):
    shots = _shots()
    hs = [_handle(P, m, p, k, "fp32_kahan", 8, eb=11) for m, p, k in shots]
    b = P.SEMBatch(hs)
    b.sem_batch_step(3)
    assert b.sem_batch_mode() == {"streamed_classes": 0, "steps_per_launch": 1}
    b.sem_batch_destroy()
    for h in hs:
        h.sem_destroy()


def test_batch_autotuned_matches_oracle(P):
    shots = [(gen.graded(24, seed=7), 4, "hilbert"), (gen.graded(12, seed=8), 4, "hilbert"),
             (gen.graded(14, seed=9), 3, "hilbert")]
    n = 80
    hs = [_handle(P, m, p, k, "fp32_kahan", n) for m, p, k in shots]
    b = P.SEMBatch(hs, autotune_steps=20)
    b.sem_batch_step(n)
    info = b.sem_batch_info()
    assert all(e > 0 for e in info["elems_per_block"])
    for (m, p, _), h in zip(shots, hs):
        S = osem.SEM(m["coords"], m["quads"], p, m["vel"], m["rho"])
        _, u_ref, tr_ref = oracle_run(m, p, n, 0.3 * S.cfl_dt(), m["receivers"])
        assert rel_l2(h.sem_read_wavefield(), u_ref) < FP32_TOL
        assert rel_l2(h.sem_read_traces(), tr_ref) < FP32_TOL
    b.sem_batch_destroy()
    for h in hs:
        h.sem_destroy()


def test_batch_rejects_mixed_precision_and_unset_dt(P):
    m = gen.graded(6, seed=1)
    a = _handle(P, m, 4, "hilbert", "fp64", 10)
    c = _handle(P, m, 4, "hilbert", "fp32_kahan", 10)
    with pytest.raises(P.SemError) as ei:
        P.SEMBatch([a, c])
    assert ei.value.status == P.SEM_ERR_STATE
    d = P.SEM(m["coords"], m["quads"], 4, "fp64")
    d.sem_set_model(m["vel"])
    with pytest.raises(P.SemError) as ei:
        P.SEMBatch([a, d])
    assert ei.value.status == P.SEM_ERR_STATE
    for h in (a, c, d):
        h.sem_destroy()
