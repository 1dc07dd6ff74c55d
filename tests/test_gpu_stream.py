"""The streamed time loop (sem_set_stream): several leapfrog steps per launch
of the persistent step kernel, units (step, block) taken in order, each
waiting for the previous step at its block's neighbours. Its arithmetic per
unit is the per-step kernel's, so wavefields and traces must be bitwise those
of one launch per step, on meshes with few and with many blocks, at launch
lengths that split runs at every possible point, in the three leapfrog
storage precisions, across sem_step calls that switch between the two, and
in every order of the units (step order, wavefront orders).
"""
import numpy as np
import pytest

import gen
from tests._gpu_common import FP32_TOL, FP64_TOL, need_gpu, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


def _handle(P, m, p, prec, order, eb, stream, nsteps):
    h = P.SEM(m["coords"], m["quads"], p, prec)
    h.sem_reorder(order, 3)
    h.sem_set_model(m["vel"], m["rho"])
    if eb:
        h.sem_set_tuning(eb, 0)
    h.sem_set_stream(stream)
    h.sem_set_source(m["f0"], m["t0"], m["amp"], *m["src_xy"])
    h.sem_set_receivers(m["receivers"], nsteps)
    h.sem_set_dt(0.3 * h.sem_cfl_dt())
    return h


def _run(P, m, p, prec, order, eb, stream, calls):
    h = _handle(P, m, p, prec, order, eb, stream, sum(calls))
    for n in calls:
        h.sem_step(n)
    out = (h.sem_read_wavefield(), h.sem_read_traces(), h.sem_launch_info()[0])
    h.sem_destroy()
    return out


CASES = [
    # n, p, precision, elements per block, steps per sem_step call
    (40, 4, "fp32_kahan", 0, [61]),
    (40, 4, "fp32_kahan", 16, [1, 2, 40]),
    (64, 4, "fp32_kahan", 32, [100]),
    (33, 3, "fp64", 0, [45]),
    (30, 5, "fp32", 24, [30, 7]),
    (24, 2, "fp32_kahan", 8, [50]),
    (20, 7, "fp64", 12, [19]),
    (18, 8, "fp32_kahan", 6, [23]),
]


@pytest.mark.parametrize("n,p,prec,eb,calls", CASES)
def test_streamed_bitwise_per_step(n, p, prec, eb, calls):
    P = need_gpu()
    m = gen.graded(n, seed=n + p)
    u0, tr0, spl0 = _run(P, m, p, prec, "hilbert", eb, 0, calls)
    assert spl0 == 1
    assert np.isfinite(u0).all() and np.linalg.norm(u0) > 0
    for stream in (1, 3, 256):
        u, tr, spl = _run(P, m, p, prec, "hilbert", eb, stream, calls)
        assert spl == stream  # the Hilbert node numbering gives a DENSE plan
        assert np.array_equal(u, u0), (stream, rel_l2(u, u0))
        assert np.array_equal(tr, tr0), (stream, rel_l2(tr, tr0))


@pytest.mark.parametrize("prec,stream", [("fp32_kahan", 0), ("fp32_kahan", 256), ("fp64", 0), ("fp32", 3)])
def test_calls_and_reads_bitwise(prec, stream):
    """The open nodes of a call's last step stay partial sums until the next
    call or a read: one call, split calls, and split calls with a state read
    between them (which finishes the open nodes first) give the same bits,
    and the read in the middle equals a run that stops there."""
    P = need_gpu()
    m = gen.graded(40, seed=17)
    one = _run(P, m, 4, prec, "hilbert", 16, stream, [41])
    split = _run(P, m, 4, prec, "hilbert", 16, stream, [17, 1, 23])
    h = _handle(P, m, 4, prec, "hilbert", 16, stream, 41)
    h.sem_step(17)
    mid = h.sem_read_wavefield()
    mid_u, mid_prev, mid_step = h.sem_get_state()
    h.sem_step(1)
    h.sem_read_traces()
    h.sem_step(23)
    read_between = (h.sem_read_wavefield(), h.sem_read_traces())
    h.sem_destroy()
    stop = _run(P, m, 4, prec, "hilbert", 16, stream, [17])
    for got in (split, read_between):
        assert np.array_equal(got[0], one[0]) and np.array_equal(got[1], one[1])
    assert mid_step == 17 and np.array_equal(mid, stop[0]) and np.array_equal(mid_u, stop[0])


def test_streamed_against_oracle():
    P = need_gpu()
    m = gen.graded(36, seed=9)
    n = 80
    h = _handle(P, m, 4, "fp64", "hilbert", 16, 256, n)
    dt = 0.3 * h.sem_cfl_dt()
    h.sem_set_dt(dt)
    h.sem_step(n)
    u, tr = h.sem_read_wavefield(), h.sem_read_traces()
    h.sem_destroy()
    _, u_ref, tr_ref = oracle_run(m, 4, n, dt, receivers=m["receivers"])
    assert rel_l2(u, u_ref) < FP64_TOL
    assert rel_l2(tr, tr_ref) < FP64_TOL
    h = _handle(P, m, 4, "fp32_kahan", "hilbert", 16, 256, n)
    h.sem_set_dt(dt)
    h.sem_step(n)
    u32 = h.sem_read_wavefield()
    h.sem_destroy()
    assert rel_l2(u32, u_ref) < FP32_TOL


def test_switching_between_streamed_and_per_step():
    P = need_gpu()
    m = gen.graded(48, seed=21)
    calls = [5, 9, 2, 30]
    u0, tr0, _ = _run(P, m, 4, "fp32_kahan", "hilbert", 32, 0, calls)
    h = _handle(P, m, 4, "fp32_kahan", "hilbert", 32, 4, sum(calls))
    for k, c in enumerate(calls):
        h.sem_set_stream(4 if k % 2 == 0 else 0)
        h.sem_step(c)
    u, tr = h.sem_read_wavefield(), h.sem_read_traces()
    h.sem_destroy()
    assert np.array_equal(u, u0)
    assert np.array_equal(tr, tr0)


@pytest.mark.parametrize("order", ["random", "none"])
def test_gather_plans_launch_per_step(order):
    P = need_gpu()
    m = gen.relabel(gen.graded(30, seed=5), seed=6)
    u0, tr0, _ = _run(P, m, 4, "fp32_kahan", order, 32, 0, [25])
    u, tr, spl = _run(P, m, 4, "fp32_kahan", order, 32, 256, [25])
    if order == "random":
        assert spl == 1
    assert np.array_equal(u, u0)
    assert np.array_equal(tr, tr0)


WAVEFRONT = [(0, 0), (1, 1), (16, 1), (16, 3), (5, 0), (16, 100), (7, 2), (255, 2)]


@pytest.mark.parametrize("prec", ["fp32_kahan", "fp64", "fp32"])
@pytest.mark.parametrize("band,window", WAVEFRONT)
def test_wavefront_orders_bitwise_per_step(prec, band, window):
    """Every wavefront order of the streamed units (sem_set_stream_tiling)
    gives bitwise the result of one launch per step, across launches split
    into whole bands and a step-ordered remainder, and across sem_step calls."""
    P = need_gpu()
    m = gen.graded(64, seed=5)
    calls = [100, 37, 3]
    u0, tr0, _ = _run(P, m, 4, prec, "hilbert", 32, 0, calls)
    h = _handle(P, m, 4, prec, "hilbert", 32, 48, sum(calls))
    h.sem_set_stream_tiling(band, window)
    for n in calls:
        h.sem_step(n)
    u, tr = h.sem_read_wavefield(), h.sem_read_traces()
    got_band, got_window = h.sem_stream_order()
    h.sem_destroy()
    assert np.array_equal(u, u0), rel_l2(u, u0)
    assert np.array_equal(tr, tr0), rel_l2(tr, tr0)
    if 0 < band <= 48:          # a launch of 48 steps holds whole bands
        assert got_band == band
        assert got_window == window or (window == 0 and got_window >= 1)
    else:
        assert got_band == 0


def test_wavefront_order_on_many_blocks():
    """A mesh of many small blocks (long wavefronts): bitwise per step."""
    P = need_gpu()
    m = gen.graded(96, seed=8)
    u0, tr0, _ = _run(P, m, 4, "fp32_kahan", "hilbert", 16, 0, [70])
    for band, window in ((16, 0), (32, 2)):
        h = _handle(P, m, 4, "fp32_kahan", "hilbert", 16, 256, 70)
        h.sem_set_stream_tiling(band, window)
        h.sem_step(70)
        u, tr = h.sem_read_wavefield(), h.sem_read_traces()
        h.sem_destroy()
        assert np.array_equal(u, u0)
        assert np.array_equal(tr, tr0)


@pytest.mark.parametrize("tiling", [(-1, 0), (4, 1)])
def test_withheld_done_flag_ends_in_an_error_not_a_hang(tiling):
    """A unit that never marks its block done (the test hook withholds the
    flag): the next step's units that wait on it give up after their bounded
    wait, the launch stops, the next read-back reports SEM_ERR_TIMEOUT, and both
    the handle (after sem_set_state) and the GPU stay usable."""
    import time

    P = need_gpu()
    m = gen.graded(40, seed=17)
    h = _handle(P, m, 4, "fp32_kahan", "hilbert", 16, 256, 40)
    h.sem_set_stream_tiling(*tiling)
    assert h.sem_launch_info()[0] in (1, 256)
    h.sem_step(1)   # builds the device data
    u0 = h.sem_read_wavefield()
    nblocks = -(-m["quads"].shape[0] // 16)
    h.sem_stream_withhold(4, nblocks // 2)
    t0 = time.perf_counter()
    h.sem_step(12)
    with pytest.raises(P.SemError) as ei:
        h.sem_read_wavefield()
    assert ei.value.status == 5   # SEM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60.0
    # the flag was cleared: a reset state steps normally, and bitwise like
    # one launch per step from the same state
    h.sem_set_state(u0, u0, 0)
    h.sem_step(7)
    u1 = h.sem_read_wavefield()
    h.sem_destroy()
    g = _handle(P, m, 4, "fp32_kahan", "hilbert", 16, 0, 40)
    g.sem_step(1)
    g.sem_set_state(u0, u0, 0)
    g.sem_step(7)
    u2 = g.sem_read_wavefield()
    g.sem_destroy()
    assert np.isfinite(u1).all()
    assert np.array_equal(u1, u2)
