"""The paper's own scheme on the GPU: the first-order pressure/velocity
system advanced by Heun's predictor-corrector (SEM_SCHEME_HEUN), against the
FP64 oracle's `run_heun` on the same inputs. Tolerances: relative L2 1e-12
(FP64) and 1e-5 (FP32)."""
import numpy as np
import pytest

import gen
from oracle import sem as osem
from tests._gpu_common import FP32_TOL, FP64_TOL, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return need_gpu()


def _run(P, m, p, prec, kind, n, dt, rec, eb=0, chunks=None, state=None):
    h = P.SEM(m["coords"], m["quads"], p, prec)
    h.sem_set_scheme("heun")
    h.sem_reorder(kind, 9)
    h.sem_set_model(m["vel"], m["rho"])
    if eb:
        h.sem_set_tuning(eb)
    if state is None:
        h.sem_set_source(m["f0"], m["t0"], m["amp"], *m["src_xy"])
    h.sem_set_receivers(rec, n)
    h.sem_set_dt(dt)
    if state is not None:
        h.sem_set_state(state, np.zeros_like(state), 0)
    for c in (chunks or [n]):
        h.sem_step(c)
    out = h.sem_read_wavefield(), h.sem_read_traces()
    h.sem_destroy()
    return out


@pytest.mark.parametrize("kind", ["hilbert", "random", "none"])
@pytest.mark.parametrize("p", [3, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_heun_matches_oracle(P, kind, p, prec):
    m = gen.relabel(gen.graded(10, seed=p), seed=4) if kind == "none" else gen.graded(10, seed=p)
    S = osem.SEM(m["coords"], m["quads"], p, m["vel"], m["rho"])
    dt = 0.1 * S.cfl_dt()
    n = 200
    rec = np.array([[0.5, 0.5], [0.1, 0.9], [0.93, 0.2], [0.4, 0.61]])
    src = (m["src_xy"][0], m["src_xy"][1], m["f0"], m["t0"], m["amp"])
    u_ref, _, tr_ref = S.run_heun(n, dt, src=src, receivers=rec)
    u, tr = _run(P, m, p, prec, kind, n, dt, rec, eb=13)
    tol = FP64_TOL if prec == "fp64" else FP32_TOL
    assert np.linalg.norm(u_ref) > 0
    assert rel_l2(u, u_ref) < tol, rel_l2(u, u_ref)
    assert rel_l2(tr, tr_ref) < tol, rel_l2(tr, tr_ref)


def test_heun_standing_mode_from_state(P):
    m = gen.unit_square(3)
    p = 6
    S = osem.SEM(m["coords"], m["quads"], p, 1.0, 1.0)
    x, y = S.node_xy[:, 0], S.node_xy[:, 1]
    u0 = np.cos(np.pi * x) * np.cos(np.pi * y)
    dt = 0.05 * S.cfl_dt()
    n = 400
    u_ref, _, _ = S.run_heun(n, dt, U0=u0)
    mm = dict(m, vel=np.ones(9), rho=np.ones(9))
    for prec, tol in (("fp64", FP64_TOL), ("fp32", FP32_TOL)):
        u, _ = _run(P, mm, p, prec, "hilbert", n, dt, np.array([[0.5, 0.5]]), state=u0)
        assert rel_l2(u, u_ref) < tol
        assert rel_l2(u, u0 * np.cos(np.pi * np.sqrt(2) * n * dt)) < 1e-4


def test_heun_split_runs_bitwise(P):
    m = gen.graded(12, seed=3)
    S = osem.SEM(m["coords"], m["quads"], 4, m["vel"], m["rho"])
    dt = 0.1 * S.cfl_dt()
    rec = np.array([[0.5, 0.5], [0.2, 0.8]])
    a = _run(P, m, 4, "fp32", "hilbert", 50, dt, rec, eb=9)
    b = _run(P, m, 4, "fp32", "hilbert", 50, dt, rec, eb=9, chunks=[20, 1, 29])
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_heun_repeated_runs_bitwise(P):
    # small blocks: many owned ranges whose 16-byte-aligned ends reach into a
    # neighbouring block's nodes; every run must give the same bits (the
    # predictor stores its rate only at the block's own closed nodes)
    m = gen.graded(16, seed=5)
    S = osem.SEM(m["coords"], m["quads"], 4, m["vel"], m["rho"])
    dt = 0.1 * S.cfl_dt()
    rec = np.array([[0.3, 0.7]])
    runs = [_run(P, m, 4, "fp32", "hilbert", 120, dt, rec, eb=5) for _ in range(3)]
    for u, tr in runs[1:]:
        assert np.array_equal(u, runs[0][0]) and np.array_equal(tr, runs[0][1])


def test_heun_rejects_kahan_and_adjoint(P):
    m = gen.unit_square(3)
    h = P.SEM(m["coords"], m["quads"], 3, "fp32_kahan")
    with pytest.raises(P.SemError) as ei:
        h.sem_set_scheme("heun")
    assert ei.value.status == P.SEM_ERR_UNSUPPORTED
    h.sem_destroy()
