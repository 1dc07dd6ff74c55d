"""Discrete adjoint on the GPU (sem_misfit_gradient, torch.autograd wrapper):
against the FP64 oracle's adjoint, invariant under the checkpoint spacing,
and against central finite differences of the GPU misfit on 20 elements of
the 256 x 256 order-4 layered case (3000 steps)."""
import numpy as np
import pytest

import gen
from oracle import sem as osem
from tests._gpu_common import need_gpu, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return need_gpu()


def _small_case(seed=11, n=8, p=3):
    m = gen.graded(n, seed=seed)
    vel_true = np.asarray(m["vel"], dtype=np.float64)
    vel = vel_true * (1.0 + 0.05 * np.sin(np.arange(vel_true.size)))
    rec = np.array([[0.1, 0.9], [0.8, 0.85], [0.5, 0.2], [0.95, 0.4], [0.8, 0.85]])   # one node twice
    src = (m["src_xy"][0], m["src_xy"][1], m["f0"], m["t0"], m["amp"])
    S_true = osem.SEM(m["coords"], m["quads"], p, vel_true, m["rho"])
    dt = 0.3 * S_true.cfl_dt()
    return m, p, vel, rec, src, dt, S_true


def _handle(P, m, p, vel, rec, dt, nsteps, prec="fp64", kind="hilbert", eb=0):
    h = P.SEM(m["coords"], m["quads"], p, prec)
    h.sem_reorder(kind, 5)
    h.sem_set_model(vel, m["rho"])
    if eb:
        h.sem_set_tuning(eb)
    h.sem_set_source(m["f0"], m["t0"], m["amp"], *m["src_xy"])
    h.sem_set_receivers(rec, nsteps)
    h.sem_set_dt(dt)
    return h


@pytest.mark.parametrize("kind", ["hilbert", "random"])
def test_gradient_matches_oracle_adjoint(P, kind):
    m, p, vel, rec, src, dt, S_true = _small_case()
    n = 150
    _, _, d_obs = S_true.run(n, dt, src=src, receivers=rec)
    S = osem.SEM(m["coords"], m["quads"], p, vel, m["rho"])
    J_ref, g_ref, _ = S.misfit_gradient(n, dt, src, rec, d_obs)
    h = _handle(P, m, p, vel, rec, dt, n, kind=kind, eb=7)
    J, g = h.sem_misfit_gradient(d_obs, n)
    assert abs(J - J_ref) <= 1e-12 * J_ref
    assert rel_l2(g, g_ref) < 1e-10, rel_l2(g, g_ref)
    # the handle is left at the end of the forward run
    assert h.sem_get_step() == n
    u_ref, _, _ = S.run(n, dt, src=src, receivers=rec)
    assert rel_l2(h.sem_read_wavefield(), u_ref) < 1e-12
    h.sem_destroy()


def test_gradient_independent_of_checkpoint_spacing(P):
    m, p, vel, rec, src, dt, S_true = _small_case(seed=4)
    n = 97
    _, _, d_obs = S_true.run(n, dt, src=src, receivers=rec)
    h = _handle(P, m, p, vel, rec, dt, n)
    ref = h.sem_misfit_gradient(d_obs, n, 0)
    for kc in (1, 7, 96, 97):
        J, g = h.sem_misfit_gradient(d_obs, n, kc)
        assert J == ref[0] and np.array_equal(g, ref[1]), kc
    h.sem_destroy()


def test_fp32_gradient_against_fp64(P):
    m, p, vel, rec, src, dt, S_true = _small_case(seed=6, n=10, p=4)
    n = 200
    _, _, d_obs = S_true.run(n, dt, src=src, receivers=rec)
    g = {}
    for prec in ("fp64", "fp32"):
        h = _handle(P, m, p, vel, rec, dt, n, prec=prec)
        g[prec] = h.sem_misfit_gradient(d_obs, n)[1]
        h.sem_destroy()
    assert rel_l2(g["fp32"], g["fp64"]) < 1e-3, rel_l2(g["fp32"], g["fp64"])


def test_set_model_after_build_matches_fresh_handle(P):
    m, p, vel, rec, src, dt, S_true = _small_case(seed=8)
    n = 60
    _, _, d_obs = S_true.run(n, dt, src=src, receivers=rec)
    h = _handle(P, m, p, np.asarray(m["vel"]), rec, dt, n)
    h.sem_misfit_gradient(d_obs, n)
    h.sem_set_model(vel, m["rho"])                  # in place, plan kept
    J1, g1 = h.sem_misfit_gradient(d_obs, n)
    f = _handle(P, m, p, vel, rec, dt, n)
    J2, g2 = f.sem_misfit_gradient(d_obs, n)
    assert J1 == J2 and np.array_equal(g1, g2)
    for x in (h, f):
        x.sem_destroy()


def test_adjoint_case_central_differences_and_autograd(P):
    """256 x 256 quads, order 4, layered true model vs the smoothed start
    model, 3000 steps, all 8 shots: the summed adjoint gradient against
    central finite differences of the summed misfit on 20 seeded random
    elements (among those whose gradient is at least 1 % of the largest), and
    the torch.autograd wrapper against sem_misfit_gradient."""
    import torch
    from paper_2104_08416_gb300.autograd import Survey, trace_misfit
    c = gen.adjoint_case()
    m = c["mesh"]
    n = 3000
    h = P.SEM(m["coords"], m["quads"], 4, "fp64")
    h.sem_reorder("hilbert")
    h.sem_set_model(c["vel_true"], m["rho"])
    dt = 0.3 * h.sem_cfl_dt()
    h.sem_destroy()
    sources = c["sources"]
    assert len(sources) == 8
    d_obs = []
    for sx, sy in sources:
        t = P.SEM(m["coords"], m["quads"], 4, "fp64")
        t.sem_reorder("hilbert")
        t.sem_set_model(c["vel_true"], m["rho"])
        t.sem_set_source(c["f0"], c["t0"], c["amp"], sx, sy)
        t.sem_set_receivers(c["receivers"], n)
        t.sem_set_dt(dt)
        t.sem_step(n)
        d_obs.append(t.sem_read_traces())
        t.sem_destroy()
    sv = Survey(m["coords"], m["quads"], 4, sources, c["receivers"], d_obs, n, dt, c["f0"], c["t0"], c["amp"],
                rho=m["rho"])
    v0 = np.asarray(c["vel_start"], dtype=np.float64)
    J, g = sv.misfit_and_gradient(v0)
    assert J > 0 and np.isfinite(g).all()
    rng = np.random.default_rng(2104)
    cand = np.flatnonzero(np.abs(g) >= 0.01 * np.abs(g).max())
    pick = rng.choice(cand, size=20, replace=False)
    for e in pick:
        hstep = 1e-4 * v0[e]
        vp, vm = v0.copy(), v0.copy()
        vp[e] += hstep
        vm[e] -= hstep
        Jp = sv.misfit_and_gradient(vp, gradient=False)[0]
        Jm = sv.misfit_and_gradient(vm, gradient=False)[0]
        fd = (Jp - Jm) / (2 * hstep)
        assert abs(fd - g[e]) <= 1e-4 * np.abs(g).max() + 1e-3 * abs(g[e]), (e, fd, g[e])
    vel = torch.tensor(v0, requires_grad=True)
    Jt = trace_misfit(vel, sv)
    Jt.backward()
    assert abs(float(Jt) - J) <= 1e-12 * J
    assert np.array_equal(vel.grad.numpy(), g)
    sv.close()
