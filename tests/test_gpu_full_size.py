"""Full-size checks of the CUDA path, in the launch configuration bench.py
times (default block size and threads, Hilbert ordering, FP32 with the Kahan
leapfrog), on the two single-GPU workloads:

* graded 512 x 512 quads, order 4 (4,198,401 nodes): the stiffness against
  the FP64 oracle on the whole field, the first steps against the oracle,
  2000 steps of FP32+Kahan against the FP64 GPU path (which the oracle pins at
  every smaller size to 1e-12), and orderings against each other;
* layered 4096 x 1024 quads, order 4 (67,129,345 nodes), 3000 steps: FP32+Kahan
  against FP64 on every 16th node (original order) and on the 256 surface
  traces.

Tolerances are the ones of the other parity tests: relative L2 1e-12 for
FP64 and 1e-5 for FP32 with the compensated leapfrog.
"""
import numpy as np
import pytest

import gen
from oracle import sem as osem
from tests._gpu_common import FP32_TOL, FP64_TOL, fp32_apply_bound, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return need_gpu()


@pytest.fixture(scope="module")
def graded():
    m = gen.graded(512)
    S = osem.SEM(m["coords"], m["quads"], 4, m["vel"], m["rho"], validate=False)
    return m, S


def _handle(P, m, prec, kind="hilbert", nsteps=0, dt=None):
    h = P.SEM(m["coords"], m["quads"], 4, prec)
    h.sem_reorder(kind)
    h.sem_set_model(m["vel"], m["rho"])
    h.sem_set_source(m["f0"], m["t0"], m["amp"], *m["src_xy"])
    if nsteps:
        h.sem_set_receivers(m["receivers"], nsteps)
    h.sem_set_dt(dt if dt is not None else 0.3 * h.sem_cfl_dt())
    return h


def test_graded_stiffness_whole_field(P, graded):
    m, S = graded
    rng = np.random.default_rng(11)
    u = rng.standard_normal(S.n_nodes)
    ref = S.apply_K(u)
    # FP32: the stated 1e-5, or the FP32 forward error bound if tighter
    for prec, tol in (("fp64", FP64_TOL), ("fp32_kahan", min(FP32_TOL, fp32_apply_bound(S, u)))):
        h = _handle(P, m, prec)
        ku = h.sem_apply_stiffness(u)
        h.sem_destroy()
        print(f"graded 512 stiffness {prec}: rel L2 {rel_l2(ku, ref):.2e} (bound {tol:.2e})")
        assert rel_l2(ku, ref) < tol, (prec, rel_l2(ku, ref))


def test_graded_first_steps_match_oracle(P, graded):
    m, S = graded
    dt = 0.3 * S.cfl_dt()
    n = 12
    src = (m["src_xy"][0], m["src_xy"][1], m["f0"], m["t0"], m["amp"])
    # start from a smooth field so that the whole mesh carries signal
    x, y = S.node_xy[:, 0], S.node_xy[:, 1]
    u0 = np.cos(3.0 * np.pi * x) * np.cos(2.0 * np.pi * y)
    um1 = u0 - 0.5 * dt * dt * S.apply_K(u0) / S.M
    u_ref, _, tr_ref = S.run(n, dt, src=src, receivers=m["receivers"], u0=u0, u_prev=um1)
    for prec, tol in (("fp64", FP64_TOL), ("fp32_kahan", FP32_TOL)):
        h = _handle(P, m, prec, nsteps=n, dt=dt)
        h.sem_set_state(u0, um1, 0)
        h.sem_step(n)
        u = h.sem_read_wavefield()
        tr = h.sem_read_traces()
        h.sem_destroy()
        assert rel_l2(u, u_ref) < tol, (prec, rel_l2(u, u_ref))
        assert rel_l2(tr, tr_ref) < tol, (prec, rel_l2(tr, tr_ref))


def test_graded_2000_steps_fp32_kahan_vs_fp64(P, graded):
    m, S = graded
    dt = 0.3 * S.cfl_dt()
    n = 2000
    out = {}
    for prec in ("fp64", "fp32_kahan"):
        h = _handle(P, m, prec, nsteps=n, dt=dt)
        h.sem_step(n)
        out[prec] = (h.sem_read_wavefield(), h.sem_read_traces())
        # 1024 element blocks per step: the time loop is streamed by default
        assert h.sem_launch_info()[0] == 256
        h.sem_destroy()
    u64, tr64 = out["fp64"]
    u32, tr32 = out["fp32_kahan"]
    assert np.isfinite(u64).all() and np.linalg.norm(u64) > 0
    assert rel_l2(u32, u64) < FP32_TOL, rel_l2(u32, u64)
    assert rel_l2(tr32, tr64) < FP32_TOL, rel_l2(tr32, tr64)


def test_graded_orderings_agree(P, graded):
    m, S = graded
    dt = 0.3 * S.cfl_dt()
    us = {}
    for kind in ("hilbert", "rowmajor", "none", "random"):
        h = _handle(P, m, "fp64", kind, dt=dt)
        h.sem_step(150)
        us[kind] = h.sem_read_wavefield()
        h.sem_destroy()
    assert np.linalg.norm(us["hilbert"]) > 0
    for kind in ("rowmajor", "none", "random"):
        assert rel_l2(us[kind], us["hilbert"]) < FP64_TOL, (kind, rel_l2(us[kind], us["hilbert"]))


def test_layered_3000_steps_fp32_kahan_vs_fp64(P):
    m = gen.layered(4096, 1024)
    n = 3000
    out = {}
    for prec in ("fp64", "fp32_kahan"):
        h = _handle(P, m, prec, nsteps=n)
        if prec == "fp64":
            dt = h.sem_cfl_dt() * 0.3
        h.sem_set_dt(dt)
        h.sem_step(n)
        if prec == "fp32_kahan":
            # 16,384 element blocks per step: one launch per step by default
            assert h.sem_launch_info()[0] == 1
        out[prec] = (h.sem_read_wavefield()[::16], h.sem_read_traces())
        h.sem_destroy()
    u64, tr64 = out["fp64"]
    u32, tr32 = out["fp32_kahan"]
    assert np.isfinite(u64).all() and np.linalg.norm(u64) > 0
    assert rel_l2(u32, u64) < FP32_TOL, rel_l2(u32, u64)
    # the wavefront has not reached the surface after 3000 steps (0.33 s at
    # 9.77 m elements): traces are compared against the field's scale
    scale = np.abs(u64).max()
    assert np.abs(tr32 - tr64).max() <= FP32_TOL * scale
