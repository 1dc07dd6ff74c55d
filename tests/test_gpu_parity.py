"""CUDA path vs the FP64 oracle, through the C ABI (needs a GPU).

Tolerances: relative L2 1e-12 for FP64 and 1e-5 for FP32 with the Kahan
leapfrog; integer/permutation results bit-exact."""
import numpy as np
import pytest

import gen
from oracle import mesh, ordering, sem as osem
from tests._gpu_common import FP32_TOL, FP64_TOL, fp32_apply_bound, gpu_run, need_gpu, oracle_run, rel_l2

pytestmark = pytest.mark.gpu
ORDERINGS = ["none", "rowmajor", "random", "hilbert", "connectivity", "distance", "hilbert_wide"]


@pytest.fixture(scope="module")
def P():
    return need_gpu()


def _small_graded(nx=13, ny=11, seed=21):
    # non-square, ragged block tail: 143 elements
    m = gen.graded(max(nx, ny), seed=seed)
    return m


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
def test_mass_fp64(P, p):
    m = gen.relabel(gen.graded(9, seed=4), seed=2)
    S = osem.SEM(m["coords"], m["quads"], p, m["vel"], m["rho"])
    for kind in ("hilbert", "random"):
        h = P.SEM(m["coords"], m["quads"], p, "fp64")
        h.sem_reorder(kind)
        h.sem_set_model(m["vel"], m["rho"])
        M = h.sem_read_mass()
        h.sem_destroy()
        assert rel_l2(M, S.M) < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_stiffness_apply(P, p, prec):
    m = gen.relabel(gen.graded(11, seed=8), seed=3)
    rng = np.random.default_rng(p)
    rho = 0.5 + rng.random(m["quads"].shape[0])
    S = osem.SEM(m["coords"], m["quads"], p, m["vel"], rho)
    xy = S.node_xy
    fields = [rng.standard_normal(S.n_nodes), np.sin(3 * xy[:, 0]) * np.cos(2 * xy[:, 1])]
    refs = [S.apply_K(u) for u in fields]
    # FP64: the stated 1e-12. FP32: the forward error bound of the FP32
    # evaluation (fp32_apply_bound), and the stated 1e-5 on white noise,
    # where the operator is well conditioned
    tols = ([FP64_TOL, FP64_TOL] if prec == "fp64" else
            [min(FP32_TOL, fp32_apply_bound(S, fields[0])), fp32_apply_bound(S, fields[1])])
    worst = [0.0, 0.0]
    for kind in ORDERINGS:
        h = P.SEM(m["coords"], m["quads"], p, prec)
        h.sem_reorder(kind, 99)
        h.sem_set_model(m["vel"], rho)
        h.sem_set_tuning(7)          # several blocks, ragged tail (121 elements)
        for f, (u, ref) in enumerate(zip(fields, refs)):
            ku = h.sem_apply_stiffness(u)
            err = rel_l2(ku, ref)
            worst[f] = max(worst[f], err)
            assert err < tols[f], (kind, f, err, tols[f])
        # constants are in the kernel of K
        k1 = h.sem_apply_stiffness(np.ones(S.n_nodes))
        assert np.abs(k1).max() < (1e-12 if prec == "fp64" else 1e-4) * np.abs(refs[0]).max()
        h.sem_destroy()
    print(f"stiffness p={p} {prec}: worst rel L2 white noise {worst[0]:.2e} (bound {tols[0]:.2e}), "
          f"smooth {worst[1]:.2e} (bound {tols[1]:.2e})")


@pytest.mark.parametrize("kind", ORDERINGS)
@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_homogeneous_32x32_400_steps(P, kind, prec):
    """Unit square, 32 x 32 quads, order 4 (16,641 nodes), c = rho = 1, Ricker
    f0 = 10 at the centre, dt = 0.3 CFL, 400 steps."""
    m = gen.unit_square(32)
    rec = m["receivers"]
    S = osem.SEM(m["coords"], m["quads"], 4, m["vel"], m["rho"])
    dt = 0.3 * S.cfl_dt()
    _, u_ref, tr_ref = oracle_run(m, 4, 400, dt, rec)
    u, tr, _ = gpu_run(P, m, 4, prec, kind, 400, dt, rec)
    tol = FP64_TOL if prec == "fp64" else FP32_TOL
    assert rel_l2(u, u_ref) < tol, rel_l2(u, u_ref)
    assert rel_l2(tr, tr_ref) < tol, rel_l2(tr, tr_ref)


@pytest.mark.parametrize("kind", ORDERINGS)
@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_graded_heterogeneous(P, kind, prec):
    """Graded (8x), perturbed (20%), c ~ U[1,3] mesh; 40 x 40 quads, order 4,
    300 steps at 0.3 CFL; several blocks and a ragged tail."""
    m = gen.graded(40, seed=77)
    rec = m["receivers"]
    S = osem.SEM(m["coords"], m["quads"], 4, m["vel"], m["rho"])
    dt = 0.3 * S.cfl_dt()
    _, u_ref, tr_ref = oracle_run(m, 4, 300, dt, rec)
    u, tr, _ = gpu_run(P, m, 4, prec, kind, 300, dt, rec, eb=37)
    tol = FP64_TOL if prec == "fp64" else FP32_TOL
    assert rel_l2(u, u_ref) < tol, rel_l2(u, u_ref)
    assert rel_l2(tr, tr_ref) < tol, rel_l2(tr, tr_ref)


@pytest.mark.parametrize("p", [1, 2, 3, 5, 6, 7, 8])
def test_other_orders_fp64(P, p):
    m = gen.relabel(gen.graded(10, seed=p), seed=p)
    S = osem.SEM(m["coords"], m["quads"], p, m["vel"], m["rho"])
    dt = 0.3 * S.cfl_dt()
    rec = np.array([[0.2, 0.9], [0.7, 0.3]])
    _, u_ref, tr_ref = oracle_run(m, p, 120, dt, rec)
    for kind in ("hilbert", "random"):
        u, tr, _ = gpu_run(P, m, p, "fp64", kind, 120, dt, rec, eb=5)
        assert rel_l2(u, u_ref) < FP64_TOL
        assert rel_l2(tr, tr_ref) < FP64_TOL
    u, tr, _ = gpu_run(P, m, p, "fp32_kahan", "hilbert", 120, dt, rec)
    assert rel_l2(u, u_ref) < FP32_TOL


def test_bitwise_reproducible(P):
    m = gen.graded(24, seed=5)
    S = osem.SEM(m["coords"], m["quads"], 4, m["vel"], m["rho"])
    dt = 0.3 * S.cfl_dt()
    a, _, _ = gpu_run(P, m, 4, "fp32_kahan", "hilbert", 200, dt)
    b, _, _ = gpu_run(P, m, 4, "fp32_kahan", "hilbert", 200, dt)
    assert np.array_equal(a, b)


def test_orderings_agree_on_gpu(P):
    m = gen.graded(30, seed=9)
    S = osem.SEM(m["coords"], m["quads"], 4, m["vel"], m["rho"])
    dt = 0.3 * S.cfl_dt()
    us = [gpu_run(P, m, 4, "fp64", k, 150, dt)[0] for k in ORDERINGS]
    for u in us[1:]:
        assert rel_l2(u, us[0]) < FP64_TOL


def test_standing_mode_from_state(P):
    """Initial-value run through sem_set_state: the Neumann standing mode
    cos(pi x) cos(pi y) cos(pi sqrt2 t) at order 6, matched to the oracle and
    close to the closed form."""
    m = gen.unit_square(3)
    p = 6
    S = osem.SEM(m["coords"], m["quads"], p, 1.0, 1.0)
    x, y = S.node_xy[:, 0], S.node_xy[:, 1]
    u0 = np.cos(np.pi * x) * np.cos(np.pi * y)
    dt = 0.1 * S.cfl_dt()
    um1 = u0 - 0.5 * dt * dt * S.apply_K(u0) / S.M
    n = 500
    u_ref, _, _ = S.run(n, dt, u0=u0, u_prev=um1)
    exact = u0 * np.cos(np.pi * np.sqrt(2) * n * dt)
    for prec, tol in (("fp64", FP64_TOL), ("fp32_kahan", FP32_TOL)):
        h = P.SEM(m["coords"], m["quads"], p, prec)
        h.sem_reorder("hilbert")
        h.sem_set_model(np.ones(9))
        h.sem_set_dt(dt)
        h.sem_set_state(u0, um1, 0)
        a, b, st = h.sem_get_state()
        assert st == 0 and rel_l2(a, u0) < (1e-15 if prec == "fp64" else 1e-7)
        h.sem_step(n)
        u = h.sem_read_wavefield()
        h.sem_destroy()
        assert rel_l2(u, u_ref) < tol
        assert rel_l2(u, exact) < 1e-4


def test_state_roundtrip_and_errors(P):
    m = gen.unit_square(4)
    h = P.SEM(m["coords"], m["quads"], 3, "fp64")
    h.sem_set_model(m["vel"])
    h.sem_set_dt(1e-3)
    h.sem_set_receivers(np.array([[0.5, 0.5]]), 5)
    h.sem_step(5)
    with pytest.raises(P.SemError) as ei:
        h.sem_step(1)                         # beyond the receivers' max_steps
    assert ei.value.status == P.SEM_ERR_INVALID_ARG
    with pytest.raises(P.SemError) as ei:
        h.sem_reorder("hilbert")              # after the device data was built
    assert ei.value.status == P.SEM_ERR_STATE
    u, up, st = h.sem_get_state()
    assert st == 5 and np.all(u == 0)         # no source: the field stays zero
    h.sem_destroy()


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan", "fp32"])
@pytest.mark.parametrize("kind", ["hilbert", "random"])
def test_split_runs_bitwise(P, prec, kind):
    """sem_step(60) equals sem_step(1), (2), (7), (50) in a row, bit for bit:
    runs that stop and restart finish the shared nodes with the same
    arithmetic as runs that carry them from step to step."""
    m = gen.graded(20, seed=13)
    S = osem.SEM(m["coords"], m["quads"], 4, m["vel"], m["rho"])
    dt = 0.3 * S.cfl_dt()
    rec = np.array([[0.5, 0.5], [0.1, 0.9], [0.9, 0.2], [0.42, 0.42]])
    outs = []
    for chunks in ([60], [1, 2, 7, 50]):
        h = P.SEM(m["coords"], m["quads"], 4, prec)
        h.sem_reorder(kind, 7)
        h.sem_set_model(m["vel"], m["rho"])
        h.sem_set_tuning(9)
        h.sem_set_source(m["f0"], m["t0"], m["amp"], *m["src_xy"])
        h.sem_set_receivers(rec, 60)
        h.sem_set_dt(dt)
        for c in chunks:
            h.sem_step(c)
        outs.append((h.sem_read_wavefield(), h.sem_read_traces(), h.sem_get_state()[1]))
        h.sem_destroy()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_plain_fp32_three_level(P):
    """SEM_FP32 (no compensation) on the homogeneous 32 x 32 case, 400 steps:
    within 1e-4 of the FP64 oracle (the compensated mode is the one held to
    1e-5)."""
    m = gen.unit_square(32)
    S = osem.SEM(m["coords"], m["quads"], 4, m["vel"], m["rho"])
    dt = 0.3 * S.cfl_dt()
    _, u_ref, tr_ref = oracle_run(m, 4, 400, dt, m["receivers"])
    u, tr, _ = gpu_run(P, m, 4, "fp32", "hilbert", 400, dt, m["receivers"])
    assert rel_l2(u, u_ref) < 1e-4, rel_l2(u, u_ref)
    assert rel_l2(tr, tr_ref) < 1e-4


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_degenerate_meshes(P, prec):
    """One element; a 1 x 9 strip; one element per block; zero steps."""
    tol = FP64_TOL if prec == "fp64" else FP32_TOL
    one = dict(gen.unit_square(1))
    strip = gen.layered(9, 1, width=9.0, depth=1.0, n_receivers=3)
    strip["src_xy"], strip["f0"], strip["t0"] = (4.5, 0.5), 2.0, 0.6
    for m, p, eb in ((one, 4, 0), (one, 1, 1), (strip, 3, 1), (strip, 5, 2)):
        S = osem.SEM(m["coords"], m["quads"], p, m["vel"], m["rho"])
        dt = 0.3 * S.cfl_dt()
        rec = np.asarray(m["receivers"])
        _, u_ref, tr_ref = oracle_run(m, p, 40, dt, rec)
        u, tr, _ = gpu_run(P, m, p, prec, "hilbert", 40, dt, rec, eb=eb)
        assert rel_l2(u, u_ref) < tol and rel_l2(tr, tr_ref) < tol
    h = P.SEM(one["coords"], one["quads"], 2, prec)
    h.sem_set_model(one["vel"])
    h.sem_set_dt(1e-3)
    h.sem_step(0)
    assert h.sem_get_step() == 0 and np.all(h.sem_read_wavefield() == 0)
    h.sem_destroy()
