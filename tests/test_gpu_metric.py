"""The per-point geometric factors G_q = w_q |J_q| / rho_e J_q^-1 J_q^-T
(Section 4.2, Eq. deriv_u with the quadrature of Eq. numerical_integ) as the
step kernels use them, against the FP64 oracle; and the FP32 path that
streams G_q computed in FP64 and rounded once (SEM_METRIC_STORED) against
the oracle and against the default path, which forms G_q in FP32 from the
FP64-derived bilinear map at every point of every step."""
import numpy as np
import pytest

import gen
from oracle import sem as osem
from tests._gpu_common import FP32_TOL, FP64_TOL, U32, fp32_apply_bound, gpu_run, need_gpu, oracle_run, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    return need_gpu()


def _oracle_metric(S):
    """(E, P, 3): gxx, gxy, gyy of the oracle's FP64 metric."""
    G = S.G
    return np.stack([G[..., 0, 0], G[..., 0, 1], G[..., 1, 1]], axis=-1)


def _point_error(g, ref):
    """Largest error of a point's three factors over the point's scale
    |gxx| + |gyy| (gxy alone can be near zero on near-rectangular elements),
    and the relative L2 error over all factors."""
    scale = np.abs(ref[..., 0]) + np.abs(ref[..., 2])
    return float((np.abs(g - ref).max(axis=-1) / scale).max()), rel_l2(g, ref)


def _handle(P, m, p, prec, metric=None, kind="hilbert"):
    h = P.SEM(m["coords"], m["quads"], p, prec)
    if metric:
        h.sem_set_metric(metric)
    h.sem_reorder(kind)
    h.sem_set_model(m["vel"], m["rho"])
    return h


@pytest.mark.parametrize("p", [2, 4, 7])
def test_fp64_metric_matches_oracle(P, p):
    m = gen.relabel(gen.graded(12, seed=5), seed=6)
    S = osem.SEM(m["coords"], m["quads"], p, m["vel"], m["rho"])
    h = _handle(P, m, p, "fp64", kind="random")
    mx, l2 = _point_error(h.sem_read_metric(), _oracle_metric(S))
    h.sem_destroy()
    assert mx <= 1e-14 and l2 <= 1e-14, (mx, l2)


def test_fp64_metric_matches_oracle_layered(P):
    """Layered model in metres: corner coordinates up to 4e4 m, elements of
    156 m here (9.8 m at 4096 x 1024), so each Jacobian entry, a difference of
    corner coordinates, carries about 4e4 / 156 = 256 FP64 roundoffs of the
    entry (4e3 at full size), in the oracle and on the GPU alike, which
    difference in another order: agreement to 1e-11 of the point's scale."""
    m = gen.layered(256, 64)
    S = osem.SEM(m["coords"], m["quads"], 4, m["vel"], m["rho"], validate=False)
    h = _handle(P, m, 4, "fp64")
    mx, l2 = _point_error(h.sem_read_metric(), _oracle_metric(S))
    h.sem_destroy()
    print(f"FP64 metric (layered): max {mx:.2e}, rel L2 {l2:.2e}")
    assert mx <= 1e-11 and l2 <= 1e-12, (mx, l2)


@pytest.mark.parametrize("make", ["graded", "layered"])
def test_fp32_formed_metric_error(P, make):
    """FP32 metric formed in the kernel from the bilinear map. Bound: the
    eight map coefficients are rounded to FP32 once (1 u each), the Jacobian
    entries take one FMA each, the determinant one FMA and one product over
    entries of similar size on these mildly distorted elements, __fdividef
    is within 2 ulp, the factors take two or three more roundings: about a
    dozen units of FP32 roundoff relative to the point's scale; 32 u32 is
    asserted, and the measured values are printed."""
    m = gen.graded(48, seed=9) if make == "graded" else gen.layered(256, 64)
    S = osem.SEM(m["coords"], m["quads"], 4, m["vel"], m["rho"], validate=False)
    h = _handle(P, m, 4, "fp32_kahan")
    mx, l2 = _point_error(h.sem_read_metric(), _oracle_metric(S))
    h.sem_destroy()
    print(f"FP32 metric formed from the bilinear map ({make}): max {mx:.2e} ({mx / U32:.1f} u32), rel L2 {l2:.2e}")
    assert mx <= 32 * U32, mx


@pytest.mark.parametrize("make", ["graded", "layered"])
def test_fp32_stored_metric_is_the_fp64_metric_rounded_once(P, make):
    m = gen.graded(48, seed=9) if make == "graded" else gen.layered(256, 64)
    S = osem.SEM(m["coords"], m["quads"], 4, m["vel"], m["rho"], validate=False)
    ref = _oracle_metric(S)
    h = _handle(P, m, 4, "fp32_kahan", "stored")
    g = h.sem_read_metric()
    h.sem_destroy()
    # each factor is the FP64 value rounded to nearest FP32: within half an
    # FP32 ulp of the oracle's value, plus the difference of the two FP64
    # evaluations relative to the point's scale (the off-diagonal factor of a
    # rectangular element is rounding noise around zero in both; on the
    # layered model the Jacobian comes from differences of corner
    # coordinates of 4e4 m across 156 m elements, 256 times the FP64
    # roundoff: see test_fp64_metric_matches_oracle_layered)
    scale = (np.abs(ref[..., 0]) + np.abs(ref[..., 2]))[..., None]
    fp64_gap = 1e-14 if make == "graded" else 1e-11
    assert np.all(np.abs(g - ref) <= U32 * np.abs(ref) * (1 + 1e-9) + fp64_gap * scale)
    mx, l2 = _point_error(g, ref)
    print(f"FP32 stored metric ({make}): max {mx:.2e} ({mx / U32:.2f} u32), rel L2 {l2:.2e}")


@pytest.mark.parametrize("p", [1, 3, 4, 6, 8])
@pytest.mark.parametrize("kind", ["hilbert", "random", "none"])
def test_stored_metric_stiffness(P, p, kind):
    m = gen.relabel(gen.graded(11, seed=8), seed=3)
    rng = np.random.default_rng(p)
    rho = 0.5 + rng.random(m["quads"].shape[0])
    S = osem.SEM(m["coords"], m["quads"], p, m["vel"], rho)
    xy = S.node_xy
    h = P.SEM(m["coords"], m["quads"], p, "fp32_kahan")
    h.sem_set_metric("stored")
    h.sem_reorder(kind, 99)
    h.sem_set_model(m["vel"], rho)
    h.sem_set_tuning(7)
    for u in (rng.standard_normal(S.n_nodes), np.sin(3 * xy[:, 0]) * np.cos(2 * xy[:, 1])):
        err = rel_l2(h.sem_apply_stiffness(u), S.apply_K(u))
        assert err < fp32_apply_bound(S, u), (err, fp32_apply_bound(S, u))
    h.sem_destroy()


def test_stored_metric_wavefield_and_streaming(P):
    """Homogeneous 32 x 32, order 4, 400 steps: the stored-metric FP32 path
    within 1e-5 of the oracle like the default path; on a graded mesh the
    streamed launch equals one launch per step bit for bit."""
    m = gen.unit_square(32)
    n = 400
    S, u_ref, tr_ref = oracle_run(m, 4, n, 0.3 * osem.SEM(m["coords"], m["quads"], 4, 1.0, 1.0).cfl_dt(),
                                  m["receivers"])
    dt = 0.3 * S.cfl_dt()
    errs = {}
    for metric in ("bilinear", "stored"):
        h = _handle(P, m, 4, "fp32_kahan", metric)
        h.sem_set_source(m["f0"], m["t0"], m["amp"], *m["src_xy"])
        h.sem_set_receivers(m["receivers"], n)
        h.sem_set_dt(dt)
        h.sem_step(n)
        errs[metric] = (rel_l2(h.sem_read_wavefield(), u_ref), rel_l2(h.sem_read_traces(), tr_ref))
        h.sem_destroy()
    print("homogeneous 32x32 400 steps, rel L2 vs oracle (wavefield, traces):", errs)
    for e in errs.values():
        assert e[0] < FP32_TOL and e[1] < FP32_TOL
    g = gen.graded(64, seed=2)
    out = []
    for stream in (0, 32):   # 16 blocks: less than one wave, so streaming is asked for explicitly
        h = _handle(P, g, 4, "fp32_kahan", "stored")
        h.sem_set_stream(stream)
        h.sem_set_source(g["f0"], g["t0"], g["amp"], *g["src_xy"])
        h.sem_set_receivers(g["receivers"], 60)
        h.sem_set_dt(0.3 * h.sem_cfl_dt())
        h.sem_step(60)
        out.append((h.sem_read_wavefield(), h.sem_read_traces(), h.sem_launch_info()[0]))
        h.sem_destroy()
    assert out[0][2] == 1 and out[1][2] == 32
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_stored_metric_refused_by_batches(P):
    m = gen.unit_square(4)
    hs = []
    for metric in ("bilinear", "stored"):
        h = _handle(P, m, 3, "fp32_kahan", metric)
        h.sem_set_dt(0.3 * h.sem_cfl_dt())
        hs.append(h)
    with pytest.raises(P.SemError) as ei:
        P.SEMBatch(hs, autotune_steps=0)
    assert ei.value.status == P.SEM_ERR_UNSUPPORTED
    for h in hs:
        h.sem_destroy()
