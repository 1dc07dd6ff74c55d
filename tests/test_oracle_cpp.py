"""Pins of the C/OpenMP oracle (oracle/sem_ref.c through oracle/cpp.py):
against the NumPy oracle (mass, K u, leapfrog with source and receivers), and
against what the mathematics fixes on its own (K 1 = 0, the mass summing to
the area, thread-count invariance of the fixed-order sums)."""
import numpy as np
import pytest

import gen
from oracle import cpp, sem


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.fixture(scope="module", autouse=True)
def _built():
    cpp.build()


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
def test_mass_and_stiffness_match_numpy_oracle(p):
    m = gen.relabel(gen.graded(7, seed=p), seed=p + 1)
    rho = 0.5 + np.random.default_rng(p).random(m["quads"].shape[0])
    S = sem.SEM(m["coords"], m["quads"], p, m["vel"], rho)
    Sc = cpp.SEMC(m["coords"], m["quads"], p, m["vel"], rho, threads=3)
    assert Sc.n_nodes == S.n_nodes
    assert _rel(Sc.M, S.M) <= 1e-14
    rng = np.random.default_rng(10 + p)
    noise = rng.standard_normal(S.n_nodes)
    assert _rel(Sc.apply_K(noise), S.apply_K(noise)) <= 1e-13
    # a smooth field is nearly in the kernel of K: both oracles round each
    # term at 2^-53 of the term, so they may differ by a few units of the sum
    # of |terms|, which is far larger than |K u| at high order
    u = np.sin(3 * S.node_xy[:, 0]) * np.cos(2 * S.node_xy[:, 1])
    a = np.bincount(S.conn.ravel(), weights=np.einsum("eab,eb->ea", np.abs(S.Ke), np.abs(u[S.conn])).ravel(),
                    minlength=S.n_nodes)
    ref = S.apply_K(u)
    assert _rel(Sc.apply_K(u), ref) <= max(1e-13, 64 * 2.0 ** -53 * np.linalg.norm(a) / np.linalg.norm(ref))
    Sc.close()


def test_constants_in_kernel_and_mass_sums_to_area():
    m = gen.graded(9, seed=4)
    Sc = cpp.SEMC(m["coords"], m["quads"], 4, 1.0, 1.0)
    # with rho = c = 1 the lumped mass sums to the domain's area (unit square)
    assert abs(Sc.M.sum() - 1.0) <= 1e-13
    u = np.random.default_rng(0).standard_normal(Sc.n_nodes)
    scale = np.abs(Sc.apply_K(u)).max()
    assert np.abs(Sc.apply_K(np.ones(Sc.n_nodes))).max() <= 1e-12 * scale


def test_leapfrog_with_source_and_receivers_matches_numpy_oracle():
    m = gen.graded(10, seed=9)
    p, n = 4, 80
    S = sem.SEM(m["coords"], m["quads"], p, m["vel"], m["rho"])
    Sc = cpp.SEMC(m["coords"], m["quads"], p, m["vel"], m["rho"])
    dt = 0.3 * S.cfl_dt()
    src = (m["src_xy"][0], m["src_xy"][1], m["f0"], m["t0"], m["amp"])
    u, up, tr = S.run(n, dt, src=src, receivers=m["receivers"])
    uc, upc, trc = Sc.run(n, dt, src=src, receivers=m["receivers"])
    assert np.linalg.norm(u) > 0
    assert _rel(uc, u) <= 1e-13 and _rel(upc, up) <= 1e-13 and _rel(trc, tr) <= 1e-13
    # split run: 30 + 50 steps from the intermediate state equal one 80-step run
    u1, up1, _ = Sc.run(30, dt, src=src)
    u2, up2, _ = Sc.run(50, dt, src=src, u0=u1, u_prev=up1, step0=30)
    assert np.array_equal(u2, uc) and np.array_equal(up2, upc)


def test_results_do_not_depend_on_thread_count():
    m = gen.relabel(gen.graded(12, seed=2), seed=5)
    u0 = None
    out = []
    for t in (1, 2, 5):
        Sc = cpp.SEMC(m["coords"], m["quads"], 3, m["vel"], m["rho"], threads=t)
        dt = 0.3 * sem.SEM(m["coords"], m["quads"], 3, m["vel"], m["rho"]).cfl_dt() if u0 is None else dt
        u0 = 0
        src = (m["src_xy"][0], m["src_xy"][1], m["f0"], m["t0"], m["amp"])
        out.append(Sc.run(40, dt, src=src, receivers=m["receivers"]))
        Sc.close()
    for o in out[1:]:
        for a, b in zip(o, out[0]):
            assert np.array_equal(a, b)


def test_rejects_clockwise_elements():
    m = gen.unit_square(2)
    with pytest.raises(ValueError):
        cpp.SEMC(m["coords"], m["quads"][:, ::-1].copy(), 2, 1.0, 1.0, validate=False)
