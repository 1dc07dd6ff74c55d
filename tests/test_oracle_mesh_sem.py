"""Pins of the oracle's mesh numbering, geometry, mass, stiffness and time
stepping (Section 4.1, Section 4.2: Eqs. deriv_u, Abar, u_change_r_effic;
leapfrog with the initial condition of Eq. initial_cond)."""
import math

import numpy as np
import pytest

import gen
from oracle import gll, mesh, sem


def _tiny_graded(n=6, seed=11):
    return gen.graded(n, ratio=8.0, perturb=0.2, seed=seed)


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_node_count_and_sharing(p):
    m = gen.unit_square(5)
    conn, n_nodes, _ = mesh.canonical_numbering(m["quads"], m["coords"].shape[0], p)
    assert n_nodes == (5 * p + 1) ** 2
    assert set(np.unique(conn)) == set(range(n_nodes))
    counts = np.bincount(conn.ravel())
    # interior-of-element nodes: 1 element; edge nodes: 1 or 2; vertices: 1..4
    assert counts.max() == 4 and counts.min() == 1
    for e in range(conn.shape[0]):
        assert len(set(conn[e])) == conn.shape[1]


@pytest.mark.parametrize("p", [2, 3, 5])
def test_shared_nodes_have_one_position(p):
    """Each slot's position from its element's bilinear map equals the global
    node's position: catches a reversed edge or a wrong local index."""
    m = gen.relabel(_tiny_graded(5), seed=3)
    coords, quads = m["coords"], m["quads"]
    conn, n_nodes, edges = mesh.canonical_numbering(quads, coords.shape[0], p)
    xy = mesh.node_coordinates(coords, quads, p, conn, edges)
    s = gll.gll_nodes(p)
    corners = coords[quads.astype(np.int64)]
    for j in range(p + 1):
        for i in range(p + 1):
            X = mesh.bilinear(corners, s[i], s[j])
            np.testing.assert_allclose(xy[conn[:, j * (p + 1) + i]], X, atol=1e-14)


def test_numbering_first_ids_are_vertices_and_edges_in_order():
    m = gen.unit_square(2)
    conn, n, edges = mesh.canonical_numbering(m["quads"], 9, 2)
    # element 0 = vertices (0,1,4,3): its bottom edge (0,1) is the first edge,
    # so its midpoint is id 9; the next edge (1,4) gets 10.
    assert conn[0, 1] == 9 and conn[0, 5] == 10
    assert edges[0].tolist() == [0, 1, 9]


@pytest.mark.parametrize("make", ["unit", "graded", "layered"])
def test_mass_sums_to_area(make):
    if make == "unit":
        m = gen.unit_square(4)
        area = 1.0
    elif make == "graded":
        m = _tiny_graded(6)
        area = 1.0
    else:
        m = gen.layered(16, 4)
        area = 40000.0 * 10000.0
    S = sem.SEM(m["coords"], m["quads"], 4, 1.0, 1.0)
    assert abs(S.M.sum() - area) <= 1e-13 * area


def test_mass_scales_with_material():
    m = _tiny_graded(4)
    v = 1.0 + np.arange(16) / 8.0
    rho = 2.0 + np.arange(16) / 16.0
    S = sem.SEM(m["coords"], m["quads"], 3, v, rho)
    S1 = sem.SEM(m["coords"], m["quads"], 3, 1.0, 1.0)
    loc = S1.w2[None, :] * S1.detJ
    areas = loc.sum(axis=1)
    # sum of the lumped mass = sum_e area_e / (rho_e c_e^2)
    assert abs(S.M.sum() - (areas / (rho * v ** 2)).sum()) < 1e-14


@pytest.mark.parametrize("p", [1, 3, 4, 7])
def test_stiffness_kills_constants(p):
    m = _tiny_graded(5)
    S = sem.SEM(m["coords"], m["quads"], p, 1.0, 1.0 + 0.1 * np.arange(25))
    assert np.abs(S.apply_K(np.ones(S.n_nodes))).max() < 1e-12


@pytest.mark.parametrize("p", [2, 4])
def test_linear_fields_on_bilinear_mesh(p):
    """For u = a x + b y: u^T K u = |(a,b)|^2 area / rho exactly (|J| is
    bilinear, so GLL integrates it exactly), and (K u) vanishes at nodes away
    from the boundary (the weak form of a harmonic field has only boundary
    flux). Catches a transposed metric J^-1 J^-T vs J^-T J^-1 on skewed quads."""
    m = _tiny_graded(6)
    rho = 2.5
    S = sem.SEM(m["coords"], m["quads"], p, 1.0, rho)
    a, b = 0.7, -1.3
    u = a * S.node_xy[:, 0] + b * S.node_xy[:, 1]
    Ku = S.apply_K(u)
    assert abs(u @ Ku - (a * a + b * b) * 1.0 / rho) < 1e-12
    x, y = S.node_xy[:, 0], S.node_xy[:, 1]
    interior = (x > 1e-12) & (x < 1 - 1e-12) & (y > 1e-12) & (y < 1 - 1e-12)
    assert np.abs(Ku[interior]).max() < 1e-11
    # boundary flux of grad u . n over the bottom edge (n = -y) equals -b * length
    bottom = y < 1e-12
    assert abs(Ku[bottom].sum() - (-b / rho)) < 1e-12


def test_stiffness_symmetric_psd():
    m = _tiny_graded(3)
    S = sem.SEM(m["coords"], m["quads"], 3, 1.0, 1.0 + np.arange(9) / 9)
    K = np.stack([S.apply_K(e) for e in np.eye(S.n_nodes)], axis=1)
    np.testing.assert_allclose(K, K.T, atol=1e-12)
    ev = np.linalg.eigvalsh(0.5 * (K + K.T))
    assert ev.min() > -1e-10
    assert np.sum(np.abs(ev) < 1e-9) == 1        # only the constant mode


def test_ricker_closed_form():
    f0, t0 = 10.0, 0.12
    assert sem.ricker(t0, f0, t0) == 1.0
    # zero crossings at t0 +- 1 / (pi f0 sqrt 2)
    tz = t0 + 1.0 / (math.pi * f0 * math.sqrt(2.0))
    assert abs(sem.ricker(tz, f0, t0)) < 1e-15


def test_snap_ties_go_to_lowest_id():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    assert sem.snap(xy, 0.5, 0.0) == 0
    assert sem.snap(xy, 0.9, 0.1) == 1


def _standing_mode_error(p, n=4, dt=None, t_end=0.35):
    m = gen.unit_square(n)
    S = sem.SEM(m["coords"], m["quads"], p, 1.0, 1.0)
    x, y = S.node_xy[:, 0], S.node_xy[:, 1]
    omega = math.pi * math.sqrt(2.0)
    u0 = np.cos(math.pi * x) * np.cos(math.pi * y)
    if dt is None:
        dt = 0.05 * S.cfl_dt()
    nsteps = int(round(t_end / dt))
    # u^{-1} from a second-order Taylor step (zero initial velocity)
    um1 = u0 - 0.5 * dt * dt * S.apply_K(u0) / S.M
    u, _, _ = S.run(nsteps, dt, u0=u0, u_prev=um1)
    exact = u0 * math.cos(omega * nsteps * dt)
    return np.sqrt(np.sum(S.M * (u - exact) ** 2) / np.sum(S.M * exact ** 2))


def test_standing_mode_spectral_convergence():
    """cos(pi x) cos(pi y) cos(pi sqrt2 t) solves the Neumann problem on the unit
    square; at fixed h and tiny dt the error falls exponentially with p."""
    errs = [_standing_mode_error(p, n=2, dt=1e-4) for p in (2, 3, 4, 5, 6)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 5e-6 and errs[0] > 1e-3, errs
    # roughly geometric decay: each step of p gains at least a factor 4
    assert all(b < a / 4 for a, b in zip(errs, errs[1:])), errs


def test_standing_mode_second_order_in_time():
    """At high p the leapfrog error is O(dt^2)."""
    m = gen.unit_square(2)
    e1 = _standing_mode_error(8, n=2, dt=4e-3, t_end=0.4)
    e2 = _standing_mode_error(8, n=2, dt=2e-3, t_end=0.4)
    assert 3.5 < e1 / e2 < 4.5, (e1, e2)


def test_energy_conserved_unforced():
    m = _tiny_graded(6)
    S = sem.SEM(m["coords"], m["quads"], 4, m["vel"][:36] if m["vel"].size == 36 else m["vel"], 1.0)
    rng = np.random.default_rng(0)
    x, y = S.node_xy[:, 0], S.node_xy[:, 1]
    u0 = np.exp(-40 * ((x - 0.4) ** 2 + (y - 0.6) ** 2))
    dt = 0.3 * S.cfl_dt()
    up = u0 - 0.5 * dt * dt * S.apply_K(u0) / S.M
    energies = []

    def cb(n, u, uprev):
        energies.append(S.energy(u, uprev, dt))

    S.run(300, dt, u0=u0, u_prev=up, callback=cb)
    e = np.array(energies)
    assert np.ptp(e) / e[0] < 1e-11


def test_cfl_fraction_is_stable():
    m = _tiny_graded(5)
    S = sem.SEM(m["coords"], m["quads"], 4, m["vel"], 1.0)
    dt = 0.3 * S.cfl_dt()
    assert dt < 2.0 / math.sqrt(S.lambda_max())


def test_source_and_receivers_run():
    m = gen.unit_square(4)
    S = sem.SEM(m["coords"], m["quads"], 4, 1.0, 1.0)
    dt = 0.3 * S.cfl_dt()
    u, up, tr = S.run(50, dt, src=(0.5, 0.5, 10.0, 0.12, 1.0),
                      receivers=np.array([[0.5, 0.5], [0.0, 0.0]]))
    s = sem.snap(S.node_xy, 0.5, 0.5)
    np.testing.assert_array_equal(tr[0], tr[0])
    assert tr.shape == (2, 50) and tr[0, -1] == u[s]
    # first step: u^1 = dt^2 M^-1 f(0) e_s
    f_0 = sem.ricker(0.0, 10.0, 0.12)
    assert abs(tr[0, 0] - dt * dt * f_0 / S.M[s]) < 1e-18


def test_apply_K_at_matches_full():
    m = _tiny_graded(4)
    S = sem.SEM(m["coords"], m["quads"], 3, 1.0, 1.0)
    u = np.sin(3 * S.node_xy[:, 0]) * np.cos(2 * S.node_xy[:, 1])
    nodes = np.array([0, 5, 17, S.n_nodes - 1])
    np.testing.assert_allclose(S.apply_K_at(u, nodes), S.apply_K(u)[nodes], atol=1e-13)


def test_adjoint_gradient_matches_central_differences():
    """The oracle's discrete adjoint against central finite differences of the
    misfit in single element speeds (layered-like heterogeneous model)."""
    m = gen.graded(6, seed=11)
    p, n = 3, 160
    vel_true = np.asarray(m["vel"], dtype=np.float64)
    vel = vel_true * (1.0 + 0.05 * np.sin(np.arange(vel_true.size)))
    rec = np.array([[0.1, 0.9], [0.8, 0.85], [0.5, 0.2], [0.95, 0.4]])
    src = (m["src_xy"][0], m["src_xy"][1], m["f0"], m["t0"], m["amp"])
    S_true = sem.SEM(m["coords"], m["quads"], p, vel_true, m["rho"])
    dt = 0.3 * S_true.cfl_dt()
    _, _, d_obs = S_true.run(n, dt, src=src, receivers=rec)
    S = sem.SEM(m["coords"], m["quads"], p, vel, m["rho"])
    J, grad, _ = S.misfit_gradient(n, dt, src, rec, d_obs)
    assert J > 0
    for e in (0, 7, 15, 22, 35):
        h = 1e-5 * vel[e]
        vp, vm = vel.copy(), vel.copy()
        vp[e] += h
        vm[e] -= h
        Jp = 0.5 * dt * np.sum((sem.SEM(m["coords"], m["quads"], p, vp, m["rho"]).run(n, dt, src=src, receivers=rec)[2] - d_obs) ** 2)
        Jm = 0.5 * dt * np.sum((sem.SEM(m["coords"], m["quads"], p, vm, m["rho"]).run(n, dt, src=src, receivers=rec)[2] - d_obs) ** 2)
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - grad[e]) <= 1e-5 * np.abs(grad).max(), (e, fd, grad[e])


def test_adjoint_gradient_vanishes_at_the_true_model():
    m = gen.graded(5, seed=3)
    p, n = 2, 80
    rec = np.array([[0.2, 0.8], [0.7, 0.7]])
    src = (m["src_xy"][0], m["src_xy"][1], m["f0"], m["t0"], m["amp"])
    S = sem.SEM(m["coords"], m["quads"], p, m["vel"], m["rho"])
    dt = 0.3 * S.cfl_dt()
    _, _, d_obs = S.run(n, dt, src=src, receivers=rec)
    J, grad, _ = S.misfit_gradient(n, dt, src, rec, d_obs)
    assert J == 0.0 and np.all(grad == 0.0)


def test_first_order_divergence_of_gradient_is_minus_stiffness():
    """R(V) with V = grad u / rho at the local nodes equals -K u exactly (up to
    rounding): the first-order form (Section 4.2, Eqs. v_change, u_change_r_effic)
    and the assembled stiffness describe the same operator."""
    for p in (1, 3, 5):
        m = gen.relabel(gen.graded(5, seed=p), seed=p)
        rho = 0.5 + np.random.default_rng(p).random(m["quads"].shape[0])
        S = sem.SEM(m["coords"], m["quads"], p, m["vel"], rho)
        u = np.random.default_rng(p + 1).standard_normal(S.n_nodes)
        Ud, Vd = S.first_order_rhs(u, np.zeros((S.conn.shape[0], S.conn.shape[1], 2)))
        assert np.all(Ud == 0.0)
        R_over_M, _ = S.first_order_rhs(np.zeros(S.n_nodes), Vd)
        ref = -S.apply_K(u)
        assert np.linalg.norm(R_over_M * S.M - ref) <= 1e-12 * np.linalg.norm(ref)


def test_heun_standing_mode_second_order():
    """Heun on the first-order system from U = cos(pi x) cos(pi y), V = 0 in
    the Neumann unit square: error against cos(pi x) cos(pi y) cos(pi sqrt2 t)
    at p = 7 falls by about 4 when the step halves."""
    m = gen.unit_square(2)
    p = 7
    S = sem.SEM(m["coords"], m["quads"], p, 1.0, 1.0)
    x, y = S.node_xy[:, 0], S.node_xy[:, 1]
    u0 = np.cos(np.pi * x) * np.cos(np.pi * y)
    T = 0.25
    errs = []
    for nsteps in (100, 200):
        h = T / nsteps
        U, _, _ = S.run_heun(nsteps, h, U0=u0)
        errs.append(np.abs(U - u0 * np.cos(np.pi * np.sqrt(2) * T)).max())
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


def test_leapfrog_discrete_dispersion_on_eigenmodes():
    """On an eigenvector v of the generalized problem K v = lambda M v (found
    here by a dense library eigensolver, not by the oracle), the unforced
    leapfrog started from u^0 = v, u^-1 = cos(theta) v must give exactly
    u^n = cos(n theta) v with cos(theta) = 1 - dt^2 lambda / 2: the
    three-level recurrence's discrete dispersion relation. A dropped factor 2,
    a sign or dt power, or M where M^-1 belongs breaks it."""
    import scipy.linalg

    m = _tiny_graded(4, seed=5)
    S = sem.SEM(m["coords"], m["quads"], 3, m["vel"], 1.0)
    n = S.n_nodes
    K = np.stack([S.apply_K(e) for e in np.eye(n)], axis=1)
    lam, V = scipy.linalg.eigh(0.5 * (K + K.T), np.diag(S.M))
    dt = 0.3 * S.cfl_dt()
    nsteps = 60
    for k in (1, 7, n // 2, n - 1):
        v = V[:, k] / np.linalg.norm(V[:, k])
        c = 1.0 - 0.5 * dt * dt * lam[k]
        assert -1.0 < c <= 1.0           # stable at 0.3 of the CFL step
        theta = math.acos(c)
        u, up, _ = S.run(nsteps, dt, u0=v, u_prev=c * v)
        assert np.allclose(u, math.cos(nsteps * theta) * v, rtol=0, atol=1e-9), k
        assert np.allclose(up, math.cos((nsteps - 1) * theta) * v, rtol=0, atol=1e-9), k


@pytest.mark.parametrize("n,p", [(3, 2), (4, 3), (5, 4)])
def test_lambda_max_matches_dense_generalized_eigensolver(n, p):
    """The power iteration behind the stability pin against the largest
    eigenvalue of K v = lambda M v from a dense library eigensolver (K built
    column by column from apply_K, M the lumped mass). An unconverged
    iteration or a wrong symmetrisation (M instead of sqrt(M) on one side)
    gives a different value."""
    import scipy.linalg

    m = _tiny_graded(n, seed=11)
    S = sem.SEM(m["coords"], m["quads"], p, m["vel"], 1.0)
    K = np.stack([S.apply_K(e) for e in np.eye(S.n_nodes)], axis=1)
    lam = scipy.linalg.eigh(0.5 * (K + K.T), np.diag(S.M), eigvals_only=True)
    assert abs(S.lambda_max() - lam[-1]) <= 1e-10 * lam[-1]
    # the stability pin then holds with the exact eigenvalue as well
    assert 0.3 * S.cfl_dt() < 2.0 / math.sqrt(lam[-1])


@pytest.mark.parametrize("p,gap", [(2, 0.5), (3, (1 - math.sqrt(1 / 5)) / 2), (4, (1 - math.sqrt(3 / 7)) / 2)])
def test_cfl_dt_single_element_closed_form(p, gap):
    """dt_CFL of one axis-aligned w x h element with speed c is the smallest
    gap between neighbouring GLL points on [-1, 1] (end pair: 1 - x_1) scaled
    by the shorter side over 2, divided by c. The GLL points are 0, +-1 at
    p = 2; +-sqrt(1/5), +-1 at p = 3; 0, +-sqrt(3/7), +-1 at p = 4, so the
    shortest gap in units of the element side is 0.5, (1 - sqrt(1/5))/2,
    (1 - sqrt(3/7))/2."""
    for w, h, c in ((1.0, 1.0, 2.0), (2.0, 0.5, 1.5), (0.25, 3.0, 4.0)):
        coords = np.array([[0.0, 0.0], [w, 0.0], [w, h], [0.0, h]])
        quads = np.array([[0, 1, 2, 3]])
        S = sem.SEM(coords, quads, p, c, 1.0)
        want = gap * min(w, h) / c
        assert abs(S.cfl_dt() - want) <= 1e-15 * want, (w, h, c, S.cfl_dt(), want)


def test_mesh_validate_accepts_and_rejects():
    """mesh.validate passes the generators' meshes and refuses each kind of
    broken input with its own message."""
    for m in (gen.unit_square(3), _tiny_graded(4), gen.relabel(_tiny_graded(4), seed=2)):
        mesh.validate(m["coords"], m["quads"], 4)
    m = gen.unit_square(2)
    coords, quads = m["coords"], m["quads"].copy()
    bad = quads.copy()
    bad[0, 0] = coords.shape[0]
    with pytest.raises(ValueError, match="out of range"):
        mesh.validate(coords, bad, 2)
    bad = quads.copy()
    bad[0, 0] = -1
    with pytest.raises(ValueError, match="out of range"):
        mesh.validate(coords, bad, 2)
    with pytest.raises(ValueError, match="unreferenced"):
        mesh.validate(np.vstack([coords, [[5.0, 5.0]]]), quads, 2)
    # clockwise corners: negative Jacobian everywhere
    with pytest.raises(ValueError, match="Jacobian"):
        mesh.validate(coords, quads[:, ::-1].copy(), 2)
    # a bow-tie (two corners swapped): the Jacobian changes sign inside
    bt = quads.copy()
    bt[0, [1, 2]] = bt[0, [2, 1]]
    with pytest.raises(ValueError):
        mesh.validate(coords, bt, 2)
    # a third element on an existing edge
    c3 = np.vstack([coords, [[0.25, -0.5], [0.75, -0.5]]])
    nv = coords.shape[0]
    e0 = quads[0]
    extra = np.array([[nv, nv + 1, e0[1], e0[0]]])      # below element 0, sharing its bottom edge
    dup = np.array([[nv, nv + 1, e0[1], e0[0]]])
    with pytest.raises(ValueError, match="more than two"):
        mesh.validate(c3, np.vstack([quads, extra, dup]), 2)
