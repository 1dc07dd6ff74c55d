"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the spectral-element method or of the
memory reorderings: it only emits meshes (vertex coordinates and CCW quad
connectivity), per-element material values, and source/receiver positions.
Both the CUDA path (through the C-ABI) and the FP64 oracle consume its output.

The paper benchmarks on Gmsh meshes that are not available (Section 6.1.1,
Section 6.1.2, Table "mesh_variation"); these generators stand in for them with
the same structure: a homogeneous mesh, a strongly graded and perturbed mesh
(element-size ratio 8 between the smallest and the largest element), and a
multilayered velocity model whose velocities grow with depth (Section 6.2,
Table "layer_velocities").

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): uniform doubles are
``(next() >> 11) * 2**-53``. Stream ``seed+0`` draws mesh perturbations,
``seed+1`` draws the material model, ``seed+4`` draws test relabellings.
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_SEED = 2104084160
_MASK = (1 << 64) - 1


class SplitMix64:
    """splitmix64 stream (public-domain reference definition by S. Vigna)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniforms(self, n: int) -> np.ndarray:
        """n consecutive uniform draws (vectorised; same values as n calls)."""
        if n == 0:
            return np.zeros(0)
        g = np.uint64(0x9E3779B97F4A7C15)
        with np.errstate(over="ignore"):
            ks = np.arange(1, n + 1, dtype=np.uint64)
            z = np.uint64(self.state) + ks * g
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * 0x9E3779B97F4A7C15) & _MASK
        return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _grid_quads(nx: int, ny: int) -> np.ndarray:
    """Row-major CCW quads of an (nx+1) x (ny+1) vertex lattice."""
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    v0 = j * (nx + 1) + i
    q = np.stack([v0, v0 + 1, v0 + nx + 2, v0 + nx + 1], axis=-1)
    return q.reshape(-1, 4).astype(np.int32)


def _lattice(xs: np.ndarray, ys: np.ndarray) -> np.ndarray:
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel()], axis=-1).astype(np.float64)


def unit_square(n: int = 32, f0: float = 10.0, n_receivers: int = 8) -> dict:
    """Homogeneous unit square, n x n equal quads listed row-major (c = rho = 1).

    The workload of the homogeneous benchmark at 32 x 32: 16,641 GLL nodes at
    order 4; Ricker source at the centre; receivers along the top edge.
    """
    t = np.arange(n + 1, dtype=np.float64) / n
    coords = _lattice(t, t)
    quads = _grid_quads(n, n)
    ne = quads.shape[0]
    rec = np.stack([(np.arange(n_receivers) + 0.5) / n_receivers,
                    np.ones(n_receivers)], axis=-1)
    return dict(name=f"unit_square_{n}x{n}", coords=coords, quads=quads,
                vel=np.ones(ne), rho=np.ones(ne), src_xy=(0.5, 0.5), f0=f0,
                t0=1.2 / f0, amp=1.0, receivers=rec, width=1.0, height=1.0)


def graded(n: int = 512, ratio: float = 8.0, perturb: float = 0.2,
           vmin: float = 1.0, vmax: float = 3.0, seed: int = DEFAULT_SEED,
           f0: float = 10.0, n_receivers: int = 16) -> dict:
    """Graded heterogeneous unit square: widths grow geometrically by `ratio`
    from the (0,0) corner along each axis, interior vertices are shifted by
    U[-perturb, perturb] times the smaller adjacent width (x and y drawn
    independently, row-major, x then y), velocities U[vmin, vmax] per element.
    """
    k = np.arange(n, dtype=np.float64)
    w = ratio ** (k / max(n - 1, 1))
    w = w / w.sum()
    edges = np.concatenate([[0.0], np.cumsum(w)])
    edges[-1] = 1.0
    coords = _lattice(edges, edges)
    rng = SplitMix64(seed + 0)
    if n > 1 and perturb > 0:
        m = n - 1
        u = rng.uniforms(2 * m * m).reshape(m, m, 2)
        wmin = np.minimum(w[:-1], w[1:])          # smaller adjacent width at lattice line 1..n-1
        jj, ii = np.meshgrid(np.arange(1, n), np.arange(1, n), indexing="ij")
        idx = (jj * (n + 1) + ii).ravel()
        dx = ((2.0 * perturb) * u[..., 0] - perturb) * wmin[ii - 1]
        dy = ((2.0 * perturb) * u[..., 1] - perturb) * wmin[jj - 1]
        coords[idx, 0] += dx.ravel()
        coords[idx, 1] += dy.ravel()
    quads = _grid_quads(n, n)
    ne = quads.shape[0]
    vel = vmin + (vmax - vmin) * SplitMix64(seed + 1).uniforms(ne)
    rec = np.stack([(np.arange(n_receivers) + 0.5) / n_receivers,
                    np.ones(n_receivers)], axis=-1)
    return dict(name=f"graded_{n}x{n}", coords=coords, quads=quads, vel=vel,
                rho=np.ones(ne), src_xy=(0.5, 0.5), f0=f0, t0=1.2 / f0, amp=1.0,
                receivers=rec, width=1.0, height=1.0)


def layered(nx: int = 4096, nz: int = 1024, width: float = 40000.0,
            depth: float = 10000.0, n_layers: int = 8, vp_top: float = 1500.0,
            vp_bottom: float = 4500.0, seed: int = DEFAULT_SEED, f0: float = 10.0,
            n_receivers: int = 256) -> dict:
    """Multilayered model on a uniform nx x nz quad grid (y up, surface at y=depth).

    Interfaces k = 1..n_layers-1 lie at depth k*depth/n_layers + A_k sin(2 pi x /
    lambda_k + phi_k) with A_k ~ U[0,200] m, lambda_k ~ U[5,20] km,
    phi_k ~ U[0, 2 pi) (drawn in that order per interface); an element takes the
    velocity of the layer holding its centroid, vp_top + (vp_bottom-vp_top) * L /
    (n_layers-1) for layer L counted from the surface; rho = 1.
    """
    xs = np.arange(nx + 1, dtype=np.float64) * (width / nx)
    ys = np.arange(nz + 1, dtype=np.float64) * (depth / nz)
    xs[-1], ys[-1] = width, depth
    coords = _lattice(xs, ys)
    quads = _grid_quads(nx, nz)
    rng = SplitMix64(seed + 1)
    params = rng.uniforms(3 * (n_layers - 1)).reshape(n_layers - 1, 3)
    amp_k = 200.0 * params[:, 0]
    lam_k = 5000.0 + 15000.0 * params[:, 1]
    phi_k = 2.0 * math.pi * params[:, 2]
    xc = 0.5 * (xs[:-1] + xs[1:])
    yc = 0.5 * (ys[:-1] + ys[1:])
    dc = depth - yc                                   # depth of centroid rows
    layer = np.zeros((nz, nx), dtype=np.int64)
    for k in range(1, n_layers):
        dk = k * depth / n_layers + amp_k[k - 1] * np.sin(2 * math.pi * xc / lam_k[k - 1] + phi_k[k - 1])
        layer += (dc[:, None] > dk[None, :]).astype(np.int64)
    vel = (vp_top + (vp_bottom - vp_top) * layer / (n_layers - 1)).ravel()
    rec = np.stack([(np.arange(n_receivers) + 0.5) * (width / n_receivers),
                    np.full(n_receivers, depth)], axis=-1)
    ne = quads.shape[0]
    return dict(name=f"layered_{nx}x{nz}", coords=coords, quads=quads, vel=vel,
                rho=np.ones(ne), src_xy=(0.5 * width, 0.5 * depth), f0=f0,
                t0=1.2 / f0, amp=1.0, receivers=rec, width=width, height=depth)


def relabel(mesh: dict, seed: int = DEFAULT_SEED) -> dict:
    """Same geometry, scrambled input: random vertex ids, random element order and
    a random cyclic rotation of each quad's corners (CCW orientation kept).
    Used to check that nothing depends on the generators' row-major emission."""
    rng = SplitMix64(seed + 4)
    nv = mesh["coords"].shape[0]
    ne = mesh["quads"].shape[0]
    vperm = np.argsort(rng.uniforms(nv), kind="stable")       # new vertex slot -> old id
    v_new_of_old = np.empty(nv, dtype=np.int64)
    v_new_of_old[vperm] = np.arange(nv)
    eperm = np.argsort(rng.uniforms(ne), kind="stable")
    rot = (rng.uniforms(ne) * 4).astype(np.int64)
    q = v_new_of_old[mesh["quads"][eperm]]
    r = rot[:, None]
    q = np.take_along_axis(q, (np.arange(4)[None, :] + r) % 4, axis=1)
    out = dict(mesh)
    out.update(coords=mesh["coords"][vperm].copy(), quads=q.astype(np.int32),
               vel=np.asarray(mesh["vel"])[eperm].copy(),
               rho=np.asarray(mesh["rho"])[eperm].copy(), name=mesh["name"] + "_relabelled")
    return out


def batched(n_shots: int = 64, nmin: int = 64, nmax: int = 1024, orders=(3, 4, 5, 6, 7),
            seed: int = DEFAULT_SEED) -> list:
    """Independent shots for the batched path: square layered models of
    n x n quads over 10 km x 10 km with n uniform in [nmin, nmax], the order
    uniform over `orders`, and the source at a uniformly drawn interior point
    (stream seed+5: n, order, source x, source y per shot, in that order)."""
    rng = SplitMix64(seed + 5)
    shots = []
    for k in range(n_shots):
        n = nmin + min(int(rng.uniform() * (nmax - nmin + 1)), nmax - nmin)
        p = orders[min(int(rng.uniform() * len(orders)), len(orders) - 1)]
        sx, sy = 1000.0 + 8000.0 * rng.uniform(), 1000.0 + 8000.0 * rng.uniform()
        m = layered(n, n, width=10000.0, depth=10000.0, seed=seed + 17 * k, n_receivers=32)
        m["src_xy"] = (sx, sy)
        m["order"] = p
        m["name"] = f"shot{k}_{n}x{n}_p{p}"
        shots.append(m)
    return shots


def adjoint_case(n: int = 256, n_shots: int = 8, n_receivers: int = 64, width: float = 1000.0,
                 f0: float = 30.0, smooth: int = 16, seed: int = DEFAULT_SEED) -> dict:
    """Velocity-gradient case: a layered true model on n x n quads over a
    width x width square (surface at the top), a start model smoothed from it
    by a (2 smooth + 1)^2 moving average over the element grid, n_shots
    sources evenly spaced just below the surface and n_receivers on it."""
    m = layered(n, n, width=width, depth=width, seed=seed, f0=f0, n_receivers=n_receivers)
    v = np.asarray(m["vel"], dtype=np.float64).reshape(n, n)
    pad = np.pad(v, smooth, mode="edge")
    c = np.cumsum(np.cumsum(np.pad(pad, ((1, 0), (1, 0))), axis=0), axis=1)
    k = 2 * smooth + 1
    sm = (c[k:, k:] - c[:-k, k:] - c[k:, :-k] + c[:-k, :-k]) / (k * k)
    xs = (np.arange(n_shots) + 0.5) * (width / n_shots)
    return dict(mesh=m, vel_true=m["vel"], vel_start=sm.ravel(),
                sources=[(float(x), 0.97 * width) for x in xs], receivers=m["receivers"],
                f0=f0, t0=1.2 / f0, amp=1.0)


def config(name: str, seed: int = DEFAULT_SEED) -> dict:
    """The three single-GPU workloads by name, with their step counts."""
    if name == "homogeneous_32":
        m = unit_square(32)
        m["nsteps"] = 400
    elif name == "graded_512":
        m = graded(512, seed=seed)
        m["nsteps"] = 2000
    elif name == "layered_4096x1024":
        m = layered(4096, 1024, seed=seed)
        m["nsteps"] = 3000
    else:
        raise KeyError(name)
    m["order"] = 4
    m["cfl_fraction"] = 0.3
    return m
