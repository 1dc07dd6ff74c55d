"""Shared helpers of the GPU parity tests: build/load the library, run the
CUDA path through the C ABI, run the FP64 oracle on the same seeded input."""
import numpy as np
import pytest

from oracle import sem as osem

FP64_TOL = 1e-12   # relative L2, FP64 GPU vs FP64 oracle
FP32_TOL = 1e-5    # relative L2, FP32 (+Kahan) GPU vs FP64 oracle


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08416_gb300 import build
    build.build()
    import paper_2104_08416_gb300 as P
    P.load()
    return P


# unit roundoff of FP32 (round to nearest)
U32 = 2.0 ** -24


def fp32_apply_bound(S, u):
    """Relative L2 bound for K u computed in FP32 by the sum-factorised path.

    Forward error analysis: every output (K u)_nu is a chain of sums and
    products of the FP32-rounded input u, the GLL derivative entries and the
    per-point metric G_q (formed in FP32 from the element's bilinear map).
    Each floating-point operation contributes at most one unit roundoff U32
    relative to the absolute value of what it combines, so
        |fl(K u) - K u| <= gamma * a,   a = sum_e |B|^T |G_q| |B| |u_e|
    elementwise (a is K u with every term taken in absolute value, in the
    factorisation the kernels evaluate: gradient, metric, transposed
    gradient), with gamma = (2 (p+1) + 24) U32: p+1 terms in each of the two
    contractions, the input rounding, the metric's own error (a few ulps from
    the bilinear coefficients, the determinant and the division) and the
    assembly of at most four element contributions, with a margin. Returned
    as gamma ||a|| / ||K u||: for white noise ||a|| / ||K u|| is 2 to 3, for
    smooth fields it grows like 1/h^2 (K u is small where u is nearly in
    the kernel of K), which is the cancellation any FP32 evaluation of the
    operator meets, whatever the implementation."""
    ae = np.einsum("qda,eqdk,qkb,eb->ea", np.abs(S.B), np.abs(S.G), np.abs(S.B), np.abs(u[S.conn]),
                   optimize=True)
    a = np.bincount(S.conn.ravel(), weights=ae.ravel(), minlength=S.n_nodes)
    gamma = (2 * (S.p + 1) + 24) * U32
    return float(gamma * np.linalg.norm(a) / np.linalg.norm(S.apply_K(u)))


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def gpu_run(P, m, p, precision, ordering, nsteps, dt, receivers=None, eb=0, seed=12345):
    h = P.SEM(m["coords"], m["quads"], p, precision)
    h.sem_reorder(ordering, seed)
    h.sem_set_model(m["vel"], m["rho"])
    if eb:
        h.sem_set_tuning(eb)
    h.sem_set_source(m["f0"], m["t0"], m["amp"], *m["src_xy"])
    if receivers is not None:
        h.sem_set_receivers(receivers, nsteps)
    h.sem_set_dt(dt)
    h.sem_step(nsteps)
    u = h.sem_read_wavefield()
    tr = h.sem_read_traces() if receivers is not None else None
    info = h.sem_launch_info()
    h.sem_destroy()
    return u, tr, info


def oracle_run(m, p, nsteps, dt, receivers=None):
    S = osem.SEM(m["coords"], m["quads"], p, m["vel"], m["rho"])
    src = (m["src_xy"][0], m["src_xy"][1], m["f0"], m["t0"], m["amp"])
    u, up, tr = S.run(nsteps, dt, src=src, receivers=receivers)
    return S, u, tr
