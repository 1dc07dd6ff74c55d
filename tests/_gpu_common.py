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
