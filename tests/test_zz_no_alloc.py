"""The allocation-free stiffness entry point (sem_apply_stiffness_dev_noalloc).

Some callers cannot allocate device memory at the moment they need the
operator: a real-time loop that must never reach the allocator (an allocation
can synchronise the device and take unbounded time), or a process that hands
all device memory out from its own pool sized up front. This entry
point keeps its scratch (the partial sums of nodes shared between element
blocks) in a fixed-size device array inside the library, so a call allocates
nothing. Checked here through the C ABI against sem_apply_stiffness, on two
calls in a row. This file is collected last on purpose.
"""
import numpy as np
import pytest

import gen
from tests._gpu_common import FP32_TOL, FP64_TOL, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_noalloc_matches_apply_stiffness_twice(prec):
    P = need_gpu()
    import torch

    m = gen.graded(48, seed=31)
    h = P.SEM(m["coords"], m["quads"], 4, prec)
    h.sem_reorder("hilbert")
    h.sem_set_model(m["vel"], m["rho"])
    rng = np.random.default_rng(5)
    fields = [rng.standard_normal(h.n_nodes), np.cos(7.0 * h.sem_node_coordinates()[:, 0])]
    _, node_new = h.sem_get_permutation()
    tdt = torch.float64 if prec == "fp64" else torch.float32
    tol = FP64_TOL if prec == "fp64" else FP32_TOL
    dev_u = torch.empty(h.n_nodes, dtype=tdt, device="cuda")
    dev_ku = torch.empty(h.n_nodes, dtype=tdt, device="cuda")
    for u in fields:                       # two calls in a row
        ref = h.sem_apply_stiffness(u)     # existing entry point (builds device data on first use)
        u_store = np.empty_like(u)
        u_store[node_new] = u
        dev_u.copy_(torch.from_numpy(u_store).to(tdt))
        dev_ku.fill_(float("nan"))
        h.sem_apply_stiffness_dev_noalloc(dev_u.data_ptr(), dev_ku.data_ptr())
        torch.cuda.synchronize()
        out = dev_ku.double().cpu().numpy()[node_new]
        assert np.isfinite(out).all()
        assert rel_l2(out, ref) < tol, rel_l2(out, ref)
    h.sem_destroy()


def test_noalloc_requires_built_handle_and_rejects_large_meshes():
    P = need_gpu()
    import torch

    m = gen.unit_square(4)
    h = P.SEM(m["coords"], m["quads"], 2, "fp64")
    h.sem_set_model(m["vel"])
    buf = torch.zeros(2 * h.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(P.SemError) as ei:
        h.sem_apply_stiffness_dev_noalloc(buf.data_ptr(), buf.data_ptr() + 8 * h.n_nodes)
    assert ei.value.status == P.SEM_ERR_STATE
    h.sem_destroy()
    # random ordering of a 512 x 512 order-4 mesh: several million open entries
    m = gen.graded(512)
    h = P.SEM(m["coords"], m["quads"], 4, "fp64")
    h.sem_reorder("random")
    h.sem_set_model(m["vel"], m["rho"])
    h.sem_read_mass()                      # builds the device data
    big = torch.zeros(2 * h.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(P.SemError) as ei:
        h.sem_apply_stiffness_dev_noalloc(big.data_ptr(), big.data_ptr() + 8 * h.n_nodes)
    assert ei.value.status == P.SEM_ERR_INVALID_ARG
    h.sem_destroy()
