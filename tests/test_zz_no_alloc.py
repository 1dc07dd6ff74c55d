"""The allocation-free stiffness entry point (sem_apply_stiffness_dev_noalloc).

Some callers cannot allocate device memory at the moment they need the
operator: a real-time loop that must never reach the allocator (an allocation
can synchronise the device and take unbounded time), or a process that hands
all device memory out from its own pool sized up front. This entry
point keeps its scratch (the partial sums of nodes shared between element
blocks) in a fixed-size device array inside the library, so a call allocates
nothing. Checked here through the C ABI against sem_apply_stiffness, on two
calls in a row, and against the FP64 oracle's K u. The cases cover both kinds
of block plan (DENSE for Hilbert ordering, GATHER for random ordering) and
device arrays that are not 16-byte aligned (element-wise copies and stores).
This file is collected last on purpose.
"""
import numpy as np
import pytest

import gen
from oracle import sem as osem
from tests._gpu_common import FP64_TOL, fp32_apply_bound, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ordering,offset", [("hilbert", 0), ("random", 0), ("hilbert", 1)])
@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_noalloc_matches_apply_stiffness_twice(prec, ordering, offset):
    """offset: the device arrays start that many values past a 16-byte
    aligned base (1 = misaligned)."""
    P = need_gpu()
    import torch

    m = gen.graded(48 if ordering == "hilbert" else 24, seed=31)
    S = osem.SEM(m["coords"], m["quads"], 4, m["vel"], m["rho"], validate=False)
    h = P.SEM(m["coords"], m["quads"], 4, prec)
    h.sem_reorder(ordering)
    h.sem_set_model(m["vel"], m["rho"])
    rng = np.random.default_rng(5)
    fields = [rng.standard_normal(h.n_nodes), np.cos(7.0 * h.sem_node_coordinates()[:, 0])]
    _, node_new = h.sem_get_permutation()
    tdt = torch.float64 if prec == "fp64" else torch.float32
    base_u = torch.empty(h.n_nodes + 4, dtype=tdt, device="cuda")
    base_ku = torch.empty(h.n_nodes + 4, dtype=tdt, device="cuda")
    dev_u = base_u[offset:offset + h.n_nodes]
    dev_ku = base_ku[offset:offset + h.n_nodes]
    assert (dev_u.data_ptr() % 16 == 0) == (offset == 0)
    for u in fields:                       # two calls in a row
        ref = h.sem_apply_stiffness(u)     # existing entry point (builds device data on first use)
        u_store = np.empty_like(u)
        u_store[node_new] = u
        dev_u.copy_(torch.from_numpy(u_store).to(tdt))
        base_ku.fill_(float("nan"))
        h.sem_apply_stiffness_dev_noalloc(dev_u.data_ptr(), dev_ku.data_ptr())
        torch.cuda.synchronize()
        out = dev_ku.double().cpu().numpy()[node_new]
        assert np.isfinite(out).all()
        # nothing written outside the output array
        assert torch.isnan(base_ku[:offset]).all() and torch.isnan(base_ku[offset + h.n_nodes:]).all()
        # the same kernel arithmetic as the allocating entry point
        assert rel_l2(out, ref) <= 1e-12, rel_l2(out, ref)
        # and the oracle's K u within the tolerance of the other parity tests
        ref_o = S.apply_K(u)
        tol = FP64_TOL if prec == "fp64" else fp32_apply_bound(S, u)
        assert rel_l2(out, ref_o) < tol, (rel_l2(out, ref_o), tol)
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
