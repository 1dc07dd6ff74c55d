"""Device allocations through a caller's allocator (sem_set_allocator).

* torch's caching allocator: the run is bitwise the one with cudaMalloc;
* an allocator whose pointers sit 8 bytes off a 16-byte boundary: the
  library hands every such pointer back (the kernels copy node arrays with
  16-byte vectors) and the first call that needs device memory fails with
  SEM_ERR_OOM before any kernel is launched; the next handle, with the
  default allocator again, runs normally.
"""
import numpy as np
import pytest

import gen
from tests._gpu_common import gpu_run, need_gpu

pytestmark = pytest.mark.gpu

SEM_ERR_OOM = 4


def _run(P, m, prec):
    h = P.SEM(m["coords"], m["quads"], 4, "fp64")
    h.sem_set_model(m["vel"], m["rho"])
    dt = 0.3 * h.sem_cfl_dt()
    h.sem_destroy()
    u, tr = gpu_run(P, m, 4, prec, "hilbert", 40, dt, receivers=m["receivers"])[:2]
    return u, tr


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_torch_allocator_bitwise_same(prec):
    P = need_gpu()
    m = gen.graded(20, seed=41)
    u0, tr0 = _run(P, m, prec)
    P.sem_set_allocator_torch()
    try:
        u1, tr1 = _run(P, m, prec)
    finally:
        P.sem_set_allocator_default()
    assert np.array_equal(u0, u1)
    assert np.array_equal(tr0, tr1)


def test_misaligned_allocator_is_refused():
    P = need_gpu()
    import torch

    lib = P.load()
    handed_back = []

    def _alloc(nbytes, stream, ctx):
        base = torch.cuda.caching_allocator_alloc(int(nbytes) + 16, torch.cuda.current_device(),
                                                  stream if stream else 0)
        return int(base) + 8

    def _free(ptr, nbytes, stream, ctx):
        handed_back.append(int(ptr))
        torch.cuda.caching_allocator_delete(int(ptr) - 8)

    a, f = P._ALLOC(_alloc), P._FREE(_free)
    assert lib.sem_set_allocator(a, f, None) == 0
    m = gen.graded(12, seed=43)
    try:
        h = P.SEM(m["coords"], m["quads"], 4, "fp32_kahan")
        with pytest.raises(P.SemError) as ei:
            # whichever of these first needs device memory fails
            h.sem_set_model(m["vel"], m["rho"])
            h.sem_set_dt(1e-6)
            h.sem_step(3)
        assert ei.value.status == SEM_ERR_OOM
        h.sem_destroy()
    finally:
        P.sem_set_allocator_default()
    assert handed_back and all(p % 16 == 8 for p in handed_back)
    torch.cuda.synchronize()
    # the default allocator again: a normal run
    u, _ = _run(P, m, "fp32_kahan")
    assert np.isfinite(u).all() and np.linalg.norm(u) > 0
