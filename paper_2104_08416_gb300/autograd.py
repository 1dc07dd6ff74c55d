"""The L2 trace misfit as a differentiable function of the per-element wave
speeds, for torch.autograd.

`Survey` holds the shots of one mesh (source positions, receivers, observed
traces, steps, dt) and one library handle per shot, built once and updated in
place with each new model (sem_set_model). `trace_misfit(vel, survey)` returns
the misfit summed over the shots; its backward pass uses the gradient that
sem_misfit_gradient computes with the discrete adjoint of the time step on the
GPU (sqrt(T) checkpointing). Everything numerical runs in the library; this
module only marshals arrays and adds the per-shot results.
"""
from __future__ import annotations

import numpy as np
import torch

from . import SEM


class Survey:
    def __init__(self, coords, quads, order: int, sources, receivers, d_obs, nsteps: int, dt: float,
                 f0: float, t0: float, amp: float = 1.0, rho=None, precision: str = "fp64",
                 ordering: str = "hilbert", checkpoint_every: int = 0):
        self.coords = np.asarray(coords, dtype=np.float64)
        self.quads = np.asarray(quads, dtype=np.int32)
        self.order = int(order)
        self.sources = [tuple(s) for s in sources]
        self.receivers = np.asarray(receivers, dtype=np.float64)
        self.d_obs = [np.ascontiguousarray(d, dtype=np.float64) for d in d_obs]
        if len(self.d_obs) != len(self.sources):
            raise ValueError("one observed trace set per source")
        self.nsteps, self.dt = int(nsteps), float(dt)
        self.f0, self.t0, self.amp = float(f0), float(t0), float(amp)
        self.rho = None if rho is None else np.asarray(rho, dtype=np.float64)
        self.precision, self.ordering = precision, ordering
        self.checkpoint_every = int(checkpoint_every)
        self._handles = None

    def _ensure(self, vel):
        if self._handles is None:
            self._handles = []
            for sx, sy in self.sources:
                h = SEM(self.coords, self.quads, self.order, self.precision)
                h.sem_reorder(self.ordering)
                h.sem_set_model(vel, self.rho)
                h.sem_set_source(self.f0, self.t0, self.amp, sx, sy)
                h.sem_set_receivers(self.receivers, self.nsteps)
                h.sem_set_dt(self.dt)
                self._handles.append(h)
        else:
            for h in self._handles:
                h.sem_set_model(vel, self.rho)

    def misfit_and_gradient(self, vel, gradient: bool = True):
        """(sum of the shots' misfits, sum of their gradients or None)."""
        vel = np.ascontiguousarray(vel, dtype=np.float64)
        self._ensure(vel)
        J, G = 0.0, (np.zeros(vel.size) if gradient else None)
        for h, obs in zip(self._handles, self.d_obs):
            j, g = h.sem_misfit_gradient(obs, self.nsteps, self.checkpoint_every, gradient)
            J += j
            if gradient:
                G += g
        return J, G

    def close(self):
        for h in self._handles or []:
            h.sem_destroy()
        self._handles = None


class TraceMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vel, survey):
        v = vel.detach().to("cpu", torch.float64).numpy()
        J, g = survey.misfit_and_gradient(v, gradient=True)
        ctx.save_for_backward(torch.from_numpy(g).to(device=vel.device, dtype=vel.dtype))
        return vel.new_tensor(J)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None


def trace_misfit(vel: torch.Tensor, survey: Survey) -> torch.Tensor:
    return TraceMisfit.apply(vel, survey)
