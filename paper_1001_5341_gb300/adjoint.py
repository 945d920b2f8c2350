"""Detector traces as a differentiable function of the shower's charge table.

``TraceModel(sim, ...)`` wraps a ``Simulation`` (PEC, Mur or CPML) with detectors: calling it
with a float64 tensor q of charges per bin (Sec. III.B) runs the FDTD on the
GPU and returns the traces [n_probes][max_steps][2] (float32, CUDA); the
backward pass returns dL/dq from the library's adjoint
(``fdtd_adjoint_gradient``: the transposed leapfrog, Sec. III.A, run from the
last step to the first).  Argument marshalling only: the forward steps, the
transposed steps, the detector transpose and the deposit reduction are CUDA
kernels.  The traces are linear in q, so the backward pass needs no stored
forward state and no checkpoints.
"""
from __future__ import annotations

import numpy as np


class TraceModel:
    def __init__(self, sim, z0, bin_dz, v, lateral_w, L, steps):
        if steps > sim.max_steps:
            raise ValueError("steps exceed the trace capacity of the simulation")
        self.sim, self.z0, self.bin_dz, self.v, self.w, self.L = sim, z0, bin_dz, v, lateral_w, L
        self.steps = steps

    def _run(self, q):
        import torch
        s = self.sim
        s.reset()
        s.set_shower(np.ascontiguousarray(q.detach().double().cpu().numpy()), self.z0, self.bin_dz, self.v,
                     self.w, self.L)
        s.step(self.steps)
        out = torch.empty((s.np, s.max_steps, 2), dtype=torch.float32, device="cuda")
        return s.probes(out=out)

    def __call__(self, q):
        return _Traces.apply(q, self)


def _function():
    import torch

    class Traces(torch.autograd.Function):
        @staticmethod
        def forward(ctx, q, model):
            ctx.model = model
            ctx.q_device, ctx.q_dtype = q.device, q.dtype
            return model._run(q)

        @staticmethod
        def backward(ctx, g):
            m = ctx.model
            grad = m.sim.adjoint_gradient(g.detach().float().contiguous(), m.steps)
            return torch.from_numpy(grad).to(device=ctx.q_device, dtype=ctx.q_dtype), None

    return Traces


class _Lazy:
    fn = None

    @classmethod
    def apply(cls, *a):
        if cls.fn is None:
            cls.fn = _function()
        return cls.fn.apply(*a)


_Traces = _Lazy
