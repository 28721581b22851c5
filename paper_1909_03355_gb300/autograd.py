"""torch.autograd wrapper of the FED-FEM forward run and its reverse-time adjoint.

trace = FedFemTrace.apply(kscale, source, fem, T0, n_steps, sensors, sample_every, ckpt_every)
runs n_steps explicit steps from T0 with per-element conductivity scales `kscale` and
volumetric sources `source` (1-D tensors over elements, original order), sampling the sensor
nodes after every `sample_every`-th step; backward() runs fedfem_adjoint and returns
dL/dkscale and dL/dsource.  The forward and the adjoint run in libfedfem.so's CUDA kernels;
torch only carries the tensors.
"""
from __future__ import annotations

import numpy as np
import torch


class FedFemTrace(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kscale, source, fem, T0, n_steps, sensors, sample_every, ckpt_every):
        fem.set_params(kscale.detach().double().cpu().numpy(), source.detach().double().cpu().numpy())
        fem.set_T(np.asarray(T0, dtype=np.float64))
        trace = fem.forward_record(int(n_steps), np.asarray(sensors, np.int32), int(sample_every), int(ckpt_every))
        ctx.fem = fem
        ctx.dev = kscale.device
        return torch.as_tensor(trace, dtype=torch.float64, device=kscale.device)

    @staticmethod
    def backward(ctx, grad_trace):
        gk, gs = ctx.fem.adjoint(grad_trace.detach().double().cpu().numpy())
        return (torch.as_tensor(gk, device=ctx.dev), torch.as_tensor(gs, device=ctx.dev),
                None, None, None, None, None, None)


def trace(kscale, source, fem, T0, n_steps, sensors, sample_every, ckpt_every):
    return FedFemTrace.apply(kscale, source, fem, T0, n_steps, sensors, sample_every, ckpt_every)
