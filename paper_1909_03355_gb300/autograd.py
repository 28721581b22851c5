"""torch.autograd wrapper of the FED-FEM forward run and its reverse-time adjoint.

trace = FedFemTrace.apply(kscale, source, fem, T0, n_steps, sensors, sample_every, ckpt_every)
runs n_steps explicit steps from T0 with per-element conductivity scales `kscale` and
volumetric sources `source` (1-D tensors over elements, original order), sampling the sensor
nodes after every `sample_every`-th step; backward() runs the adjoint and returns dL/dkscale
and dL/dsource.  The forward and the adjoint run in libfedfem.so's CUDA kernels.  With CUDA
tensors the parameters, the initial field (if given as a CUDA tensor), the trace and both
gradients stay on the device (fedfem_set_params_device, fedfem_forward_record_device,
fedfem_adjoint_device); CPU tensors take the host entry points.
"""
from __future__ import annotations

import numpy as np
import torch


class FedFemTrace(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kscale, source, fem, T0, n_steps, sensors, sample_every, ckpt_every):
        sensors = np.asarray(sensors, np.int32)
        ctx.fem = fem
        ctx.dev = kscale.device
        if kscale.is_cuda:
            fem.set_params_device(kscale.detach().to(torch.float64).contiguous(),
                                  source.detach().to(torch.float64).contiguous())
            if isinstance(T0, torch.Tensor) and T0.is_cuda:
                fem.set_T_device(T0.detach().to(torch.float64).contiguous())
            else:
                fem.set_T(np.asarray(T0.cpu() if isinstance(T0, torch.Tensor) else T0, dtype=np.float64))
            out = torch.empty((int(n_steps) // int(sample_every), len(sensors)), dtype=torch.float64,
                              device=kscale.device)
            return fem.forward_record_device(int(n_steps), sensors, int(sample_every), int(ckpt_every), out)
        fem.set_params(kscale.detach().double().numpy(), source.detach().double().numpy())
        fem.set_T(np.asarray(T0, dtype=np.float64))
        tr = fem.forward_record(int(n_steps), sensors, int(sample_every), int(ckpt_every))
        return torch.as_tensor(tr, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_trace):
        fem = ctx.fem
        if ctx.dev.type == "cuda":
            gk = torch.empty(fem.n_elems, dtype=torch.float64, device=ctx.dev)
            gs = torch.empty_like(gk)
            fem.adjoint_device(grad_trace.detach().to(torch.float64).contiguous(), gk, gs)
        else:
            gk_np, gs_np = fem.adjoint(grad_trace.detach().double().numpy())
            gk, gs = torch.as_tensor(gk_np), torch.as_tensor(gs_np)
        return gk, gs, None, None, None, None, None, None


def trace(kscale, source, fem, T0, n_steps, sensors, sample_every, ckpt_every):
    return FedFemTrace.apply(kscale, source, fem, T0, n_steps, sensors, sample_every, ckpt_every)
