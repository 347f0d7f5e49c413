"""PyTorch autograd front end of the engine's discrete adjoint.

``CNTraceFn.apply(gnabar, gkbar, gpas, model, tstop)`` runs the model from
step 0 to ``tstop`` with the given per-cell maximal conductances and returns
the recorded voltage traces as a tensor [n_rec, K+1]; its backward pass
calls ``cn_run_adjoint`` (reverse Hines solves and HH gate sensitivities on
the GPU, with checkpointed recompute) and returns gradients for the three
parameter tensors.  Marshalling only: all arithmetic runs in libcn.so.
"""
from __future__ import annotations

import numpy as np
import torch

from . import cn


class CNTraceFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gnabar, gkbar, gpas, model, tstop):
        model.cn_reset()
        for pid, t in ((cn.CN_PARAM_GNABAR, gnabar), (cn.CN_PARAM_GKBAR, gkbar), (cn.CN_PARAM_GPAS, gpas)):
            model.cn_set_cell_param(pid, t.detach().to("cpu", torch.float64).numpy())
        model.cn_run(float(tstop))
        model.cn_sync()
        tr = np.stack([model.cn_get_trace(r) for r in range(model.n_rec)])
        ctx.model = model
        ctx.device = gnabar.device
        return torch.from_numpy(tr).to(gnabar.device)

    @staticmethod
    def backward(ctx, grad_traces):
        g = ctx.model.cn_run_adjoint(grad_traces.detach().to("cpu", torch.float64).numpy())
        out = torch.from_numpy(g).to(ctx.device)
        return out[0], out[1], out[2], None, None


def trace_model(sc, checkpoint_ms=5.0, device=0):
    """A model of a scenario prepared for CNTraceFn (records, adjoint on)."""
    md = cn.from_scenario(sc, device=device, record=True)
    md.cn_enable_adjoint(max(1, int(round(checkpoint_ms / sc.dt))))
    return md
