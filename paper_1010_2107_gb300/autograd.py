"""torch.autograd.Function over the adjoint pass (vegas_grad in include/gvegas.h).

The value is the iteration estimate I(theta) of one pass on a frozen grid
with the random numbers of a fixed Philox iteration (common random numbers),
so I is a smooth function of theta and its gradient is the estimator of
dI/dtheta the adjoint kernel computes: (1/NCALL) sum_s J_s df/dtheta(x_s).
Both come from one adjoint pass in forward(); backward() scales the stored
gradient.  Argument marshalling only: the arithmetic runs in the CUDA
library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import gvegas as gv
from . import workloads as wl


def theta_slots(kind: int, ndim: int):
    """Indices into the integrand's parameter vector of theta, in the order of
    vegas_grad: (M, Gamma, T) for RAMBO_BW, (c1, c2, w) for DOUBLE_GAUSSIAN,
    (u_1..u_d, a_1..a_d) for GENZ_GAUSSIAN."""
    if kind == wl.RAMBO_BW:
        return [wl.RB_M, wl.RB_GAMMA, wl.RB_T]
    if kind == wl.DOUBLE_GAUSSIAN:
        return [0, 1, 2]
    if kind == wl.GENZ_GAUSSIAN:
        return list(range(ndim, 2 * ndim)) + list(range(ndim))
    raise ValueError("no adjoint for this integrand kind")


class VegasEstimate(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, ctx, it, params, slots):
        p = np.array(params, dtype=np.float64, copy=True)
        p[slots] = theta.detach().to("cpu", torch.float64).numpy()
        gv.vegas_set_params(ctx, p)
        grad, I = gv.vegas_grad(ctx, it)
        fctx.save_for_backward(torch.as_tensor(grad, dtype=theta.dtype, device=theta.device))
        return torch.as_tensor(I, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(fctx, gout):
        (g,) = fctx.saved_tensors
        return gout * g, None, None, None, None


def vegas_estimate(theta: torch.Tensor, ctx: gv.Context, it: int, params, kind: int) -> torch.Tensor:
    """I(theta) with autograd support; `params` is the full parameter vector
    whose theta slots are replaced by `theta`."""
    return VegasEstimate.apply(theta, ctx, int(it), np.asarray(params, np.float64),
                               theta_slots(kind, ctx.ndim))
