"""torch.autograd.Function over the C ABI: net production rates with hand-written
reverse mode (pyro_vjp) and forward mode (pyro_jvp).

    omega = NetProductionRates.apply(mech, rho, T, Y)       # [N, n]
    omega.backward(w_bar)     -> rho.grad, T.grad, Y.grad   (pyro_vjp)
    forward-mode AD with torch.autograd.forward_ad dual tensors -> d omega (pyro_jvp)

All tensors are float64 CUDA tensors in the library's layout (Y[k, p]).  The
backward of the backward is not provided (the VJP kernel is not itself
differentiable through torch).
"""
from __future__ import annotations

import torch

from . import binding as B


class NetProductionRates(torch.autograd.Function):
    """omega(rho, T, Y) of Eq. production_rates for a loaded mechanism."""

    @staticmethod
    def forward(mech: "B.Mechanism", rho, T, Y):
        return mech.net_production_rates(rho.contiguous(), Y.contiguous(), T=T.contiguous())

    @staticmethod
    def setup_context(ctx, inputs, output):
        mech, rho, T, Y = inputs
        ctx.mech = mech
        ctx.save_for_backward(rho, T, Y)
        ctx.save_for_forward(rho, T, Y)

    @staticmethod
    def backward(ctx, w_bar):
        rho, T, Y = ctx.saved_tensors
        rb, Tb, Yb = ctx.mech.vjp(rho.contiguous(), T.contiguous(), Y.contiguous(), w_bar.contiguous())
        return None, rb, Tb, Yb

    @staticmethod
    def jvp(ctx, _mech_t, d_rho, d_T, d_Y):
        rho, T, Y = ctx.saved_tensors
        z1 = lambda t, ref: torch.zeros_like(ref) if t is None else t.contiguous()
        return ctx.mech.jvp(rho.contiguous(), T.contiguous(), Y.contiguous(), z1(d_rho, rho), z1(d_T, T), z1(d_Y, Y))


def net_production_rates(mech: "B.Mechanism", rho, T, Y):
    """Differentiable omega [N, n] (reverse and forward mode through the library kernels)."""
    return NetProductionRates.apply(mech, rho, T, Y)
