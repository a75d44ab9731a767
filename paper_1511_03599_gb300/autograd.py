"""Differentiable polyphase filter bank: torch.autograd glue over the C ABI.

Forward and backward both run in the CUDA library (ppf_execute_batched and
ppf_backward); this module only orders the calls and hands tensors over.
Gradients follow PyTorch's convention for complex tensors (dL/dRe + i dL/dIm).
"""
from __future__ import annotations

import torch

from . import ppf


class _PFBFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, taps, plan, n_streams):
        plan.update_taps(taps)
        y = plan.execute(x, n_streams=n_streams)
        ctx.plan = plan
        ctx.n_streams = n_streams
        ctx.save_for_backward(x, taps)
        return y

    @staticmethod
    def backward(ctx, gy):
        x, taps = ctx.saved_tensors
        plan = ctx.plan
        plan.update_taps(taps)      # a later forward may have changed the plan's taps
        gx, gh = plan.backward(gy.contiguous(), x, want_input=ctx.needs_input_grad[0],
                               want_taps=ctx.needs_input_grad[1])
        if gh is not None:
            gh = gh.view_as(taps)
        return gx, gh, None, None


class PolyphaseFilterBank(torch.nn.Module):
    """PFB with learnable taps (C*T FP32, tap-major h[t*C + c]) on complex64 input.

    forward(x): x is complex64 of shape (n_raw*C,) or (streams, n_raw*C) /
    (streams, n_raw, C); returns (S, C) or (streams, S, C) complex64.
    """

    def __init__(self, C: int, T: int, taps):
        super().__init__()
        self.C, self.T = int(C), int(T)
        t = torch.as_tensor(taps, dtype=torch.float32).reshape(-1).clone()
        self.taps = torch.nn.Parameter(t)
        self._plan = None

    def plan(self):
        if self._plan is None:
            self._plan = ppf.Plan(self.C, self.T, self.taps.detach().cpu().numpy(), "cf32", "c64")
        return self._plan

    def forward(self, x):
        if x.dtype != torch.complex64:
            raise TypeError("PolyphaseFilterBank takes complex64 input")
        batched = x.dim() >= 2
        xs = x.contiguous()
        n_streams = xs.shape[0] if batched else None
        return _PFBFunction.apply(xs, self.taps, self.plan(), n_streams)
