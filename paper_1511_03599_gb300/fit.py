"""Fit PFB taps by gradient descent through the hand-written adjoint.

The loss is the out-of-band leakage of a tone set: stream i carries one tone
between the centres of channel k_i and its neighbour; the filter bank should
keep its energy in bins k_i - 1 .. k_i + 1 (the leakage and scalloping the
PFB exists to reduce, Sec. 2).  loss = mean_i E_out(i) / E_total(i).

``fit_taps`` runs each step as four explicit phases on the current stream --
forward (ppf_execute_batched), loss and its closed-form gradient wrt the
spectra, adjoint (ppf_backward, tap gradient only) and the Adam update --
and times each with CUDA events.  ``leakage_loss`` is the same loss written
for torch.autograd (used with the autograd module).
"""
from __future__ import annotations

import math
import time

import torch

from . import autograd, ppf, synth


def _inband(k, C: int, device) -> torch.Tensor:
    """(streams, C) bool: bins k-1, k, k+1 (mod C) of each stream's tone."""
    idx = torch.arange(C, device=device)
    kk = torch.as_tensor(k, device=device).reshape(-1, 1)
    dist = torch.remainder(idx.reshape(1, -1) - kk, C)
    return (dist <= 1) | (dist >= C - 1)


def leakage_loss(Y: torch.Tensor, k) -> torch.Tensor:
    """Mean over streams of the energy outside bins k-1, k, k+1 over the total."""
    C = Y.shape[-1]
    P = (Y.real ** 2 + Y.imag ** 2).sum(dim=-2)           # (streams, C) energy per bin
    inband = _inband(k, C, Y.device)
    total = P.sum(dim=-1)
    return ((P * (~inband)).sum(dim=-1) / total).mean()


def leakage_loss_and_grad(Y: torch.Tensor, inband: torch.Tensor, gY: torch.Tensor | None = None):
    """The leakage loss of Y (streams, S, C) and its gradient wrt Y in PyTorch's
    convention (dL/dRe + i dL/dIm), in closed form:

        P[i][m] = sum_s |Y[i][s][m]|^2,  L_i = E_out(i) / E_tot(i),  L = mean_i L_i,
        dL/dP[i][m] = (out[i][m] - L_i) / (n E_tot(i)),  grad_Y = 2 Y dL/dP.

    One pass over Y for P, one for the gradient (written into ``gY`` if given).
    """
    n = Y.shape[0]
    Yr = torch.view_as_real(Y)
    P = torch.linalg.vector_norm(Yr, ord=2, dim=(1, 3)).double().square()   # (streams, C), no temporary
    out = (~inband).to(torch.float64)
    e_tot = P.sum(dim=-1)
    e_out = (P * out).sum(dim=-1)
    Li = e_out / e_tot
    dP = ((out - Li[:, None]) / (n * e_tot[:, None])).to(torch.float32)
    if gY is None:
        gY = torch.empty_like(Y)
    torch.mul(Yr, (2.0 * dP)[:, None, :, None], out=torch.view_as_real(gY))
    return Li.mean(), gY


def fit_taps(C: int = 256, T: int = 16, n_streams: int = 64, S: int = 8192, steps: int = 300, lr: float = 2e-3,
             lr_final: float = 1e-6, noise: float = 1e-2, seed: int = 151103604, device="cuda") -> dict:
    """Adam (cosine-decayed learning rate) on the taps; returns the loss history,
    the time per step and its split over the four phases (ms, CUDA events)."""
    x, k, _ = synth.tone_set(C, S + T - 1, n_streams, seed, device=device)
    h0 = synth.noisy_taps(C, T, noise, seed + 1)
    taps = torch.tensor(h0, dtype=torch.float32, device=device)
    inband = _inband(k, C, device)
    plan = ppf.Plan(C, T, h0, "cf32", "c64")
    st = torch.cuda.current_stream()
    y = plan.empty_output(S, device=device, n_streams=n_streams)
    gY = torch.empty_like(y)
    m = torch.zeros_like(taps)
    v = torch.zeros_like(taps)
    b1, b2, eps = 0.9, 0.999, 1e-8
    names = ("forward", "loss_and_grad", "adjoint", "adam")
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)] for _ in range(steps)]
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        e = ev[i]
        e[0].record(st)
        plan.update_taps(taps, stream=st)
        plan.execute(x, out=y, n_streams=n_streams, stream=st)
        e[1].record(st)
        loss, _ = leakage_loss_and_grad(y, inband, gY)
        e[2].record(st)
        _, gh = plan.backward(gY, x, want_input=False, stream=st)
        e[3].record(st)
        a = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * i / max(1, steps - 1)))
        m.mul_(b1).add_(gh, alpha=1 - b1)
        v.mul_(b2).addcmul_(gh, gh, value=1 - b2)
        mh = m / (1 - b1 ** (i + 1))
        vh = v / (1 - b2 ** (i + 1))
        taps.addcdiv_(mh, vh.sqrt_().add_(eps), value=-a)
        e[4].record(st)
        losses.append(loss)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / max(1, steps)
    plan.check_device()
    hist = [float(l) for l in losses]
    skip = min(2, steps - 1)                   # first steps include one-time set-up
    phase = {n: sum(ev[i][j].elapsed_time(ev[i][j + 1]) for i in range(skip, steps)) / (steps - skip)
             for j, n in enumerate(names)}
    step_ms = sum(ev[i][0].elapsed_time(ev[i][-1]) for i in range(skip, steps)) / (steps - skip)
    with torch.no_grad():
        clean = autograd.PolyphaseFilterBank(C, T, synth.design_taps(C, T)).to(device)
        ref = float(leakage_loss(clean(x), k))
    plan.close()
    return {"loss": hist, "ms_per_step": step_ms, "wall_ms_per_step": wall * 1e3, "phase_ms": phase,
            "steps": steps, "optimizer": f"Adam lr {lr:g} cosine-decayed to {lr_final:g}",
            "sinc_hamming_loss": ref, "taps": taps.detach().cpu()}
