"""Fit PFB taps by gradient descent through the hand-written adjoint.

The loss is the out-of-band leakage of a tone set: stream i carries one tone
between the centres of channel k_i and its neighbour; the filter bank should
keep its energy in bins k_i - 1 .. k_i + 1 (the leakage and scalloping the
PFB exists to reduce, Sec. 2).  loss = mean_i E_out(i) / E_total(i).
"""
from __future__ import annotations

import time

import torch

from . import autograd, synth


def leakage_loss(Y: torch.Tensor, k) -> torch.Tensor:
    """Mean over streams of the energy outside bins k-1, k, k+1 over the total."""
    C = Y.shape[-1]
    P = (Y.real ** 2 + Y.imag ** 2).sum(dim=-2)           # (streams, C) energy per bin
    idx = torch.arange(C, device=Y.device)
    kk = torch.as_tensor(k, device=Y.device).reshape(-1, 1)
    dist = torch.remainder(idx.reshape(1, -1) - kk, C)
    inband = (dist <= 1) | (dist >= C - 1)
    total = P.sum(dim=-1)
    return ((P * (~inband)).sum(dim=-1) / total).mean()


def fit_taps(C: int = 256, T: int = 16, n_streams: int = 64, S: int = 8192, steps: int = 50, lr: float = 1e-3,
             noise: float = 1e-2, seed: int = 151103604, device="cuda") -> dict:
    """Adam on the taps; returns the loss history and the time per step."""
    x, k, _ = synth.tone_set(C, S + T - 1, n_streams, seed, device=device)
    m = autograd.PolyphaseFilterBank(C, T, synth.noisy_taps(C, T, noise, seed + 1)).to(device)
    opt = torch.optim.Adam(m.parameters(), lr=lr)
    hist = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        opt.zero_grad(set_to_none=True)
        loss = leakage_loss(m(x), k)
        loss.backward()
        opt.step()
        hist.append(float(loss.detach()))
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / max(1, steps)
    with torch.no_grad():
        clean = autograd.PolyphaseFilterBank(C, T, synth.design_taps(C, T)).to(device)
        ref = float(leakage_loss(clean(x), k))
    return {"loss": hist, "ms_per_step": dt * 1e3, "sinc_hamming_loss": ref, "taps": m.taps.detach().cpu()}
