"""FP64 CPU oracle for the polyphase filter bank (PFB).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import or call
this module: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA path.

Plain, slow, obviously correct: every quantity is upcast exactly to FP64
(int8/int16/fp32 samples and FP32 coefficients are all exact in FP64) and
the two steps of the PFB are written as their definitions:

* FIR (Alg. 1, Sec. 3.2; the index convention of Alg. 2/3, which Eq. 1's
  garbled index is read to mean):
      y[s][c] = sum_{t=0}^{T-1} h[t*C + c] * x[(s+t)*C + c],   0 <= s < S, 0 <= c < C
  with S = n_raw - T + 1 outputs (no zero-padded history).
* DFT (Eq. 2, Sec. 2), unnormalised, sign -i, natural bin order:
      Y[s][m] = sum_{c=0}^{C-1} y[s][c] * exp(-2 pi i (c*m mod C) / C)
  The integer product c*m is reduced mod C before the FP64 angle is formed.

Also here: the adjoint of that linear map (the gradients used to fit taps),
the effective-FLOP count of the FIR (Sec. 4.1) and the read/write efficiency
epsilon (Sec. 4.1).  Parity of the FIR/DFT against the paper's own numeric
outputs is unpinned: the paper prints none; these functions are pinned by the
CPU tests against brute force, closed forms, invariants and library routines.
"""
from __future__ import annotations

import numpy as np


def as_complex(x_raw: np.ndarray) -> np.ndarray:
    """Interleaved (N, 2) int8/int16/fp32 samples -> complex128, value taken as-is.

    Integers are two's complement with no offset or scale (Sec. 3.1 input
    precisions, read as signed); every value is exact in FP64.
    """
    x_raw = np.asarray(x_raw)
    if x_raw.ndim != 2 or x_raw.shape[1] != 2:
        raise ValueError("expected interleaved (N, 2) samples")
    return x_raw[:, 0].astype(np.float64) + 1j * x_raw[:, 1].astype(np.float64)


def fir(x: np.ndarray, h: np.ndarray, C: int, T: int) -> np.ndarray:
    """Per-channel T-tap FIR (Alg. 1): returns y of shape (S, C), complex128.

    ``x`` is complex (length C*(S+T-1)) or interleaved raw samples.
    ``h`` holds C*T real coefficients, tap-major: h[t*C + c].
    """
    if x.ndim == 2:
        x = as_complex(x)
    h = np.asarray(h, dtype=np.float64)
    if h.shape != (C * T,):
        raise ValueError("h must have C*T coefficients")
    if x.shape[0] % C:
        raise ValueError("stream length must be a multiple of C")
    n_raw = x.shape[0] // C
    S = n_raw - T + 1
    if S < 1:
        return np.zeros((0, C), dtype=np.complex128)
    X = x.reshape(n_raw, C)
    H = h.reshape(T, C)
    y = np.zeros((S, C), dtype=np.complex128)
    for t in range(T):                      # Alg. 1 inner loop, t ascending
        y += H[t][None, :] * X[t:t + S, :]
    return y


def dft_matrix(C: int) -> np.ndarray:
    """W[c][m] = exp(-2 pi i ((c*m) mod C) / C), FP64 (Eq. 2)."""
    c = np.arange(C, dtype=np.int64)
    e = np.outer(c, c) % C
    return np.exp(-2j * np.pi * e.astype(np.float64) / C)


def dft(y: np.ndarray, chunk: int = 4096) -> np.ndarray:
    """Unnormalised C-point DFT of every row of y (Eq. 2), naive O(C^2) per row."""
    S, C = y.shape
    W = dft_matrix(C)
    Y = np.empty((S, C), dtype=np.complex128)
    for lo in range(0, S, chunk):
        Y[lo:lo + chunk] = y[lo:lo + chunk] @ W
    return Y


def pfb(x: np.ndarray, h: np.ndarray, C: int, T: int) -> np.ndarray:
    """Raw spectra -> filtered spectra -> frequency spectra (Sec. 2): (S, C) complex128."""
    return dft(fir(x, h, C, T))


def pfb_spectra(x: np.ndarray, h: np.ndarray, C: int, T: int, spectra) -> np.ndarray:
    """PFB output rows for the listed output spectra only (for sampled parity checks).

    Output spectrum s depends on raw spectra s .. s+T-1 only, so each row is
    the PFB of that slice of the stream.
    """
    rows = [fir(x[s * C:(s + T) * C], h, C, T)[0] for s in np.asarray(spectra, dtype=np.int64)]
    return dft(np.stack(rows)) if rows else np.zeros((0, C), np.complex128)


# --------------------------------------------------------------------------
# Adjoint (gradients), conjugate-Wirtinger convention of PyTorch: for a real
# loss L and complex z, grad_z = dL/dRe(z) + i dL/dIm(z).
# --------------------------------------------------------------------------

def idft_unnormalised(G: np.ndarray, chunk: int = 4096) -> np.ndarray:
    """g_y = F^H g_Y: the adjoint of Eq. 2 (sign +i, no 1/C)."""
    S, C = G.shape
    Wh = np.conj(dft_matrix(C)).T
    out = np.empty((S, C), dtype=np.complex128)
    for lo in range(0, S, chunk):
        out[lo:lo + chunk] = G[lo:lo + chunk] @ Wh
    return out


def pfb_grad_input(gY: np.ndarray, h: np.ndarray, C: int, T: int) -> np.ndarray:
    """grad_x[(s+t)C + c] = sum over (s, t) of h[tC + c] * g_y[s][c]; length C*(S+T-1)."""
    gy = idft_unnormalised(gY)
    S = gy.shape[0]
    H = np.asarray(h, dtype=np.float64).reshape(T, C)
    gx = np.zeros((S + T - 1, C), dtype=np.complex128)
    for t in range(T):
        gx[t:t + S, :] += H[t][None, :] * gy
    return gx.reshape(-1)


def pfb_grad_taps(gY: np.ndarray, x: np.ndarray, C: int, T: int) -> np.ndarray:
    """grad_h[tC + c] = sum_s Re(conj(g_y[s][c]) * x[(s+t)C + c]); length C*T, FP64."""
    if x.ndim == 2:
        x = as_complex(x)
    gy = idft_unnormalised(gY)
    S = gy.shape[0]
    X = x.reshape(-1, C)
    gh = np.zeros((T, C), dtype=np.float64)
    for t in range(T):
        gh[t] = np.sum((np.conj(gy) * X[t:t + S, :]).real, axis=0)
    return gh.reshape(-1)


# --------------------------------------------------------------------------
# Reporting arithmetic (Sec. 4.1)
# --------------------------------------------------------------------------

def fir_effective_flops(S: int, C: int, T: int) -> int:
    """Effective FLOPs of the FIR: 2*S*C*T multiplications + 2*S*C*(T-1) additions.

    The factor 2 is for complex samples times real coefficients (Sec. 4.1).
    Divided by an execution time it gives F_FIR in FLOP/s.
    """
    return 2 * S * C * T + 2 * S * C * (T - 1)


def efficiency(S: int, T: int) -> float:
    """Ideal written/read ratio for S filtered spectra: S / (S + T - 1) (Sec. 4.1)."""
    return S / (S + T - 1)


def rel_l2_max_per_spectrum(a: np.ndarray, ref: np.ndarray) -> float:
    """max over spectra s of ||a[s] - ref[s]||_2 / ||ref[s]||_2, in FP64.

    ``a`` and ``ref`` have shape (..., C) (the last axis is the bins of one
    spectrum).  A spectrum whose reference is all zero contributes its
    absolute error norm.
    """
    a = np.asarray(a).astype(np.complex128)
    ref = np.asarray(ref).astype(np.complex128)
    if a.shape != ref.shape or a.ndim < 1:
        raise ValueError("a and ref must have the same shape (..., C)")
    if a.size == 0:
        return 0.0
    C = ref.shape[-1]
    num = np.linalg.norm((a - ref).reshape(-1, C), axis=1)
    den = np.linalg.norm(ref.reshape(-1, C), axis=1)
    r = np.where(den > 0, num / np.where(den > 0, den, 1.0), num)
    return float(np.max(r))


def rel_l2(a: np.ndarray, ref: np.ndarray) -> float:
    """||a - ref||_2 / ||ref||_2 over all elements, evaluated in FP64."""
    a = np.asarray(a).astype(np.complex128).ravel()
    ref = np.asarray(ref).astype(np.complex128).ravel()
    den = np.linalg.norm(ref)
    num = np.linalg.norm(a - ref)
    return float(num / den) if den > 0 else float(num)
