"""Seeded synthetic inputs and filter-coefficient design.

This module is shared by the tests, the benchmark and the oracle's callers.
It holds no arithmetic of the polyphase filter itself (no FIR, no DFT); it
only produces the numbers that go *into* it:

* ``design_taps``   -- sinc x window prototype filter of length C*T, designed
  in FP64 and rounded once to FP32 (Sec. 2: coefficients from a sinc
  multiplied by a window; Sec. 3.1: coefficients are stored as 32-bit floats).
* ``stream``        -- complex sample streams, "contiguous in channels"
  (Sec. 3.1), interleaved (re, im) pairs of int8 / int16 / fp32.
* ``workload``      -- the named workloads (sizes, distributions, tones, seeds).

Readings where the paper is silent (seed, window, sigma, tone) are fixed here
and listed in the design notes of the repository.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 151103599

IN_DTYPES = ("ci8", "ci16", "cf32")
OUT_DTYPES = ("c64", "c16")
_IN_NP = {"ci8": np.int8, "ci16": np.int16, "cf32": np.float32}
_IN_LIMIT = {"ci8": 127, "ci16": 32767}


def in_bytes_per_sample(in_dtype: str) -> int:
    """Bytes of one complex input sample (re and im)."""
    return {"ci8": 2, "ci16": 4, "cf32": 8}[in_dtype]


def out_bytes_per_sample(out_dtype: str) -> int:
    """Bytes of one complex output sample (re and im)."""
    return {"c64": 8, "c16": 4}[out_dtype]


def design_taps(C: int, T: int, window: str = "hamming", scale: float = 1.0) -> np.ndarray:
    """Prototype low-pass filter of length C*T, FP32, tap-major h[t*C + c].

    h[n] = sinc((n - (CT-1)/2) / C) * w[n],  n = 0 .. CT-1, sinc(x) = sin(pi x)/(pi x):
    the sinc has its zeros every C samples (cut-off at one channel width) and
    w is a Hamming (0.54 - 0.46 cos) or Hanning (0.5 - 0.5 cos) window of the
    same length (Sec. 2, coefficient figure).  No normalisation.  ``scale``
    multiplies the FP64 design before the single rounding to FP32.
    """
    if C < 1 or T < 1:
        raise ValueError("C and T must be >= 1")
    n = np.arange(C * T, dtype=np.float64)
    L = C * T
    if L > 1:
        phase = 2.0 * np.pi * n / (L - 1)
        if window == "hamming":
            w = 0.54 - 0.46 * np.cos(phase)
        elif window == "hanning":
            w = 0.5 - 0.5 * np.cos(phase)
        elif window == "rect":
            w = np.ones(L)
        else:
            raise ValueError(f"unknown window {window!r}")
    else:
        w = np.ones(1)
    h = np.sinc((n - (L - 1) / 2.0) / C) * w * scale
    return h.astype(np.float32)


def _quantise(z: np.ndarray, in_dtype: str) -> np.ndarray:
    """Complex128 -> interleaved (N, 2) array of the input type.

    Integers: round half to even, then clip to +-(2^(b-1)-1); fp32: one rounding.
    """
    out = np.empty((z.shape[0], 2), dtype=_IN_NP[in_dtype])
    if in_dtype == "cf32":
        out[:, 0] = z.real.astype(np.float32)
        out[:, 1] = z.imag.astype(np.float32)
    else:
        lim = _IN_LIMIT[in_dtype]
        out[:, 0] = np.clip(np.rint(z.real), -lim, lim).astype(_IN_NP[in_dtype])
        out[:, 1] = np.clip(np.rint(z.imag), -lim, lim).astype(_IN_NP[in_dtype])
    return out


def stream(C: int, n_raw: int, in_dtype: str, sigma: float, seed: int,
           tones: tuple = (), chunk: int = 1 << 24) -> np.ndarray:
    """Seeded stream of ``n_raw`` raw spectra of C channels, shape (n_raw*C, 2).

    Per component re, im ~ N(0, sigma^2) independently (numpy PCG64), plus
    tones ``(channel k0, amplitude A)``: A * exp(+2 pi i k0 n / C) with n the
    global sample index from 0 (a tone at the centre of channel k0).
    Generated in chunks so multi-GB streams do not need a complex128 copy.
    """
    if in_dtype not in IN_DTYPES:
        raise ValueError(f"unknown input dtype {in_dtype!r}")
    N = int(C) * int(n_raw)
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((N, 2), dtype=_IN_NP[in_dtype])
    for lo in range(0, N, chunk):
        hi = min(N, lo + chunk)
        m = hi - lo
        re = rng.standard_normal(m) * sigma
        im = rng.standard_normal(m) * sigma
        z = re + 1j * im
        if tones:
            n = np.arange(lo, hi, dtype=np.int64)
            for k0, amp in tones:
                # integer phase reduction keeps the angle exact for long streams
                ph = ((n * int(k0)) % C).astype(np.float64) * (2.0 * np.pi / C)
                z += amp * np.exp(1j * ph)
        out[lo:hi] = _quantise(z, in_dtype)
    return out


def impulse_stream(C: int, n_raw: int, in_dtype: str, r: int, c0: int, value=1) -> np.ndarray:
    """All-zero stream with a single real sample ``value`` at raw spectrum r, channel c0."""
    out = np.zeros((C * n_raw, 2), dtype=_IN_NP[in_dtype])
    out[r * C + c0, 0] = value
    return out


@dataclass
class Workload:
    """A named workload: sizes, input recipe and taps."""
    name: str
    C: int
    T: int
    S: int
    in_dtype: str
    out_dtype: str
    sigma: float
    seed: int
    tones: tuple = ()
    tap_scale: float = 1.0

    @property
    def n_raw(self) -> int:
        return self.S + self.T - 1

    def taps(self) -> np.ndarray:
        return design_taps(self.C, self.T, "hamming", self.tap_scale)

    def input(self, S: int | None = None) -> np.ndarray:
        """The stream; with ``S`` given, only the raw spectra of the first S outputs."""
        n_raw = self.n_raw if S is None else S + self.T - 1
        return stream(self.C, n_raw, self.in_dtype, self.sigma, self.seed, self.tones)

    def describe(self) -> dict:
        return {"workload": self.name, "C": self.C, "T": self.T, "spectra": self.S,
                "in": self.in_dtype, "out": self.out_dtype, "sigma": self.sigma,
                "tones": [list(t) for t in self.tones], "taps": "sinc-hamming fp32"
                + ("" if self.tap_scale == 1.0 else f" x{self.tap_scale:.6g}")}


def small_parity_workload() -> Workload:
    """C=256, T=8, 4096 spectra, c64 noise sigma=1 + 0.5 tone at channel 37."""
    return Workload("pfb_c256_t8_s4096_cf32", 256, 8, 4096, "cf32", "c64", 1.0,
                    SEED_BASE + 0, ((37, 0.5),))


def target_workload(in_dtype: str = "ci8", S: int = 1 << 20) -> Workload:
    """C=512, T=8, 2^20 spectra; int8 sigma=16 (+ tone ch 101, amp 32) or fp32 sigma=1."""
    if in_dtype == "ci8":
        return Workload(f"pfb_c512_t8_s{S}_ci8_c64", 512, 8, S, "ci8", "c64", 16.0,
                        SEED_BASE + 1, ((101, 32.0),))
    if in_dtype == "cf32":
        return Workload(f"pfb_c512_t8_s{S}_cf32_c64", 512, 8, S, "cf32", "c64", 1.0,
                        SEED_BASE + 1 + 100, ((101, 2.0),))
    if in_dtype == "ci16":
        return Workload(f"pfb_c512_t8_s{S}_ci16_c64", 512, 8, S, "ci16", "c64", 2000.0,
                        SEED_BASE + 1 + 200, ((101, 4000.0),))
    raise ValueError(in_dtype)


def sweep_workload(T: int, in_dtype: str, out_dtype: str, S: int = 1 << 18) -> Workload:
    """C=512 tap/precision sweep cell; c16 cells scale the taps by 1/sqrt(C)."""
    Ts = (8, 16, 32, 64)
    ti = Ts.index(T) if T in Ts else 0
    di = {"ci16": 0, "cf32": 1}[in_dtype]
    sigma = 2000.0 if in_dtype == "ci16" else 1.0
    scale = 1.0 / math.sqrt(512) if out_dtype == "c16" else 1.0
    return Workload(f"pfb_c512_t{T}_s{S}_{in_dtype}_{out_dtype}", 512, T, S, in_dtype,
                    out_dtype, sigma, SEED_BASE + 2 + 1000 * ti + di, (), scale)


def stream_torch(C: int, n_raw: int, in_dtype: str, sigma: float, seed: int, tones: tuple = (),
                 device="cuda", chunk: int = 1 << 26):
    """The ``stream`` recipe drawn with torch's generator on ``device`` (fast for GB-sized
    benchmark inputs).  Same distribution, quantisation and tones as ``stream``; the
    random numbers differ from numpy's, so parity tests use ``stream``."""
    import torch
    N = int(C) * int(n_raw)
    tdt = {"ci8": torch.int8, "ci16": torch.int16, "cf32": torch.float32}[in_dtype]
    out = torch.empty((N, 2), dtype=tdt, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    for lo in range(0, N, chunk):
        hi = min(N, lo + chunk)
        z = torch.randn((hi - lo, 2), generator=g, device=device, dtype=torch.float32) * sigma
        if tones:
            n = torch.arange(lo, hi, device=device, dtype=torch.int64)
            for k0, amp in tones:
                ph = ((n * int(k0)) % C).to(torch.float32) * (2.0 * math.pi / C)
                z[:, 0] += amp * torch.cos(ph)
                z[:, 1] += amp * torch.sin(ph)
        if in_dtype == "cf32":
            out[lo:hi] = z
        else:
            lim = _IN_LIMIT[in_dtype]
            out[lo:hi] = torch.clamp(torch.round(z), -lim, lim).to(tdt)
    return out


def tone_set(C: int, n_raw: int, n_streams: int, seed: int, device="cuda"):
    """One tone per stream for fitting taps: stream i carries
    exp(+2 pi i (k_i + d_i) n / C), k_i a channel, d_i in +-{0.1, 0.2, 0.3, 0.45}
    (between bin centres, where leakage and scalloping are largest, Sec. 2).
    Returns (x complex64 of shape (n_streams, n_raw*C), k, d)."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    k = rng.integers(0, C, n_streams)
    d = rng.choice([-0.45, -0.3, -0.2, -0.1, 0.1, 0.2, 0.3, 0.45], n_streams)
    n = torch.arange(n_raw * C, device=device, dtype=torch.float64)
    xs = []
    for ki, di in zip(k, d):
        ph = torch.remainder(n * (float(ki) + float(di)) / C, 1.0) * (2 * math.pi)
        xs.append(torch.polar(torch.ones_like(ph), ph).to(torch.complex64))
    return torch.stack(xs), k, d


def noisy_taps(C: int, T: int, noise: float, seed: int) -> np.ndarray:
    """sinc-Hamming taps plus seeded Gaussian noise of the given standard deviation (FP32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (design_taps(C, T).astype(np.float64) + noise * rng.standard_normal(C * T)).astype(np.float32)
