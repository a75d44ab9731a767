"""Many beams (uneven C, T, spectrum counts) in one persistent launch.

``BeamSet`` wraps the ``ppf_beams_*`` calls of the C ABI; ``capture_graph``
records the queue reset + launch in a CUDA graph; ``autotune`` picks the tile
size and CTAs per SM by timing the actual beam set and caches the choice in a
JSON file keyed by the beam set's shape classes and the device name.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os

import numpy as np

from . import ppf

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json")


class BeamSet:
    """Beams i = 0..n-1 with C[i] channels, T[i] taps, S[i] output spectra, taps[i] (C*T FP32)."""

    def __init__(self, C, T, S, taps, in_dtype="ci8", out_dtype="c64"):
        n = len(C)
        if not (len(T) == len(S) == len(taps) == n):
            raise ValueError("C, T, S and taps must have the same length")
        self.C = [int(c) for c in C]
        self.T = [int(t) for t in T]
        self.S = [int(s) for s in S]
        self._taps = [np.ascontiguousarray(np.asarray(h, dtype=np.float32).reshape(-1)) for h in taps]
        for i in range(n):
            if self._taps[i].size != self.C[i] * self.T[i]:
                raise ValueError(f"beam {i}: expected {self.C[i] * self.T[i]} taps")
        Ca = (ctypes.c_int * n)(*self.C)
        Ta = (ctypes.c_int * n)(*self.T)
        Sa = (ctypes.c_longlong * n)(*self.S)
        Pa = (ctypes.POINTER(ctypes.c_float) * n)(*[h.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) for h in self._taps])
        self._h = None
        h = ctypes.c_void_p()
        ppf.check(ppf.lib().ppf_beams_plan(ctypes.byref(h), n, Ca, Ta, Sa, Pa, ppf.IN_CODES[in_dtype],
                                           ppf.OUT_CODES[out_dtype]))
        self._h = h
        self.n = n
        self.ctas_per_sm = 0
        self._bound = None

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("beam set is closed")
        return self._h

    def n_raw(self, i):
        return self.S[i] + self.T[i] - 1

    def samples(self) -> int:
        return sum(c * s for c, s in zip(self.C, self.S))

    def bytes_moved(self) -> int:
        """Algorithmic bytes of one launch: int8 complex in, complex FP32 out, FP32 taps."""
        return sum(c * (s + t - 1) * 2 + c * s * 8 + 4 * c * t for c, t, s in zip(self.C, self.T, self.S))

    def bind(self, ins, outs):
        """Device buffers per beam (torch CUDA tensors): int8 (n_raw*C, 2) in, complex64 (S, C) out."""
        ia = (ctypes.c_void_p * self.n)(*[x.data_ptr() for x in ins])
        oa = (ctypes.c_void_p * self.n)(*[y.data_ptr() for y in outs])
        ppf.check(ppf.lib().ppf_beams_bind(self.handle, ia, oa))
        self._bound = (list(ins), list(outs))

    def set_tiling(self, tile_samples: int):
        ppf.check(ppf.lib().ppf_beams_set_tiling(self.handle, int(tile_samples)))

    def execute(self, ctas_per_sm: int | None = None, stream=None):
        c = self.ctas_per_sm if ctas_per_sm is None else ctas_per_sm
        ppf.check(ppf.lib().ppf_beams_execute(self.handle, int(c), ppf._stream_handle(stream)))

    def info(self) -> dict:
        a = (ctypes.c_longlong * 7)()
        ppf.check(ppf.lib().ppf_beams_info(self.handle, a))
        return dict(zip(("beams", "tiles", "tile_samples", "max_ctas_per_sm", "sms", "smem", "wide_tiles"),
                        list(a)))

    def launches_per_execute(self) -> int:
        """Kernel launches one execute() enqueues: the one persistent launch (after a queue reset)."""
        return 1 if self.info()["tiles"] > 0 else 0

    def check_device(self, stream=None):
        ppf.check(ppf.lib().ppf_beams_check_device(self.handle, ppf._stream_handle(stream)))

    def capture_graph(self):
        """A CUDA graph of one execute (queue reset + the persistent launch)."""
        import torch
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.execute(stream=s)          # warm up outside capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.execute(stream=torch.cuda.current_stream())
        return g

    def signature(self) -> str:
        """Shape classes of the beam set (for the tuning cache)."""
        import torch
        classes = sorted((c, t, int(np.log2(max(s, 1)))) for c, t, s in zip(self.C, self.T, self.S))
        key = json.dumps([classes, torch.cuda.get_device_name()])
        return hashlib.sha1(key.encode()).hexdigest()[:16]

    def close(self):
        if self._h is not None:
            ppf.check(ppf.lib().ppf_beams_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _time(fn, reps=3):
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def autotune(bs: BeamSet, tile_candidates=(1 << 18, 1 << 19, 1 << 20, 1 << 21, 1 << 22),
             cache_path: str | None = DEFAULT_CACHE, use_cache: bool = True) -> dict:
    """Pick (tile_samples, ctas_per_sm) for this beam set by timing it; cache the choice."""
    sig = bs.signature()
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and sig in cache:
        best = cache[sig]
        bs.set_tiling(best["tile_samples"])
        bs.ctas_per_sm = best["ctas_per_sm"]
        return dict(best, cached=True)
    occ = bs.info()["max_ctas_per_sm"]
    trials = []
    for ts in tile_candidates:
        bs.set_tiling(ts)
        for c in range(1, occ + 1):
            ms = _time(lambda: bs.execute(ctas_per_sm=c))
            trials.append({"tile_samples": ts, "ctas_per_sm": c, "ms": ms})
    best = min(trials, key=lambda r: r["ms"])
    bs.set_tiling(best["tile_samples"])
    bs.ctas_per_sm = best["ctas_per_sm"]
    result = {"tile_samples": best["tile_samples"], "ctas_per_sm": best["ctas_per_sm"], "ms": best["ms"]}
    if cache_path:
        cache[sig] = result
        try:
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
        except OSError:
            pass
    return dict(result, cached=False, trials=trials)
