"""Python binding of the C ABI in ``include/ppf.h`` (ctypes; argument marshalling only).

Every step of the transform runs in the CUDA library ``libppf.so``; PyTorch
supplies device memory and the current stream.  There is no CPU fallback:
if the library is missing, every call raises.

    plan = Plan(C=512, T=8, taps=h, in_dtype="ci8", out_dtype="c64")
    Y = plan(x)            # x: CUDA tensor of C*(S+T-1) samples -> (S, C) complex64
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libppf.so")

PPF_OK = 0
STATUS_NAMES = {0: "PPF_OK", 1: "PPF_ERR_INVALID_ARG", 2: "PPF_ERR_UNSUPPORTED", 3: "PPF_ERR_ALIGNMENT",
                4: "PPF_ERR_CUDA", 5: "PPF_ERR_DEVICE_TIMEOUT", 6: "PPF_ERR_OUT_OF_MEMORY"}
IN_CODES = {"ci8": 0, "ci16": 1, "cf32": 2}
OUT_CODES = {"c64": 0, "c16": 1}

# exported symbols and their ctypes signatures (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "ppf_plan": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                ctypes.c_int, ctypes.c_int]),
    "ppf_execute": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong, _P]),
    "ppf_execute_batched": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P, ctypes.c_longlong, ctypes.c_longlong,
                                           ctypes.c_longlong, _P]),
    "ppf_backward": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_longlong, ctypes.c_longlong, _P]),
    "ppf_update_taps": (ctypes.c_int, [_P, _P, _P]),
    "ppf_fir": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong, _P]),
    "ppf_beams_plan": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.POINTER(ctypes.c_float)), ctypes.c_int, ctypes.c_int]),
    "ppf_beams_bind": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "ppf_beams_set_tiling": (ctypes.c_int, [_P, ctypes.c_longlong]),
    "ppf_beams_execute": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "ppf_beams_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    "ppf_beams_check_device": (ctypes.c_int, [_P, _P]),
    "ppf_beams_destroy": (ctypes.c_int, [_P]),
    "ppf_fft": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong, _P]),
    "ppf_backward_noalloc": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_longlong, ctypes.c_longlong, _P]),
    "ppf_execute_host": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong, _P]),
    "ppf_destroy": (ctypes.c_int, [_P]),
    "ppf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ppf_last_error_message": (ctypes.c_char_p, []),
    "ppf_plan_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "ppf_check_device": (ctypes.c_int, [_P, _P]),
    "ppf_set_debug_flags": (ctypes.c_int, [_P, ctypes.c_int]),
    "ppf_probe_rates": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "ppf_probe_stream": (ctypes.c_int, [_P, _P, ctypes.c_longlong, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
}

_lib = None


class PPFError(RuntimeError):
    """A non-OK status from the C ABI."""

    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")


def lib() -> ctypes.CDLL:
    """Load libppf.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1511_03599_gb300._build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != PPF_OK:
        msg = lib().ppf_last_error_message()
        raise PPFError(status, msg.decode() if msg else "")


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


_TORCH_IN = {"ci8": "int8", "ci16": "int16", "cf32": "float32"}


def bytes_per_sample(in_dtype: str) -> int:
    return {"ci8": 2, "ci16": 4, "cf32": 8}[in_dtype]


class Plan:
    """A PFB plan: C channels, T taps, FP32 coefficients h[t*C + c], input/output types."""

    def __init__(self, C: int, T: int, taps, in_dtype: str = "ci8", out_dtype: str = "c64"):
        if in_dtype not in IN_CODES or out_dtype not in OUT_CODES:
            raise ValueError(f"unknown dtype pair {in_dtype!r}, {out_dtype!r}")
        if hasattr(taps, "detach"):
            taps = taps.detach().cpu().numpy()
        h = np.ascontiguousarray(np.asarray(taps, dtype=np.float32).reshape(-1))
        if h.size != C * T:
            raise ValueError(f"expected {C * T} coefficients, got {h.size}")
        self.C, self.T, self.in_dtype, self.out_dtype = int(C), int(T), in_dtype, out_dtype
        self._h = None
        handle = ctypes.c_void_p()
        check(lib().ppf_plan(ctypes.byref(handle), self.C, self.T,
                             h.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                             IN_CODES[in_dtype], OUT_CODES[out_dtype]))
        self._h = handle

    # ------------------------------------------------------------------
    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan is closed")
        return self._h

    def info(self) -> dict:
        a = (ctypes.c_int * 8)()
        check(lib().ppf_plan_info(self.handle, a))
        keys = ("threads", "batch", "grid", "smem", "tap_bucket", "fft_stages", "variant", "ctas_per_sm")
        return dict(zip(keys, list(a)))

    def n_spectra_for(self, x) -> int:
        """Output spectra for one stream of interleaved samples (the last dimensions of x)."""
        n_samples = x.numel() if x.is_complex() else x.numel() // 2
        if n_samples % self.C:
            raise ValueError("input length is not a whole number of raw spectra")
        return n_samples // self.C - self.T + 1

    def empty_output(self, n_spectra: int, device=None, n_streams: int | None = None):
        import torch
        lead = () if n_streams is None else (n_streams,)
        if self.out_dtype == "c64":
            return torch.empty(lead + (n_spectra, self.C), dtype=torch.complex64, device=device)
        return torch.empty(lead + (n_spectra, self.C, 2), dtype=torch.float16, device=device)

    def _check_input(self, x):
        import torch
        want = getattr(torch, _TORCH_IN[self.in_dtype])
        ok = x.dtype == want or (self.in_dtype == "cf32" and x.dtype == torch.complex64)
        if not ok:
            raise TypeError(f"input dtype {x.dtype} does not match plan input {self.in_dtype}")
        if not x.is_contiguous():
            raise ValueError("input must be contiguous")

    def execute(self, x, out=None, stream=None, n_streams: int | None = None):
        """Transform the CUDA tensor ``x``; returns (S, C) complex64 or (S, C, 2) float16.

        With ``n_streams`` the leading dimension of x indexes independent streams
        (all the same length) and the output gains the same leading dimension.
        """
        self._check_input(x)
        if not x.is_cuda:
            raise ValueError("execute() needs a CUDA tensor; use execute_host() for host buffers")
        ns = 1 if n_streams is None else int(n_streams)
        if n_streams is not None and (ns < 1 or x.shape[0] != ns):
            raise ValueError("the leading dimension of x must equal n_streams")
        per = x.reshape(ns, -1)[0] if ns > 1 else x
        S = self.n_spectra_for(per)
        if S < 1:
            raise ValueError(f"input holds fewer than T={self.T} raw spectra")
        if out is None:
            out = self.empty_output(S, device=x.device, n_streams=n_streams)
        in_stride = self.C * (S + self.T - 1)
        check(lib().ppf_execute_batched(self.handle, ctypes.c_void_p(x.data_ptr()), in_stride,
                                        ctypes.c_void_p(out.data_ptr()), S * self.C, S, ns, _stream_handle(stream)))
        return out

    def fir(self, x, y=None, stream=None):
        """FIR alone (unfused ablation): (S, C) complex64 filtered spectra."""
        import torch
        self._check_input(x)
        S = self.n_spectra_for(x)
        if y is None:
            y = torch.empty((S, self.C), dtype=torch.complex64, device=x.device)
        check(lib().ppf_fir(self.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), S,
                            _stream_handle(stream)))
        return y

    def fft(self, y, out=None, stream=None):
        """DFT alone (unfused ablation) of (S, C) complex64 rows."""
        S = y.numel() // self.C
        if out is None:
            out = self.empty_output(S, device=y.device)
        check(lib().ppf_fft(self.handle, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(out.data_ptr()), S,
                            _stream_handle(stream)))
        return out

    def update_taps(self, taps, stream=None):
        """Copy C*T FP32 taps (a CUDA tensor) into the plan, ordered on the stream."""
        import torch
        t = taps.detach().reshape(-1)
        if not t.is_cuda or t.dtype != torch.float32 or t.numel() != self.C * self.T:
            raise TypeError("update_taps() takes C*T float32 CUDA taps")
        t = t.contiguous()
        check(lib().ppf_update_taps(self.handle, ctypes.c_void_p(t.data_ptr()), _stream_handle(stream)))
        self._taps_ref = t   # keep the source alive until the copy has run

    def backward(self, grad_out, x, want_input: bool = True, want_taps: bool = True, stream=None):
        """Adjoint: (grad wrt x or None, grad wrt taps (C*T float32) or None).

        grad_out: complex64 CUDA tensor (..., S, C); x: the forward input in the
        plan's input type (complex64 / interleaved float32, int16 or int8), with the
        same leading stream dimension if any.  The input gradient is complex64,
        one value per input sample, shaped like x (complex) or like x with the
        interleaved real/imaginary axis folded (real-pair inputs).
        """
        import torch
        if not (grad_out.is_cuda and x.is_cuda) or grad_out.dtype != torch.complex64:
            raise TypeError("backward() takes a complex64 CUDA gradient and a CUDA input")
        self._check_input(x)
        grad_out = grad_out.contiguous()
        x = x.contiguous()
        S = grad_out.shape[-2]
        ns = grad_out.numel() // (S * self.C)
        n_samples = x.numel() if x.is_complex() else x.numel() // 2
        if n_samples != ns * self.C * (S + self.T - 1):
            raise ValueError("x does not hold n_streams * C * (S + T - 1) samples")
        if x.is_complex():
            gx_shape = tuple(x.shape)
        elif x.dim() >= 2 and x.shape[-1] == 2:
            gx_shape = tuple(x.shape[:-1])          # (..., 2) real/imag pairs
        else:
            gx_shape = tuple(x.shape[:-1]) + (x.shape[-1] // 2,)   # interleaved along the last axis
        gx = torch.empty(gx_shape, dtype=torch.complex64, device=x.device) if want_input else None
        gh = torch.empty(self.C * self.T, dtype=torch.float32, device=x.device) if want_taps else None
        check(lib().ppf_backward(self.handle, ctypes.c_void_p(grad_out.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                 ctypes.c_void_p(gx.data_ptr() if gx is not None else 0),
                                 ctypes.c_void_p(gh.data_ptr() if gh is not None else 0), S, ns,
                                 _stream_handle(stream)))
        return gx, gh

    __call__ = execute

    def execute_host(self, x, out=None, stream=None):
        """Transform host buffers (numpy arrays or CPU tensors, pinned for full speed)."""
        import torch
        if isinstance(x, np.ndarray):
            x = torch.from_numpy(np.ascontiguousarray(x))
        self._check_input(x)
        if x.is_cuda:
            raise ValueError("execute_host() takes host buffers")
        S = self.n_spectra_for(x)
        if out is None:
            out = self.empty_output(S, device="cpu")
        check(lib().ppf_execute_host(self.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     S, _stream_handle(stream)))
        return out

    def check_device(self, stream=None):
        """Synchronise ``stream`` and raise PPFError if a bounded device wait gave up."""
        check(lib().ppf_check_device(self.handle, _stream_handle(stream)))

    def set_debug_flags(self, flags: int):
        """Testing aids (see ppf.h): 1 makes launches run out a bounded wait,
        2 makes backward() take its three-pass path where the fused kernel exists."""
        check(lib().ppf_set_debug_flags(self.handle, int(flags)))

    def close(self):
        if self._h is not None:
            check(lib().ppf_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def probe_rates() -> dict:
    """Device micro-benchmarks (ops/s): FP32 FMA, f32x2 FMA, int8/int16 -> FP32 conversions."""
    r = (ctypes.c_double * 5)()
    check(lib().ppf_probe_rates(r, 5))
    keys = ("ffma", "ffma2", "cvt_s8", "cvt_s8_bias", "cvt_s16")
    return dict(zip(keys, list(r)))


def probe_stream(in_bytes: int, ratio: int, device=None) -> float:
    """Achievable DRAM bytes/s of a read-in_bytes, write-ratio*in_bytes streaming kernel."""
    import torch
    a = torch.empty(in_bytes, dtype=torch.uint8, device=device or "cuda")
    b = torch.empty(max(16, in_bytes * ratio), dtype=torch.uint8, device=device or "cuda")
    r = ctypes.c_double()
    check(lib().ppf_probe_stream(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), in_bytes, ratio,
                                 ctypes.byref(r)))
    return r.value
