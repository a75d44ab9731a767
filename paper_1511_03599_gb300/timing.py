"""Time one forward or adjoint case of the C ABI with CUDA events.

    python -m paper_1511_03599_gb300.timing forward C T IN [OUT] [--spectra S] [--streams N]
    python -m paper_1511_03599_gb300.timing backward C T [IN] [--spectra S] [--streams N]

Inputs are the seeded synthetic streams of ``synth`` (drawn on the device);
the default spectrum count gives 2^28 samples per stream, above the L2 size.
Prints one line: the case, the plan's launch shape and the rate.  Used to
make the ncu summaries of single kernels.
"""
from __future__ import annotations

import argparse
import json
import sys


def _events(fn, warmup: int, reps: int) -> float:
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def forward(C: int, T: int, in_dtype: str, out_dtype: str, S: int, n_streams: int, warmup: int, reps: int) -> dict:
    import torch
    from . import ppf, synth
    sigma = {"ci8": 16.0, "ci16": 2000.0, "cf32": 1.0}[in_dtype]
    xs = [synth.stream_torch(C, S + T - 1, in_dtype, sigma, synth.SEED_BASE + 10 + i, (), device="cuda")
          for i in range(n_streams)]
    x = xs[0] if n_streams == 1 else torch.stack(xs)
    scale = 1.0 / C ** 0.5 if out_dtype == "c16" else 1.0
    with ppf.Plan(C, T, synth.design_taps(C, T, scale=scale), in_dtype, out_dtype) as plan:
        ns = None if n_streams == 1 else n_streams
        y = plan.empty_output(S, device="cuda", n_streams=ns)
        ms = _events(lambda: plan(x, out=y, n_streams=ns), warmup, reps)
        plan.check_device()
        info = plan.info()
    b = C * (S + T - 1) * synth.in_bytes_per_sample(in_dtype) + C * S * synth.out_bytes_per_sample(out_dtype)
    return {"case": "forward", "C": C, "T": T, "in": in_dtype, "out": out_dtype, "spectra": S,
            "streams": n_streams, "ms": ms, "gsps": n_streams * C * S / ms / 1e6,
            "GB_s": n_streams * b / ms / 1e6, "launch": info}


def backward(C: int, T: int, in_dtype: str, S: int, n_streams: int, warmup: int, reps: int) -> dict:
    import torch
    from . import ppf, synth
    g = torch.Generator(device="cuda")
    g.manual_seed(synth.SEED_BASE + 20)
    sigma = {"ci8": 16.0, "ci16": 2000.0, "cf32": 1.0}[in_dtype]
    xs = [synth.stream_torch(C, S + T - 1, in_dtype, sigma, synth.SEED_BASE + 21 + i, (), device="cuda")
          for i in range(n_streams)]
    x = xs[0] if n_streams == 1 else torch.stack(xs)
    G = torch.randn((n_streams, S, C) if n_streams > 1 else (S, C), dtype=torch.complex64, device="cuda", generator=g)
    with ppf.Plan(C, T, synth.design_taps(C, T), in_dtype, "c64") as plan:
        ms = _events(lambda: plan.backward(G, x), warmup, reps)
        plan.check_device()
    b = n_streams * (C * S * 8 + C * (S + T - 1) * (synth.in_bytes_per_sample(in_dtype) + 8))
    return {"case": "backward", "C": C, "T": T, "in": in_dtype, "spectra": S, "streams": n_streams, "ms": ms,
            "gsps": n_streams * C * S / ms / 1e6, "GB_s": b / ms / 1e6}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    sub = ap.add_subparsers(dest="case", required=True)
    f = sub.add_parser("forward")
    f.add_argument("C", type=int)
    f.add_argument("T", type=int)
    f.add_argument("in_dtype", choices=["ci8", "ci16", "cf32"])
    f.add_argument("out_dtype", nargs="?", default="c64", choices=["c64", "c16"])
    bw = sub.add_parser("backward")
    bw.add_argument("C", type=int)
    bw.add_argument("T", type=int)
    bw.add_argument("in_dtype", nargs="?", default="cf32", choices=["ci8", "ci16", "cf32"])
    for p in (f, bw):
        p.add_argument("--spectra", type=int, default=None)
        p.add_argument("--streams", type=int, default=1)
        p.add_argument("--warmup", type=int, default=3)
        p.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    S = a.spectra if a.spectra else max(1, (1 << 28) // a.C // a.streams)
    if a.case == "forward":
        r = forward(a.C, a.T, a.in_dtype, a.out_dtype, S, a.streams, a.warmup, a.reps)
    else:
        r = backward(a.C, a.T, a.in_dtype, S, a.streams, a.warmup, a.reps)
    print(json.dumps(r), flush=True)


if __name__ == "__main__":
    sys.exit(main())
