#!/usr/bin/env python
"""Benchmark of the fused PFB channeliser on GB300.

One step = one pass of the whole hot path (load, convert, FIR, FFT, store)
over one batch of synthetic input: C=512 channels, T=8 taps, 2^20 output
spectra of complex int8 input (sigma=16 Gaussian + a tone at channel 101),
complex FP32 output.  Inputs (1.07 GB) and outputs (4.29 GB) are larger than
L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  ``value`` is input GSamples/s over all ranks
(C * spectra / time, the sample rate f_s of Sec. 3); ``roofline`` relates the
kernel's algorithmic bytes to the measured HBM copy bandwidth; ``e2e`` is the
same metric through the host-buffer entry point (copies included);
``cpu_baseline`` is the FP64 oracle on a bounded sample of the same input on
the host cores, with the GPU output's error against it.  Beside the headline:
``precision`` (the same shape with fp32 and int16 input, each with its own
roofline), ``sweep`` (C=512, T in {8,16,32,64} x {int16, fp32} in x
{complex64, complex FP16} out, 2^18 spectra, against min(HBM, FP32) roofs),
``large_c`` (C=2048 and 4096), ``fwd_bwd``, ``batched_beams`` and the unfused
ablation.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 outside torchrun, the script launches N ranks of itself
through torch.distributed.run (one process per GPU, rendezvous on 127.0.0.1).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PFB input GSamples/s and % of HBM peak at C=512,T=8; fwd+bwd vs fwd time"
UNIT = "GSamples/s"
FALLBACK_HBM_GBS = 6800.0
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "pfb_fwd_c512_t8_ci8_c64.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--in-dtype", default="ci8", choices=["ci8", "ci16", "cf32"])
    ap.add_argument("--spectra", type=int, default=1 << 20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fwd-bwd", action="store_true")
    ap.add_argument("--no-ablation", action="store_true")
    ap.add_argument("--no-beams", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-large-c", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target length of the CPU sample")
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)   # internal: one timed oracle run
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = ("ppf_device.cuh", "ppf_fwd.cuh", "ppf_fwd_carry.cuh")


def kernel_source_sha():
    """SHA-256 over the forward kernel's device sources (identifies the profiled code)."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1511_03599_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch from the committed ncu summary; None unless the
    summary was taken on the kernel sources as they are now."""
    vals = {}
    try:
        with open(PROFILE_SUMMARY) as f:
            for line in f:
                for key in ("traffic_bytes_per_launch:", "kernel_source_sha:"):
                    if line.startswith(key):
                        vals[key] = line.split(":", 1)[1].strip()
    except OSError:
        return None
    v = vals.get("traffic_bytes_per_launch:")
    if v in (None, "", "null") or vals.get("kernel_source_sha:") != kernel_source_sha():
        return None
    return float(v)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_name(w, info):
    name = "pfb_fwd_carry_kernel" if info["variant"] & 4 else "pfb_fwd_kernel"
    return f"{name}<{w.C},{info['tap_bucket']},{w.in_dtype},{w.out_dtype}>"


def fp32_peak_flops(dev, sm_mhz=None):
    """FP32 CUDA-core peak: SMs x 128 lanes x 2 flops (FMA) x clock."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = sm_mhz
    if not mhz:
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                mhz = float(json.load(f)["sm_max_mhz"])
        except Exception:
            mhz = 2070.0
    return sms * 128 * 2 * mhz * 1e6


def flops_per_sample(C: int, T: int) -> float:
    """Algorithmic FP32 work per input sample: the FIR's 2(2T-1) (Sec. 4.1) plus
    the radix-2 FFT count 5 log2 C (3 * 2^k: the same formula, as a reference)."""
    import math
    return 2 * (2 * T - 1) + 5 * math.log2(C)


def time_launches(fn, steps: int, warmup: int, stream) -> float:
    """Mean ms per call of fn over `steps` calls, CUDA events on `stream`, after warm-up."""
    import torch
    for _ in range(max(3, warmup)):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def measure_case(w, steps: int, warmup: int, dev, peak: float, fp32_peak: float) -> dict:
    """One forward workload: kernel time (CUDA events), input GS/s, its own
    roofline (algorithmic bytes / time against the HBM copy peak) and, for the
    FP32 co-bound, the fraction of min(HBM roof, FP32 roof) in samples/s."""
    import torch
    from paper_1511_03599_gb300 import ppf, synth
    x = synth.stream_torch(w.C, w.n_raw, w.in_dtype, w.sigma, w.seed, w.tones, device=dev)
    st = torch.cuda.current_stream()
    with ppf.Plan(w.C, w.T, w.taps(), w.in_dtype, w.out_dtype) as plan:
        y = plan.empty_output(w.S, device=dev)
        ms = time_launches(lambda: plan.execute(x, out=y, stream=st), steps, warmup, st)
        plan.check_device()
        info = plan.info()
        finite = bool(torch.isfinite(y.float() if w.out_dtype == "c16" else torch.view_as_real(y)).all())
    b_in, b_out = synth.in_bytes_per_sample(w.in_dtype), synth.out_bytes_per_sample(w.out_dtype)
    alg = w.C * w.n_raw * b_in + w.C * w.S * b_out + 4 * w.C * w.T
    gsps = w.C * w.S / ms / 1e6
    achieved = alg / ms / 1e6
    hbm_roof = peak * 1e9 / (alg / (w.C * w.S)) / 1e9
    fp_roof = fp32_peak / flops_per_sample(w.C, w.T) / 1e9
    del x, y
    return {"workload": w.name, "C": w.C, "T": w.T, "spectra": w.S, "in": w.in_dtype, "out": w.out_dtype,
            "ms": ms, "gsps": gsps, "all_outputs_finite": finite,
            "roofline": {"bound": "hbm" if hbm_roof <= fp_roof else "fp32", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "algorithmic_bytes_per_launch": alg},
            "hbm_roof_gsps": hbm_roof, "fp32_roof_gsps": fp_roof,
            "frac_of_min_roof": gsps / min(hbm_roof, fp_roof), "launch": info}


def measure_fwd_bwd(steps: int, warmup: int, dev):
    """Forward vs forward+backward on the differentiable workload: C=256, T=16,
    64 streams x 8192 spectra of complex64 noise; backward = grad wrt input and
    taps (inverse DFT, transposed FIR, tap correlation + reduction)."""
    import torch
    from paper_1511_03599_gb300 import ppf, synth
    C, T, S, ns = 256, 16, 8192, 64
    n_raw = S + T - 1
    g = torch.Generator(device=dev)
    g.manual_seed(synth.SEED_BASE + 5)
    x = torch.randn((ns, n_raw * C), dtype=torch.complex64, device=dev, generator=g)
    G = torch.randn((ns, S, C), dtype=torch.complex64, device=dev, generator=g)
    plan = ppf.Plan(C, T, synth.design_taps(C, T), "cf32", "c64")
    y = plan.empty_output(S, device=dev, n_streams=ns)
    gx = torch.empty_like(x)
    gh = torch.empty(C * T, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()

    def fwd():
        plan.execute(x, out=y, n_streams=ns, stream=st)

    def fwd_bwd():
        fwd()
        ppf.check(ppf.lib().ppf_backward(plan.handle, ppf.ctypes.c_void_p(G.data_ptr()),
                                         ppf.ctypes.c_void_p(x.data_ptr()), ppf.ctypes.c_void_p(gx.data_ptr()),
                                         ppf.ctypes.c_void_p(gh.data_ptr()), S, ns,
                                         ppf.ctypes.c_void_p(st.cuda_stream)))

    def timed(fn):
        for _ in range(max(3, warmup)):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(steps):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    t_f = timed(fwd)
    t_fb = timed(fwd_bwd)
    plan.check_device()
    info = plan.info()
    plan.close()
    samples = ns * S * C
    return {"workload": f"pfb_c{C}_t{T}_{ns}x{S}_cf32_c64", "fwd_ms": t_f, "fwd_bwd_ms": t_fb,
            "fwd_bwd_over_fwd": t_fb / t_f, "fwd_gsps": samples / t_f / 1e6, "fwd_bwd_gsps": samples / t_fb / 1e6,
            "fwd_launch": info, "backward": "grad wrt input and taps, tap-gradient two-pass reduction"}


def measure_fwd_bwd_headline(plan, w, x, y, steps: int, warmup: int, dev):
    """Forward vs forward + adjoint (grad wrt input and taps) at the benchmark
    workload itself (C=512, T=8, int8 input): the adjoint reads the int8 input,
    the incoming complex64 gradient and writes a complex64 input gradient."""
    import torch
    from paper_1511_03599_gb300 import ppf, synth
    st = torch.cuda.current_stream()
    g = torch.Generator(device=dev)
    g.manual_seed(synth.SEED_BASE + 6)
    G = torch.randn((w.S, w.C), dtype=torch.complex64, device=dev, generator=g)
    gx = torch.empty(w.n_raw * w.C, dtype=torch.complex64, device=dev)
    gh = torch.empty(w.C * w.T, dtype=torch.float32, device=dev)

    def bwd():
        ppf.check(ppf.lib().ppf_backward(plan.handle, ppf.ctypes.c_void_p(G.data_ptr()),
                                         ppf.ctypes.c_void_p(x.data_ptr()), ppf.ctypes.c_void_p(gx.data_ptr()),
                                         ppf.ctypes.c_void_p(gh.data_ptr()), w.S, 1,
                                         ppf.ctypes.c_void_p(st.cuda_stream)))

    t_f = time_launches(lambda: plan.execute(x, out=y, stream=st), steps, warmup, st)
    t_fb = time_launches(lambda: (plan.execute(x, out=y, stream=st), bwd()), steps, warmup, st)
    plan.check_device()
    del G, gx, gh
    b_in = synth.in_bytes_per_sample(w.in_dtype)
    return {"workload": w.name, "fwd_ms": t_f, "fwd_bwd_ms": t_fb, "fwd_bwd_over_fwd": t_fb / t_f,
            "bwd_ms": t_fb - t_f, "backward": "grad wrt input and taps",
            "bwd_bytes_per_sample": 8 + b_in + 8}


def measure_fwd_bwd_shape(C: int, T: int, in_dtype: str, S: int, steps: int, warmup: int, dev):
    """Forward vs forward + adjoint (both gradients) for one single-stream
    shape; outside the fused adjoint kernel's shapes the adjoint is the
    three-pass path (inverse DFT, transposed FIR, tap correlation)."""
    import torch
    from paper_1511_03599_gb300 import ppf, synth
    st = torch.cuda.current_stream()
    sigma = {"ci8": 16.0, "ci16": 2000.0, "cf32": 1.0}[in_dtype]
    x = synth.stream_torch(C, S + T - 1, in_dtype, sigma, synth.SEED_BASE + 7, (), device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(synth.SEED_BASE + 8)
    G = torch.randn((S, C), dtype=torch.complex64, device=dev, generator=g)
    with ppf.Plan(C, T, synth.design_taps(C, T), in_dtype, "c64") as plan:
        y = plan.empty_output(S, device=dev)
        t_f = time_launches(lambda: plan.execute(x, out=y, stream=st), steps, warmup, st)
        t_fb = time_launches(lambda: (plan.execute(x, out=y, stream=st), plan.backward(G, x, stream=st)),
                             steps, warmup, st)
        plan.check_device()
        fused = plan.info()  # launch shape of the forward
    del x, G, y
    return {"workload": f"pfb_c{C}_t{T}_s{S}_{in_dtype}_c64", "fwd_ms": t_f, "fwd_bwd_ms": t_fb,
            "fwd_bwd_over_fwd": t_fb / t_f, "bwd_ms": t_fb - t_f, "fwd_launch": fused,
            "backward": "three-pass: inverse DFT, transposed FIR, tap correlation + fixed-order reduction"}


def measure_ablation(plan, x, y, steps: int, warmup: int, dev):
    """Fused kernel vs the unfused pair (FIR kernel, filtered spectra to HBM,
    then the DFT kernel) on the benchmark workload (E3 of the paper: the FIR/DFT
    split of the PPF's time)."""
    import torch
    st = torch.cuda.current_stream()
    yf = torch.empty(y.shape, dtype=torch.complex64, device=dev)

    def timed(fn):
        for _ in range(max(3, warmup)):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(steps):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    t_fused = timed(lambda: plan.execute(x, out=y, stream=st))
    t_fir = timed(lambda: plan.fir(x, y=yf, stream=st))
    t_fft = timed(lambda: plan.fft(yf, out=y, stream=st))
    del yf
    return {"fused_ms": t_fused, "fir_ms": t_fir, "fft_ms": t_fft, "unfused_ms": t_fir + t_fft,
            "fusion_speedup": (t_fir + t_fft) / t_fused, "fft_share_unfused": t_fft / (t_fir + t_fft),
            "note": "unfused = FIR kernel writing complex64 filtered spectra to HBM, then the DFT kernel"}


def measure_beams(steps: int, dev, seed: int = 4):
    """The multi-beam workload: 96 beams, C in {64..4096}, T in {4, 8, 16},
    spectra per beam uniform in [2^12, 2^17], complex int8 sigma=16 in, complex
    FP32 out: one persistent launch (C >= 2048 tiles on whole CTAs, C <= 1024 tiles on
    half-CTA groups), replayed from a CUDA graph after autotuning."""
    import numpy as np
    import torch
    from paper_1511_03599_gb300 import beams, synth
    rng = np.random.default_rng(synth.SEED_BASE + seed)
    n = 96
    C = [int(c) for c in rng.choice([64, 128, 256, 512, 1024, 2048, 4096], n)]
    T = [int(t) for t in rng.choice([4, 8, 16], n)]
    S = [int(s) for s in rng.integers(1 << 12, (1 << 17) + 1, n)]
    taps = [synth.design_taps(c, t) for c, t in zip(C, T)]
    bs = beams.BeamSet(C, T, S, taps)
    ins = [synth.stream_torch(c, s + t - 1, "ci8", 16.0, synth.SEED_BASE + seed + 17 * i, (), device=dev)
           for i, (c, t, s) in enumerate(zip(C, T, S))]
    outs = [torch.empty((s, c), dtype=torch.complex64, device=dev) for c, s in zip(C, S)]
    bs.bind(ins, outs)
    tune = beams.autotune(bs, cache_path=None)
    g = bs.capture_graph()
    st = torch.cuda.current_stream()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(steps):
        g.replay()
    b.record(st)
    torch.cuda.synchronize()
    bs.check_device()
    ms = a.elapsed_time(b) / steps
    peak, kind = measured_peaks()
    gbs = bs.bytes_moved() / ms / 1e6
    res = {"workload": f"{n} beams, C in 64..4096, T in 4/8/16, S in [2^12, 2^17], ci8->c64",
           "samples": bs.samples(), "ms": ms, "gsps": bs.samples() / ms / 1e6, "GB_s": gbs,
           "hbm_frac": gbs / peak, "tile_samples": tune["tile_samples"], "ctas_per_sm": tune["ctas_per_sm"],
           "launches_per_step": bs.launches_per_execute(), "graph": True, "tiles": bs.info()["tiles"],
           "wide_tiles": bs.info()["wide_tiles"]}
    bs.close()
    del ins, outs
    return res


def cpu_baseline(w, target_s: float, x_dev=None, y_dev=None):
    """The FP64 oracle as it stands, on a bounded sample of the same workload.

    With the benchmark's device input and output given, the sample is the
    first S spectra of that very input (copied to the host), and the GPU
    output of the timed run is compared with the oracle's on those spectra and
    on the last 2T spectra of the stream: whole-sample relative L2 and the
    per-spectrum maximum of the same ratio."""
    import numpy as np

    import oracle
    from paper_1511_03599_gb300 import synth

    h = w.taps()

    def sample_input(S):
        if x_dev is None:
            return synth.stream(w.C, S + w.T - 1, w.in_dtype, w.sigma, w.seed, w.tones)
        return x_dev[: (S + w.T - 1) * w.C].cpu().numpy()

    def run(S):
        x = sample_input(S)
        t0 = time.perf_counter()
        Y = oracle.pfb(x, h, w.C, w.T)
        return time.perf_counter() - t0, Y

    S = 256
    dt, _ = run(S)
    S = int(max(256, min(w.S, S * target_s / max(dt, 1e-3))))
    dt, Y = run(S)
    cores = os.cpu_count()
    res = {"value": w.C * S / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{S} of {w.S} spectra of {w.name} (FP64 direct FIR + naive O(C^2) DFT, numpy)",
           "seconds": dt}
    if y_dev is not None:
        def as_np(y):
            if w.out_dtype == "c64":
                return y.cpu().numpy().astype(np.complex128)
            a = y.float().cpu().numpy()
            return a[..., 0].astype(np.float64) + 1j * a[..., 1]
        got = as_np(y_dev[:S])
        n_tail = min(w.S, 2 * w.T)
        s0 = w.S - n_tail
        xt = x_dev[s0 * w.C:].cpu().numpy()
        Yt = oracle.pfb(xt, h, w.C, w.T)
        gt = as_np(y_dev[s0:])
        res["parity"] = {"spectra_compared": S + n_tail,
                         "rel_l2": oracle.rel_l2(np.concatenate([got, gt]), np.concatenate([Y, Yt])),
                         "max_per_spectrum_rel_l2": max(oracle.rel_l2_max_per_spectrum(got, Y),
                                                        oracle.rel_l2_max_per_spectrum(gt, Yt)),
                         "tolerance": 1e-5 if w.out_dtype == "c64" else 2e-3,
                         "compared": f"first {S} and last {n_tail} output spectra of the timed run"}
    # the same oracle on one core: a child process with every BLAS / OpenMP pool at one thread
    try:
        s1 = max(64, S // max(1, cores) // 2)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                   BLIS_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1", NUMEXPR_NUM_THREADS="1")
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(s1),
                            "--in-dtype", w.in_dtype, "--spectra", str(w.S)],
                           env=env, capture_output=True, text=True, timeout=600)
        d1 = json.loads(r.stdout.strip().splitlines()[-1])
        res["single_core"] = {"value": w.C * s1 / d1["seconds"] / 1e9, "unit": UNIT, "cores": 1,
                              "sample": f"{s1} of {w.S} spectra", "seconds": d1["seconds"]}
    except Exception as e:  # noqa: BLE001 - context beside the metric
        res["single_core"] = {"error": str(e)}
    return res


def oracle_sample(w, S: int):
    """One timed oracle run on S spectra (the child process of the single-core baseline)."""
    import oracle
    from paper_1511_03599_gb300 import synth
    x = synth.stream(w.C, S + w.T - 1, w.in_dtype, w.sigma, w.seed, w.tones)
    h = w.taps()
    t0 = time.perf_counter()
    oracle.pfb(x, h, w.C, w.T)
    print(json.dumps({"seconds": time.perf_counter() - t0}), flush=True)


def cpu_fast(w, target_s: float):
    """The paper's CPU shape (its CPU channeliser: a multithreaded FP32 FIR, then a
    library batched FFT), here torch's CPU kernels on all host cores, on a bounded
    sample of the same workload.  A context number beside the oracle, not the oracle."""
    import torch
    from paper_1511_03599_gb300 import synth

    h = torch.from_numpy(w.taps()).view(w.T, w.C)
    s_max = min(w.S, 1 << 17)
    x_all = synth.stream_torch(w.C, s_max + w.T - 1, w.in_dtype, w.sigma, w.seed, w.tones, device="cpu")

    def run(S):
        x = x_all[: (S + w.T - 1) * w.C]
        t0 = time.perf_counter()
        xc = torch.view_as_complex(x.float().view(S + w.T - 1, w.C, 2))
        y = xc[0:S] * h[0]
        for t in range(1, w.T):
            y.add_(xc[t:t + S] * h[t])
        torch.fft.fft(y, dim=1)
        return time.perf_counter() - t0

    S = min(4096, s_max)
    dt = run(S)
    S = int(max(S, min(s_max, S * target_s / max(dt, 1e-3))))
    dt = run(S)
    return {"value": w.C * S / dt / 1e9, "unit": UNIT, "cores": torch.get_num_threads(),
            "kind": "fp32 FIR + torch CPU FFT (the paper's CPU shape)",
            "sample": f"{S} of {w.S} spectra of {w.name} (input conversion, FIR and FFT timed)", "seconds": dt}


def run_reference(args, w):
    """Reference arm: the FP64 oracle (the CPU program the GPU path is checked against)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1511_03599_gb300 import synth  # noqa: F401
    import numpy as np

    import oracle
    h = w.taps()
    S = 2048
    x = synth.stream(w.C, S + w.T - 1, w.in_dtype, w.sigma, w.seed, w.tones)
    for _ in range(args.warmup):
        oracle.pfb(x[: (64 + w.T - 1) * w.C], h, w.C, w.T)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.pfb(x, h, w.C, w.T)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    v = w.C * S / t / 1e9
    world = int(os.environ.get("WORLD_SIZE", "1"))
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(w.describe(), sample_spectra_per_step=S),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{S} of {w.S} spectra per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def free_port() -> int:
    import socket
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def relaunch_command(n: int, argv, port: int):
    """torch.distributed.run command that starts n ranks of this script (one per GPU)."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
            "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + list(argv)


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ and args.oracle_sample == 0:
        # one process per GPU: launch the ranks, wait for them, pass their status on
        r = subprocess.run(relaunch_command(args.gpus, sys.argv[1:], free_port()))
        sys.exit(r.returncode)
    from paper_1511_03599_gb300 import synth
    w = synth.target_workload(args.in_dtype, args.spectra)
    if args.oracle_sample > 0:
        oracle_sample(w, args.oracle_sample)
        return
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    import torch.distributed as dist
    from paper_1511_03599_gb300 import ppf

    from paper_1511_03599_gb300 import dist as pdist
    rank, local, world = pdist.env_rank_world()
    if world != args.gpus:
        raise SystemExit(f"bench.py: --gpus {args.gpus} but {world} rank(s) were launched")
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    barrier = pdist.barrier

    # each rank processes its own stream shard of the same shape (weak scaling)
    x = synth.stream_torch(w.C, w.n_raw, w.in_dtype, w.sigma, pdist.rank_seed(w.seed, rank), w.tones, device=dev)
    h = w.taps()
    plan = ppf.Plan(w.C, w.T, h, w.in_dtype, w.out_dtype)
    y = plan.empty_output(w.S, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(max(3, args.warmup)):
        plan.execute(x, out=y, stream=stream)
    torch.cuda.synchronize()

    # one event pair around the K back-to-back launches on the launching stream:
    # the average launch duration (events between launches would add a gap each)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        t0 = time.perf_counter()
        e0.record(stream)
        for i in range(args.steps):
            plan.execute(x, out=y, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    barrier()
    total_ms = e0.elapsed_time(e1)
    t_step = pdist.max_over_ranks(total_ms / 1e3 / args.steps, device=dev)

    info = plan.info()
    samples = w.C * w.S
    b_in, b_out = synth.in_bytes_per_sample(w.in_dtype), synth.out_bytes_per_sample(w.out_dtype)
    alg_bytes = w.C * w.n_raw * b_in + w.C * w.S * b_out + 4 * w.C * w.T
    value = world * samples / t_step / 1e9
    kern_s = total_ms / 1e3 / args.steps
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / kern_s / 1e9
    traffic = profiled_traffic()

    # achievable DRAM bandwidth for this kernel's read:write mix (context for the roofline)
    mix = None
    try:
        ratio = max(1, round(b_out / b_in))
        mix = {"read_write_ratio": f"1:{ratio}", "GB_s": ppf.probe_stream(256 << 20, ratio) / 1e9}
        mix["frac_of_mix"] = achieved / mix["GB_s"]
    except Exception as e:  # noqa: BLE001 - context only
        mix = {"error": str(e)}

    # end to end through the host-buffer entry point: H2D + kernel + D2H every step
    e2e = None
    if not args.no_e2e:
        xh = x.cpu().pin_memory()
        yh = torch.empty(y.shape, dtype=y.dtype).pin_memory()
        plan.execute_host(xh, out=yh)
        barrier()
        n_e2e = max(2, min(5, args.steps))
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            plan.execute_host(xh, out=yh)
        te = pdist.max_over_ranks((time.perf_counter() - t0) / n_e2e, device=dev)
        e2e = {"value": world * samples / te / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(xh.numel() * xh.element_size()),
               "d2h_bytes_per_step": int(yh.numel() * yh.element_size()),
               "ms_per_step": te * 1e3, "path": "ppf_execute_host, pinned host buffers, chunk pipeline on copy-in / compute / copy-out streams"}
        # the host link alone: the same bytes copied concurrently (D2H of the
        # output, H2D of the input) with no kernel -- the bound of this number
        try:
            s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

            def copies():
                with torch.cuda.stream(s1):
                    yh.copy_(y, non_blocking=True)
                with torch.cuda.stream(s2):
                    x.copy_(xh, non_blocking=True)   # the same values back into the input buffer
            copies()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(n_e2e):
                copies()
            torch.cuda.synchronize()
            tc = (time.perf_counter() - t0) / n_e2e
            e2e["copy_only_ms"] = tc * 1e3
            e2e["frac_of_copy_only"] = tc / te
        except Exception as e:  # noqa: BLE001 - context only
            e2e["copy_only_error"] = str(e)
        del xh, yh

    abl = None
    if not args.no_ablation:
        try:
            abl = measure_ablation(plan, x, y, max(5, args.steps // 2), args.warmup, dev)
        except Exception as e:  # noqa: BLE001 - the ablation is context, not the metric
            abl = {"error": str(e)}
    bm = None
    if not args.no_beams:
        try:
            bm = measure_beams(max(5, args.steps // 2), dev)
        except Exception as e:  # noqa: BLE001 - reported beside the metric
            bm = {"error": str(e)}
    fb = None
    if not args.no_fwd_bwd:
        fb = measure_fwd_bwd(max(5, args.steps), args.warmup, dev)
        try:
            fb["headline"] = measure_fwd_bwd_headline(plan, w, x, y, max(5, args.steps // 2), args.warmup, dev)
        except Exception as e:  # noqa: BLE001 - reported beside the metric
            fb["headline"] = {"error": str(e)}
        try:
            fb["long_taps"] = measure_fwd_bwd_shape(512, 32, "ci8", 1 << 18, max(5, args.steps // 2), args.warmup, dev)
        except Exception as e:  # noqa: BLE001 - reported beside the metric
            fb["long_taps"] = {"error": str(e)}
        try:
            from paper_1511_03599_gb300 import fit
            r = fit.fit_taps()
            fb["tap_fit"] = {k: r[k] for k in ("optimizer", "steps", "ms_per_step", "phase_ms", "sinc_hamming_loss")}
            fb["tap_fit"].update({"leakage_first": r["loss"][0], "leakage_last": r["loss"][-1],
                                  "loss": "out-of-band energy of a per-stream off-centre tone set"})
        except Exception as e:  # noqa: BLE001 - context beside the metric
            fb["tap_fit"] = {"error": str(e)}

    # the same shape with fp32 and int16 input, the tap/precision sweep (C=512,
    # 2^18 spectra) and large channel counts: kernel time of each, own roofline
    fp32_peak = fp32_peak_flops(dev, clk.summary().get("sm_mhz"))
    cell_steps = max(5, args.steps // 2)
    prec = None
    if not args.no_precision:
        prec = {}
        for d in ("cf32", "ci16"):
            if d != w.in_dtype:
                try:
                    prec[d] = measure_case(synth.target_workload(d, args.spectra), cell_steps, args.warmup, dev,
                                           peak, fp32_peak)
                except Exception as e:  # noqa: BLE001 - reported beside the metric
                    prec[d] = {"error": str(e)}
    sweep = None
    if not args.no_sweep:
        sweep = []
        for T in (8, 16, 32, 64):
            for d in ("ci16", "cf32"):
                for o in ("c64", "c16"):
                    try:
                        sweep.append(measure_case(synth.sweep_workload(T, d, o), cell_steps, args.warmup, dev,
                                                  peak, fp32_peak))
                    except Exception as e:  # noqa: BLE001
                        sweep.append({"workload": f"T={T} {d}->{o}", "error": str(e)})
    large = None
    if not args.no_large_c:
        large = []
        for C in (1024, 2048, 4096):
            try:
                lw = synth.Workload(f"pfb_c{C}_t8_s{(1 << 28) // C}_ci8_c64", C, 8, (1 << 28) // C, "ci8", "c64",
                                    16.0, synth.SEED_BASE + 30 + C, ())
                large.append(measure_case(lw, cell_steps, args.warmup, dev, peak, fp32_peak))
            except Exception as e:  # noqa: BLE001
                large.append({"workload": f"C={C}", "error": str(e)})

    if rank == 0:
        cpu = cpu_f = None
        if world == 1 and not args.no_cpu_baseline:
            plan.execute(x, out=y, stream=stream)     # y holds the fused result again (the ablation overwrote it)
            torch.cuda.synchronize()
            cpu = cpu_baseline(w, args.cpu_seconds, x, y)
            try:
                cpu_f = cpu_fast(w, min(5.0, args.cpu_seconds))
            except Exception as e:  # noqa: BLE001 - context beside the metric
                cpu_f = {"error": str(e)}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(w.describe(), spectra_per_gpu=w.S, parallelism=f"replicas{world}" if world > 1 else "single",
                           l2=f"inputs larger than L2: {w.C * (w.S + w.T - 1) * synth.in_bytes_per_sample(w.in_dtype) / 1e9:.2f}"
                              f" GB in + {w.C * w.S * synth.out_bytes_per_sample(w.out_dtype) / 1e9:.2f} GB out per step,"
                              " no flush",
                           launch=info),
            "hbm_frac": achieved / peak,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": kernel_name(w, info), "algorithmic_bytes_per_launch": alg_bytes,
                         "kernel_ms": kern_s * 1e3, "streaming_mix_peak": mix},
            "clocks": clk.summary(),
            "gpu_launches": args.steps,
            "gpu_launches_fwd_bwd": None if fb is None else 3 * max(5, args.steps),
            "e2e": e2e,
            "fwd_bwd": fb,
            "unfused_ablation": abl,
            "batched_beams": bm,
            "precision": prec,
            "sweep": sweep,
            "large_c": large,
            "cpu_baseline": cpu,
            "cpu_fast": cpu_f,
            "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
