"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (relative L2 error of the whole compared output against the FP64
oracle): <= 1e-5 for complex FP32 output, <= 2e-3 for complex FP16 output.
The same bound holds for the per-spectrum maximum of that ratio wherever the
inputs are noise (every spectrum carries energy).  Sizes span several CTA
batches and a ragged tail; the full-size workloads are checked on sampled
spectra (first T, last T and at least 16 384 seeded random ones).
"""
import numpy as np
import pytest

import oracle
from conftest import record_parity
from paper_1511_03599_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "c16": 2e-3}
SIGMA = {"ci8": 16.0, "ci16": 2000.0, "cf32": 1.0}


@pytest.fixture(scope="module")
def ppf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_03599_gb300 import ppf as m
    m.lib()
    return m


def to_device(x_raw):
    return torch.from_numpy(np.ascontiguousarray(x_raw)).cuda()


def out_to_numpy(y, out_dtype):
    y = y.cpu()
    if out_dtype == "c64":
        return y.numpy().astype(np.complex128)
    a = y.float().numpy()
    return a[..., 0].astype(np.float64) + 1j * a[..., 1].astype(np.float64)


def run_case(ppf, C, T, S, in_dtype, out_dtype, seed, taps=None, tones=()):
    scale = 1.0 / np.sqrt(C) if out_dtype == "c16" else 1.0
    h = synth.design_taps(C, T, scale=scale) if taps is None else taps
    x = synth.stream(C, S + T - 1, in_dtype, SIGMA[in_dtype], seed, tones)
    with ppf.Plan(C, T, h, in_dtype, out_dtype) as plan:
        y = plan(to_device(x))
        torch.cuda.synchronize()
    got = out_to_numpy(y, out_dtype)
    ref = oracle.pfb(x, h, C, T)
    assert got.shape == ref.shape
    assert np.all(np.isfinite(got))
    check_errors(f"C={C} T={T} S={S} {in_dtype}->{out_dtype}", got, ref, out_dtype)
    return got, ref


def check_errors(case, got, ref, out_dtype, per_spectrum=True):
    """Whole-output relative L2 and its per-spectrum maximum, both within the tolerance."""
    err = oracle.rel_l2(got, ref)
    emax = oracle.rel_l2_max_per_spectrum(got, ref)
    record_parity(case, err, emax, TOL[out_dtype])
    assert err <= TOL[out_dtype], f"{case}: rel L2 {err:.3e}"
    if per_spectrum:
        assert emax <= TOL[out_dtype], f"{case}: per-spectrum max rel L2 {emax:.3e}"


# every channel count, several tap counts (bucket edges and a runtime tap loop),
# ragged spectrum counts that span several CTA batches
@pytest.mark.parametrize("C", [32, 64, 128, 256, 512, 1024, 2048, 4096])
@pytest.mark.parametrize("T", [1, 3, 8, 17, 64])
def test_parity_channels_taps_ci8(ppf, C, T):
    S = max(3, 24576 // C) + 5
    run_case(ppf, C, T, S, "ci8", "c64", seed=1000 + C + T)


# shapes whose batch is halved so the TMA ring fits beside it: 16/32-bit input
# at C = 32 (128-spectrum batches of 8-output segments, up to 64 taps) and
# 16-tap int16 input at C = 768 (4-spectrum batches, a 6-slot ring); ragged
# counts spanning several batches
@pytest.mark.parametrize("C,T,in_dtype,out_dtype", [(32, 1, "ci16", "c64"), (32, 8, "cf32", "c64"),
                                                    (32, 16, "ci16", "c16"), (32, 40, "cf32", "c64"),
                                                    (32, 64, "ci16", "c64"), (768, 16, "ci16", "c64"),
                                                    (768, 13, "ci16", "c16")])
def test_parity_halved_batches(ppf, C, T, in_dtype, out_dtype):
    S = 5 * 128 + 7 if C == 32 else 6 * 152 * 4 + 9
    with ppf.Plan(C, T, synth.design_taps(C, T), in_dtype, out_dtype) as plan:
        assert plan.info()["variant"] & 1, "expected the TMA-ring mode for this shape"
    run_case(ppf, C, T, S, in_dtype, out_dtype, seed=4500 + C + T)


# C = 3 * 2^k: a radix-3 DFT stage, then power-of-two stages (the paper's
# non-power-of-two example is C = 3072)
@pytest.mark.parametrize("C", [384, 768, 1536, 3072])
@pytest.mark.parametrize("T,in_dtype,out_dtype", [(1, "cf32", "c64"), (8, "ci8", "c64"), (16, "ci16", "c16"),
                                                  (5, "cf32", "c64"), (64, "ci8", "c64")])
def test_parity_non_power_of_two_channels(ppf, C, T, in_dtype, out_dtype):
    S = max(3, 12288 // C) + 3
    run_case(ppf, C, T, S, in_dtype, out_dtype, seed=4000 + C + T)


# Large C: the thread-block-cluster kernel (a slice of channels per CTA, the
# first DFT stage gathered across the cluster) where the plan picks it, else
# the generic kernel.  Enough spectra that every work unit carries its FIR
# state over several batches.
@pytest.mark.parametrize("C", [768, 1024, 1536, 2048, 3072, 4096])
@pytest.mark.parametrize("T,in_dtype,out_dtype", [(8, "ci8", "c64"), (4, "cf32", "c64"), (16, "ci16", "c16"),
                                                  (1, "ci8", "c64"), (13, "ci8", "c64"), (2, "cf32", "c16"),
                                                  (8, "ci16", "c64"), (5, "ci16", "c64")])
def test_parity_cluster_channels(ppf, C, T, in_dtype, out_dtype):
    S = 6 * 152 * 16 // max(1, C // 512) + 7
    h = synth.design_taps(C, T, scale=(1.0 / np.sqrt(C) if out_dtype == "c16" else 1.0))
    x = synth.stream(C, S + T - 1, in_dtype, SIGMA[in_dtype], 5000 + C + T)
    with ppf.Plan(C, T, h, in_dtype, out_dtype) as plan:
        y = plan(to_device(x))
        torch.cuda.synchronize()
        idx = _sampled_indices(S, T, 96, 79 + C)
        sel = y[torch.from_numpy(idx).cuda()]
        assert bool(torch.isfinite(sel.float() if out_dtype == "c16" else torch.view_as_real(sel)).all())
        got = out_to_numpy(sel, out_dtype)
    ref = oracle.pfb_spectra(x, h, C, T, idx)
    check_errors(f"cluster C={C} T={T} {in_dtype}->{out_dtype}", got, ref, out_dtype)


@pytest.mark.parametrize("C", [768, 1024, 2048, 3072, 4096])
@pytest.mark.parametrize("in_dtype", ["ci8", "cf32"])
def test_parity_cluster_every_output_batched(ppf, C, in_dtype):
    """Several independent streams in one launch (strided), every output compared
    (the cluster kernel for fp32 input at C = 2048, the generic kernel at C = 4096)."""
    T, n_streams = 8, 3
    S = 300
    h = synth.design_taps(C, T)
    xs = [synth.stream(C, S + T - 1, in_dtype, SIGMA[in_dtype], 5100 + C + i) for i in range(n_streams)]
    with ppf.Plan(C, T, h, in_dtype, "c64") as plan:
        if C in (2048, 4096):
            assert bool(plan.info()["variant"] & 16) == (C == 2048 and in_dtype == "cf32")
        got = plan.execute(torch.stack([to_device(x) for x in xs]), n_streams=n_streams)
        torch.cuda.synchronize()
        got = got.cpu().numpy().astype(np.complex128)
    for i, x in enumerate(xs):
        ref = oracle.pfb(x, h, C, T)
        assert oracle.rel_l2(got[i], ref) <= TOL["c64"], f"stream {i}"


# Several streams in one launch with more batches than work units, so shares
# of the batch sequence cross stream boundaries (carry, generic and cluster
# kernels): bit-identical to one launch per stream, and right by the oracle.
@pytest.mark.parametrize("C,T,in_dtype,S,ns", [(512, 8, "ci8", 2000, 5), (256, 16, "cf32", 1500, 7),
                                               (4096, 16, "cf32", 400, 3), (2048, 8, "ci8", 700, 4),
                                               (64, 1, "ci16", 3000, 9), (4096, 8, "ci8", 301, 3),
                                               (2048, 16, "ci8", 333, 3), (1024, 4, "cf32", 777, 5)])
def test_batched_shares_cross_streams(ppf, C, T, in_dtype, S, ns):
    h = synth.design_taps(C, T)
    xs = [synth.stream(C, S + T - 1, in_dtype, SIGMA[in_dtype], 5200 + C + i) for i in range(ns)]
    with ppf.Plan(C, T, h, in_dtype, "c64") as plan:
        yb = plan.execute(torch.stack([to_device(x) for x in xs]), n_streams=ns)
        torch.cuda.synchronize()
        plan.check_device()
        for i, x in enumerate(xs):
            yi = plan(to_device(x))
            torch.cuda.synchronize()
            assert torch.equal(torch.view_as_real(yb[i]), torch.view_as_real(yi)), f"stream {i}"
        y1 = yb[1].cpu().numpy().astype(np.complex128)
    assert oracle.rel_l2(y1, oracle.pfb(xs[1], h, C, T)) <= TOL["c64"]


@pytest.mark.parametrize("C,T,in_dtype", [(512, 8, "ci8"), (4096, 4, "ci8"), (1536, 8, "cf32"),
                                          (384, 8, "ci8"), (32, 4, "ci8"), (4096, 2, "ci8"),
                                          (4096, 8, "ci8"), (2048, 8, "ci8"), (1024, 4, "cf32"),
                                          (384, 8, "ci16")])
def test_more_streams_than_resident_ctas(ppf, C, T, in_dtype):
    """400 short streams in one launch: several waves of carry CTAs, or shares of
    the cluster / generic kernels spanning many streams (the generic kernel in its
    TMA-ring mode at C=32, 384, 1024, 2048 and 4096, with the ring's refill slot
    (C=2048, T=8) and without it (C=4096, T=8; C=1024 and 384, 16/32-bit input));
    bit-identical per stream."""
    ns, S = 400, 5
    h = synth.design_taps(C, T)
    x = np.stack([synth.stream(C, S + T - 1, in_dtype, SIGMA[in_dtype], 5300 + i) for i in range(ns)])
    with ppf.Plan(C, T, h, in_dtype, "c64") as plan:
        yb = plan.execute(to_device(x), n_streams=ns)
        torch.cuda.synchronize()
        plan.check_device()
        for i in (0, 1, 199, 398, 399):
            yi = plan(to_device(x[i]))
            torch.cuda.synchronize()
            assert torch.equal(torch.view_as_real(yb[i]), torch.view_as_real(yi)), f"stream {i}"
        y = yb[399].cpu().numpy().astype(np.complex128)
    assert oracle.rel_l2(y, oracle.pfb(x[399], h, C, T)) <= TOL["c64"]


@pytest.mark.parametrize("in_dtype", ["ci8", "ci16", "cf32"])
@pytest.mark.parametrize("out_dtype", ["c64", "c16"])
@pytest.mark.parametrize("T", [2, 4, 8, 16, 32, 64])
def test_parity_types_c512(ppf, in_dtype, out_dtype, T):
    run_case(ppf, 512, T, 77, in_dtype, out_dtype, seed=2000 + T)


@pytest.mark.parametrize("S", [1, 2, 15, 16, 17, 31, 33, 250])
def test_parity_ragged_spectrum_counts(ppf, S):
    run_case(ppf, 512, 8, S, "ci8", "c64", seed=3000 + S)


@pytest.mark.parametrize("C", [32, 4096])
def test_parity_single_spectrum_extremes(ppf, C):
    run_case(ppf, C, 64, 1, "cf32", "c64", seed=3100 + C)
    run_case(ppf, C, 1, 1, "ci16", "c64", seed=3200 + C)


def test_parity_small_workload_full(ppf):
    """C=256, T=8, 4096 spectra, c64 noise + tone at channel 37: every output compared."""
    w = synth.small_parity_workload()
    x = w.input()
    h = w.taps()
    with ppf.Plan(w.C, w.T, h, w.in_dtype, w.out_dtype) as plan:
        got = out_to_numpy(plan(to_device(x)), "c64")
    ref = oracle.pfb(x, h, w.C, w.T)
    assert oracle.rel_l2(got, ref) <= TOL["c64"]
    assert int(np.argmax(np.abs(got).mean(axis=0))) == 37


def test_integer_extremes(ppf):
    """int8 -128 / +127 and int16 -32768 / +32767 are converted exactly."""
    C, T, S = 64, 4, 40
    h = synth.design_taps(C, T)
    rng = np.random.default_rng(5)
    for dt, lo, hi in (("ci8", -128, 127), ("ci16", -32768, 32767)):
        x = rng.choice(np.array([lo, hi, 0, -1]), size=(C * (S + T - 1), 2)).astype(np.int8 if dt == "ci8" else np.int16)
        with ppf.Plan(C, T, h, dt, "c64") as plan:
            got = out_to_numpy(plan(to_device(x)), "c64")
        assert oracle.rel_l2(got, oracle.pfb(x, h, C, T)) <= TOL["c64"]


def test_impulse_gives_polyphase_branch(ppf):
    """Impulse at (raw r, channel c0): Y[s][m] = h[(r-s)C + c0] exp(-2 pi i c0 m / C)."""
    C, T, S, r, c0 = 512, 8, 40, 20, 101
    h = synth.design_taps(C, T)
    x = synth.impulse_stream(C, S + T - 1, "cf32", r, c0)
    with ppf.Plan(C, T, h, "cf32", "c64") as plan:
        got = out_to_numpy(plan(to_device(x)), "c64")
    m = np.arange(C)
    for s in range(S):
        t = r - s
        ref = h[t * C + c0] * np.exp(-2j * np.pi * ((c0 * m) % C) / C) if 0 <= t < T else np.zeros(C)
        assert np.max(np.abs(got[s] - ref)) <= 1e-6 * max(1.0, np.max(np.abs(h)))


def test_deterministic_bitwise(ppf):
    C, T, S = 512, 8, 300
    h = synth.design_taps(C, T)
    x = to_device(synth.stream(C, S + T - 1, "ci8", 16.0, 9))
    with ppf.Plan(C, T, h, "ci8", "c64") as plan:
        a = plan(x).clone()
        b = plan(x)
    torch.cuda.synchronize()
    assert torch.equal(torch.view_as_real(a), torch.view_as_real(b))


def test_streaming_chunks_overlap_by_t_minus_1(ppf):
    """Two chunks that overlap by T-1 raw spectra reproduce the one-shot output."""
    C, T, S = 256, 8, 200
    h = synth.design_taps(C, T)
    x = synth.stream(C, S + T - 1, "ci16", 2000.0, 10)
    with ppf.Plan(C, T, h, "ci16", "c64") as plan:
        full = plan(to_device(x))
        s1 = 77
        a = plan(to_device(x[: (s1 + T - 1) * C]))
        b = plan(to_device(x[s1 * C:]))
    torch.cuda.synchronize()
    assert torch.equal(torch.cat([a, b]).view(torch.float32), full.view(torch.float32))


def test_execute_host_matches_device(ppf):
    C, T, S = 512, 8, 5000
    h = synth.design_taps(C, T)
    x = synth.stream(C, S + T - 1, "ci8", 16.0, 11)
    with ppf.Plan(C, T, h, "ci8", "c64") as plan:
        dev = plan(to_device(x)).cpu()
        host = plan.execute_host(torch.from_numpy(x).pin_memory())
    assert torch.equal(torch.view_as_real(dev), torch.view_as_real(host))


def test_execute_rejects_misaligned_and_overlapping(ppf):
    C, T = 512, 8
    h = synth.design_taps(C, T)
    with ppf.Plan(C, T, h, "ci8", "c64") as plan:
        buf = torch.zeros(C * 40 * 2 + 64, dtype=torch.int8, device="cuda")
        out = plan.empty_output(33, device="cuda")
        st = ppf.lib().ppf_execute(plan.handle, ppf.ctypes.c_void_p(buf.data_ptr() + 2),
                                   ppf.ctypes.c_void_p(out.data_ptr()), 33, None)
        assert st == 3
        st = ppf.lib().ppf_execute(plan.handle, ppf.ctypes.c_void_p(out.data_ptr()),
                                   ppf.ctypes.c_void_p(out.data_ptr()), 33, None)
        assert st == 1
        st = ppf.lib().ppf_execute(plan.handle, ppf.ctypes.c_void_p(buf.data_ptr()),
                                   ppf.ctypes.c_void_p(out.data_ptr()), 0, None)
        assert st == 1


def _sampled_indices(S, T, n_random, seed):
    rng = np.random.default_rng(seed)
    idx = set(range(min(S, T))) | set(range(max(0, S - T), S))
    idx |= set(rng.integers(0, S, n_random).tolist())
    return np.array(sorted(idx))


def _sampled_indices_distinct(S, T, n_random, seed):
    """The first T and last T spectra plus n_random distinct seeded others."""
    rng = np.random.default_rng(seed)
    ends = set(range(min(S, T))) | set(range(max(0, S - T), S))
    inner = np.setdiff1d(np.arange(S), np.array(sorted(ends)))
    pick = rng.choice(inner, size=min(n_random, inner.size), replace=False)
    return np.array(sorted(ends | set(pick.tolist())))


@pytest.mark.parametrize("in_dtype", ["ci8", "ci16", "cf32"])
def test_target_workload_full_size_sampled(ppf, in_dtype):
    """C=512, T=8, 2^20 spectra in the launch configuration the benchmark uses;
    the first T, the last T and 16 384 seeded random output spectra against the
    oracle, plus finiteness of every output."""
    w = synth.target_workload(in_dtype)
    x = w.input()
    h = w.taps()
    with ppf.Plan(w.C, w.T, h, w.in_dtype, w.out_dtype) as plan:
        xd = to_device(x)
        y = plan(xd)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(torch.view_as_real(y)).all())
        idx = _sampled_indices_distinct(w.S, w.T, 16384, 77)
        assert len(idx) >= 16384 + 2 * w.T
        got = y[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.complex128)
    ref = oracle.pfb_spectra(x, h, w.C, w.T, idx)
    check_errors(f"target C=512 T=8 S=2^20 {in_dtype}->c64 ({len(idx)} sampled spectra)", got, ref, "c64")


@pytest.mark.parametrize("T", [8, 16, 32, 64])
@pytest.mark.parametrize("in_dtype,out_dtype", [("ci16", "c64"), ("ci16", "c16"), ("cf32", "c64"), ("cf32", "c16")])
def test_sweep_cells_sampled(ppf, T, in_dtype, out_dtype):
    """C=512 tap/precision sweep at 2^18 spectra, sampled against the oracle."""
    w = synth.sweep_workload(T, in_dtype, out_dtype)
    x = w.input()
    h = w.taps()
    with ppf.Plan(w.C, w.T, h, w.in_dtype, w.out_dtype) as plan:
        y = plan(to_device(x))
        torch.cuda.synchronize()
        idx = _sampled_indices(w.S, w.T, 512, 78)
        sel = y[torch.from_numpy(idx).cuda()]
        assert bool(torch.isfinite(sel.float() if out_dtype == "c16" else torch.view_as_real(sel)).all())
        got = out_to_numpy(sel, out_dtype)
    ref = oracle.pfb_spectra(x, h, w.C, w.T, idx)
    check_errors(f"sweep C=512 T={T} S=2^18 {in_dtype}->{out_dtype}", got, ref, out_dtype)


@pytest.mark.parametrize("C,in_dtype,body", [(512, "ci8", "carry"), (2048, "cf32", "cluster"), (2048, "ci8", "ring")])
def test_bounded_wait_timeout_reported_and_context_usable(ppf, C, in_dtype, body):
    """A wait that nothing completes runs out, is reported, and the next launch is correct,
    in each TMA-staged body: the carry kernel, the cluster kernel (every CTA of each cluster
    gives up and the cluster leaves together) and the generic kernel's ring."""
    T, S = 8, 4096
    h = synth.design_taps(C, T)
    sigma = {"ci8": 16.0, "cf32": 1.0}[in_dtype]
    x = synth.stream(C, S + T - 1, in_dtype, sigma, 12)
    xd = to_device(x)
    with ppf.Plan(C, T, h, in_dtype, "c64") as plan:
        v = plan.info()["variant"]
        assert v & 1, "expected the TMA-staged kernel for this shape"
        # bit 2: FIR halo carried in registers (carry and cluster kernels); bit 4: cluster
        assert bool(v & 4) == (body != "ring") and bool(v & 16) == (body == "cluster")
        plan.set_debug_flags(1)
        plan(xd)
        with pytest.raises(ppf.PPFError) as ei:
            plan.check_device()
        assert ei.value.status == 5
        plan.set_debug_flags(0)
        y = plan(xd)
        plan.check_device()
        got = out_to_numpy(y, "c64")
    assert oracle.rel_l2(got, oracle.pfb(x, h, C, T)) <= TOL["c64"]


def test_probe_rates(ppf):
    r = ppf.probe_rates()
    assert all(v > 1e9 for v in r.values()), r
