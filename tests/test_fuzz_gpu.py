"""Seeded random shapes through every kernel family, against the FP64 oracle.

The hand-picked parity tests pin the kernel choices one by one; these draw
(C, T, input, output, spectra, streams) at random from the whole planned
range, so combinations nobody picked (a 3*2^k channel count with a long tap
count and many short streams, an adjoint on a cluster-kernel shape, ...)
are exercised too.  Every forward case compares its whole output (or, for
larger ones, the first and last T spectra plus a seeded sample) with the
oracle within the parity tolerances; every adjoint case compares both
gradients.
"""
import numpy as np
import pytest

import oracle
from paper_1511_03599_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CHANNELS = [32, 64, 128, 256, 512, 1024, 2048, 4096, 384, 768, 1536, 3072]
TAPS = [1, 2, 3, 4, 5, 8, 11, 16, 17, 24, 32, 40, 64]
SIGMA = {"ci8": 16.0, "ci16": 2000.0, "cf32": 1.0}
TOL = {"c64": 1e-5, "c16": 2e-3}


@pytest.fixture(scope="module")
def ppf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_03599_gb300 import ppf as m
    m.lib()
    return m


def _forward_cases(n, seed):
    rng = np.random.default_rng(seed)
    cases = []
    for _ in range(n):
        C = int(rng.choice(CHANNELS))
        T = int(rng.choice(TAPS))
        in_dtype = str(rng.choice(["ci8", "ci16", "cf32"]))
        out_dtype = str(rng.choice(["c64", "c64", "c16"]))
        ns = int(rng.choice([1, 1, 2, 3, 7]))
        S = int(rng.integers(1, max(2, (3 << 17) // (C * ns))))   # up to ~3.9e5 samples per stream
        cases.append((C, T, in_dtype, out_dtype, S, ns))
    return cases


@pytest.mark.parametrize("case", _forward_cases(40, 20261203))
def test_fuzz_forward(ppf, case):
    C, T, in_dtype, out_dtype, S, ns = case
    scale = 1.0 / np.sqrt(C) if out_dtype == "c16" else 1.0
    h = synth.design_taps(C, T, scale=scale)
    xs = [synth.stream(C, S + T - 1, in_dtype, SIGMA[in_dtype], 9000 + C + T + S + i) for i in range(ns)]
    with ppf.Plan(C, T, h, in_dtype, out_dtype) as plan:
        xd = torch.stack([torch.from_numpy(x).cuda() for x in xs]) if ns > 1 else torch.from_numpy(xs[0]).cuda()
        y = plan.execute(xd, n_streams=ns if ns > 1 else None)
        torch.cuda.synchronize()
        plan.check_device()
    y = y.cpu()
    if out_dtype == "c64":
        got = y.numpy().astype(np.complex128)
    else:
        a = y.float().numpy()
        got = a[..., 0].astype(np.float64) + 1j * a[..., 1].astype(np.float64)
    got = got.reshape(ns, S, C)
    for i, x in enumerate(xs):
        if S <= 64:
            idx = np.arange(S)
        else:
            rng = np.random.default_rng(C + S + i)
            idx = np.unique(np.concatenate([np.arange(T), np.arange(S - T, S), rng.integers(0, S, 48)]))
            idx = idx[(idx >= 0) & (idx < S)]
        ref = oracle.pfb_spectra(x, h, C, T, idx)
        assert np.all(np.isfinite(got[i][idx]))
        err = oracle.rel_l2(got[i][idx], ref)
        assert err <= TOL[out_dtype], f"{case} stream {i}: rel L2 {err:.3e}"


def _adjoint_cases(n, seed):
    rng = np.random.default_rng(seed)
    cases = []
    for _ in range(n):
        C = int(rng.choice(CHANNELS))
        T = int(rng.choice(TAPS))
        in_dtype = str(rng.choice(["ci8", "ci16", "cf32"]))
        ns = int(rng.choice([1, 2, 3]))
        S = int(rng.integers(1, max(2, 40000 // (C * ns))))
        cases.append((C, T, in_dtype, S, ns))
    return cases


@pytest.mark.parametrize("case", _adjoint_cases(16, 4242))
def test_fuzz_adjoint(ppf, case):
    C, T, in_dtype, S, ns = case
    rng = np.random.default_rng(C + 3 * T + S)
    h = synth.design_taps(C, T) + 0.01 * rng.standard_normal(C * T).astype(np.float32)
    xs = np.stack([synth.stream(C, S + T - 1, in_dtype, SIGMA[in_dtype], 600 + i) for i in range(ns)])
    G = (rng.standard_normal((ns, S, C)) + 1j * rng.standard_normal((ns, S, C))).astype(np.complex64)
    with ppf.Plan(C, T, h, in_dtype, "c64") as plan:
        xd = torch.from_numpy(xs if ns > 1 else xs[0]).cuda()
        gx, gh = plan.backward(torch.from_numpy(G if ns > 1 else G[0]).cuda(), xd)
        torch.cuda.synchronize()
        plan.check_device()
    gx = gx.cpu().numpy().astype(np.complex128).reshape(ns, -1)
    gh = gh.cpu().numpy().astype(np.float64)
    ref_gx = np.stack([oracle.pfb_grad_input(G[i].astype(np.complex128), h, C, T) for i in range(ns)])
    ref_gh = sum(oracle.pfb_grad_taps(G[i].astype(np.complex128), xs[i], C, T) for i in range(ns))
    assert oracle.rel_l2(gx, ref_gx) <= 1e-5, case
    assert oracle.rel_l2(gh, ref_gh) <= 1e-4, case


@pytest.mark.parametrize("seed", [7, 8])
def test_fuzz_beams(ppf, seed):
    """A random set of beams (C, T <= 16, spectrum counts) in one persistent launch."""
    from paper_1511_03599_gb300 import beams
    rng = np.random.default_rng(seed)
    n = 10
    C = [int(c) for c in rng.choice([64, 128, 256, 512, 1024, 2048, 4096], n)]
    T = [int(t) for t in rng.integers(1, 17, n)]
    S = [int(s) for s in rng.integers(1, 2000, n)]
    taps = [synth.design_taps(c, t) for c, t in zip(C, T)]
    xs = [synth.stream(c, s + t - 1, "ci8", 16.0, 777 + seed * 100 + i) for i, (c, t, s) in enumerate(zip(C, T, S))]
    bs = beams.BeamSet(C, T, S, taps)
    outs = [torch.empty((s, c), dtype=torch.complex64, device="cuda") for c, s in zip(C, S)]
    bs.bind([torch.from_numpy(x).cuda() for x in xs], outs)
    bs.set_tiling(int(rng.choice([1 << 14, 1 << 17, 1 << 20])))
    bs.execute()
    torch.cuda.synchronize()
    bs.check_device()
    for c, t, x, h, y in zip(C, T, xs, taps, outs):
        assert oracle.rel_l2(y.cpu().numpy(), oracle.pfb(x, h, c, t)) <= 1e-5, (c, t)
    bs.close()
