"""The unfused ablation (ppf_fir then ppf_fft) against the oracle's FIR and DFT."""
import numpy as np
import pytest

import oracle
from paper_1511_03599_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ppf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_03599_gb300 import ppf as m
    m.lib()
    return m


@pytest.mark.parametrize("C,T,S,dt", [(512, 8, 333, "ci8"), (512, 16, 40, "ci16"), (256, 16, 1000, "cf32"),
                                      (256, 3, 17, "ci8"), (512, 1, 5, "cf32"), (64, 8, 900, "ci16"),
                                      (128, 16, 300, "cf32"), (1024, 8, 77, "ci8")])
def test_fir_only_matches_oracle(ppf, C, T, S, dt):
    h = synth.design_taps(C, T)
    x = synth.stream(C, S + T - 1, dt, {"ci8": 16.0, "ci16": 2000.0, "cf32": 1.0}[dt], 10 + T)
    with ppf.Plan(C, T, h, dt, "c64") as plan:
        xd = torch.from_numpy(x).cuda()
        y = plan.fir(xd)
        Y = plan(xd)
        Y2 = plan.fft(y)
        torch.cuda.synchronize()
    ref_y = oracle.fir(x, h, C, T)
    assert oracle.rel_l2(y.cpu().numpy(), ref_y) <= 1e-6
    # the composition equals the fused transform up to FP32 rounding
    assert oracle.rel_l2(Y2.cpu().numpy(), Y.cpu().numpy()) <= 1e-6
    assert oracle.rel_l2(Y2.cpu().numpy(), oracle.dft(ref_y)) <= 1e-5


@pytest.mark.parametrize("C,out_dtype", [(32, "c64"), (512, "c64"), (4096, "c64"), (512, "c16")])
def test_fft_only_matches_oracle(ppf, C, out_dtype):
    rng = np.random.default_rng(C)
    S = 50
    y = (rng.standard_normal((S, C)) + 1j * rng.standard_normal((S, C))).astype(np.complex64)
    if out_dtype == "c16":
        y = y / np.float32(np.sqrt(C))
    with ppf.Plan(C, 4, synth.design_taps(C, 4), "cf32", out_dtype) as plan:
        Y = plan.fft(torch.from_numpy(y).cuda())
        torch.cuda.synchronize()
    got = Y.cpu().numpy() if out_dtype == "c64" else (Y.cpu().float().numpy() @ np.array([1, 1j]))
    assert oracle.rel_l2(got, oracle.dft(y.astype(np.complex128))) <= (1e-5 if out_dtype == "c64" else 2e-3)


def test_fir_only_unsupported_shape(ppf):
    with ppf.Plan(2048, 8, synth.design_taps(2048, 8), "ci8", "c64") as plan:
        with pytest.raises(ppf.PPFError) as ei:
            plan.fir(torch.zeros(2048 * 20 * 2, dtype=torch.int8, device="cuda"))
        assert ei.value.status == 2
