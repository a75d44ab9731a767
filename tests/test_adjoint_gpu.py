"""The hand-written adjoint (ppf_backward) and the autograd glue, on the GPU.

Gradients are compared with the FP64 oracle's analytic gradients (which the
CPU tests pin to central finite differences), and with directional finite
differences of the GPU forward itself (exact for a map linear in x and h, up
to FP32 rounding).  Tolerances: relative L2 <= 1e-5 for grad_x (a per-sample
linear map like the forward) and <= 1e-4 for grad_h (sums of up to
streams*S products per coefficient, FP32 accumulation).
"""
import numpy as np
import pytest

import oracle
from paper_1511_03599_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_03599_gb300 import autograd, ppf
    ppf.lib()
    return ppf, autograd


def crand(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


@pytest.mark.parametrize("C,T,S,ns", [(256, 16, 100, 1), (256, 8, 37, 3), (128, 3, 333, 2), (64, 1, 70, 1),
                                      (64, 16, 1, 2), (256, 16, 2000, 1), (256, 16, 8192, 3), (128, 8, 20000, 2),
                                      (64, 16, 40000, 1)])
def test_backward_matches_oracle(mods, C, T, S, ns):
    ppf, _ = mods
    rng = np.random.default_rng(C + T + S + ns)
    h = synth.design_taps(C, T) + 0.01 * rng.standard_normal(C * T).astype(np.float32)
    x = crand(rng, ns, C * (S + T - 1))
    G = crand(rng, ns, S, C)
    with ppf.Plan(C, T, h, "cf32", "c64") as plan:
        gx, gh = plan.backward(torch.from_numpy(G).cuda(), torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        plan.check_device()
    gx = gx.cpu().numpy().astype(np.complex128)
    gh = gh.cpu().numpy().astype(np.float64)
    ref_gx = np.stack([oracle.pfb_grad_input(G[i].astype(np.complex128), h, C, T) for i in range(ns)])
    ref_gh = sum(oracle.pfb_grad_taps(G[i].astype(np.complex128), x[i].astype(np.complex128), C, T)
                 for i in range(ns))
    assert oracle.rel_l2(gx, ref_gx) <= 1e-5
    assert oracle.rel_l2(gh, ref_gh) <= 1e-4


def test_backward_single_outputs(mods):
    """grad_in only / grad_taps only give the same numbers as both together."""
    ppf, _ = mods
    rng = np.random.default_rng(3)
    C, T, S = 256, 16, 300
    h = synth.design_taps(C, T)
    x = torch.from_numpy(crand(rng, C * (S + T - 1))).cuda()
    G = torch.from_numpy(crand(rng, S, C)).cuda()
    with ppf.Plan(C, T, h, "cf32", "c64") as plan:
        gx, gh = plan.backward(G, x)
        gx1, none1 = plan.backward(G, x, want_taps=False)
        none2, gh2 = plan.backward(G, x, want_input=False)
    assert none1 is None and none2 is None
    assert torch.equal(gx, gx1) and torch.equal(gh, gh2)


def test_backward_input_must_have_the_plan_type(mods):
    ppf, _ = mods
    with ppf.Plan(256, 8, synth.design_taps(256, 8), "ci8", "c64") as plan:
        with pytest.raises(TypeError):      # the input must have the plan's input type
            plan.backward(torch.zeros(4, 256, dtype=torch.complex64, device="cuda"),
                          torch.zeros(11 * 256, dtype=torch.complex64, device="cuda"))


def test_autograd_directional_finite_differences(mods):
    """d/deps L(x + eps dx, h + eps dh) at 0 equals <grad_x, dx> + <grad_h, dh>."""
    ppf, autograd = mods
    rng = np.random.default_rng(4)
    C, T, S, ns = 256, 16, 64, 2
    m = autograd.PolyphaseFilterBank(C, T, synth.design_taps(C, T)).cuda()
    x = torch.from_numpy(crand(rng, ns, (S + T - 1), C)).cuda().requires_grad_(True)
    W = torch.from_numpy(crand(rng, ns, S, C)).cuda()
    loss = torch.real(torch.sum(torch.conj(W) * m(x)))
    loss.backward()
    dx = torch.from_numpy(crand(rng, ns, (S + T - 1), C)).cuda()
    dh = torch.from_numpy(rng.standard_normal(C * T).astype(np.float32)).cuda()
    with torch.no_grad():
        h0 = m.taps.detach().clone()
        eps = 1e-2
        def L(sgn):
            m.taps.copy_(h0 + sgn * eps * dh)
            return torch.real(torch.sum(torch.conj(W) * m(x + sgn * eps * dx))).double()
        fd = (L(1) - L(-1)) / (2 * eps)
        m.taps.copy_(h0)
    pred = torch.real(torch.sum(torch.conj(x.grad) * dx)).double() + torch.sum(m.taps.grad * dh).double()
    assert abs(float(fd - pred)) <= 1e-4 * abs(float(pred)) + 1e-3


def test_autograd_matches_oracle_gradients(mods):
    ppf, autograd = mods
    rng = np.random.default_rng(5)
    C, T, S = 128, 8, 200
    h = synth.design_taps(C, T)
    m = autograd.PolyphaseFilterBank(C, T, h).cuda()
    xn = crand(rng, C * (S + T - 1))
    x = torch.from_numpy(xn).cuda().requires_grad_(True)
    Y = m(x)
    G = crand(rng, S, C)
    Y.backward(torch.from_numpy(G).cuda())
    ref_gx = oracle.pfb_grad_input(G.astype(np.complex128), h, C, T)
    ref_gh = oracle.pfb_grad_taps(G.astype(np.complex128), xn.astype(np.complex128), C, T)
    assert oracle.rel_l2(x.grad.cpu().numpy(), ref_gx) <= 1e-5
    assert oracle.rel_l2(m.taps.grad.cpu().numpy(), ref_gh) <= 1e-4
    # the forward through the module is the plain transform
    assert oracle.rel_l2(Y.detach().cpu().numpy(), oracle.pfb(xn.astype(np.complex128), h, C, T)) <= 1e-5


def test_batched_forward_matches_per_stream(mods):
    ppf, _ = mods
    rng = np.random.default_rng(6)
    C, T, S, ns = 512, 8, 99, 5
    h = synth.design_taps(C, T)
    x = np.stack([synth.stream(C, S + T - 1, "ci8", 16.0, 100 + i) for i in range(ns)])
    with ppf.Plan(C, T, h, "ci8", "c64") as plan:
        yb = plan(torch.from_numpy(x).cuda(), n_streams=ns).cpu()
        for i in range(ns):
            yi = plan(torch.from_numpy(x[i]).cuda()).cpu()
            assert torch.equal(torch.view_as_real(yb[i]), torch.view_as_real(yi))
    ref = oracle.pfb(x[2], h, C, T)
    assert oracle.rel_l2(yb[2].numpy(), ref) <= 1e-5


def test_backward_timeout_path(mods):
    ppf, _ = mods
    rng = np.random.default_rng(7)
    C, T, S = 256, 16, 500
    h = synth.design_taps(C, T)
    x = torch.from_numpy(crand(rng, C * (S + T - 1))).cuda()
    G = torch.from_numpy(crand(rng, S, C)).cuda()
    with ppf.Plan(C, T, h, "cf32", "c64") as plan:
        plan.set_debug_flags(1)
        _, gh_bad = plan.backward(G, x)
        with pytest.raises(ppf.PPFError) as ei:
            plan.check_device()
        assert ei.value.status == 5
        # the partial sums of CTAs that gave up were never written: the tap
        # gradient of that call is NaN, not silently wrong
        assert torch.isnan(gh_bad).all()
        plan.set_debug_flags(0)
        gx, gh = plan.backward(G, x)
        plan.check_device()
    ref_gh = oracle.pfb_grad_taps(G.cpu().numpy().astype(np.complex128), x.cpu().numpy().astype(np.complex128), C, T)
    assert oracle.rel_l2(gh.cpu().numpy(), ref_gh) <= 1e-4


def test_adam_fit_reduces_leakage(mods):
    """Noisy sinc-Hamming taps fitted by Adam through the adjoint: leakage falls."""
    from paper_1511_03599_gb300 import fit
    r = fit.fit_taps(C=64, T=8, n_streams=8, S=256, steps=40, lr=2e-3)
    loss = r["loss"]
    assert all(np.isfinite(loss))
    assert loss[-1] < 0.5 * loss[0], loss[:3] + loss[-3:]


def test_leakage_loss_gradient_matches_finite_difference(mods):
    """d(leakage)/d(taps) along a random direction, GPU adjoint vs FP64 oracle finite differences."""
    from paper_1511_03599_gb300 import autograd, fit
    C, T, S, ns = 64, 4, 48, 3
    x, k, _ = synth.tone_set(C, S + T - 1, ns, 5)
    h = synth.noisy_taps(C, T, 1e-2, 6)
    m = autograd.PolyphaseFilterBank(C, T, h).cuda()
    loss = fit.leakage_loss(m(x), k)
    loss.backward()
    g = m.taps.grad.double().cpu().numpy()
    xn = x.cpu().numpy().astype(np.complex128)
    d = np.random.default_rng(7).standard_normal(C * T)

    def L(hh):
        Y = np.stack([oracle.pfb(xn[i], hh, C, T) for i in range(ns)])
        P = (np.abs(Y) ** 2).sum(axis=1)
        dist = (np.arange(C)[None, :] - np.asarray(k)[:, None]) % C
        inband = (dist <= 1) | (dist >= C - 1)
        return float(((P * ~inband).sum(axis=1) / P.sum(axis=1)).mean())

    eps = 1e-4
    fd = (L(h.astype(np.float64) + eps * d) - L(h.astype(np.float64) - eps * d)) / (2 * eps)
    assert abs(fd - g @ d) <= 1e-3 * abs(fd) + 1e-6


def test_closed_form_leakage_gradient_matches_autograd(mods):
    """The fit's closed-form loss gradient wrt the spectra equals autograd's of leakage_loss."""
    from paper_1511_03599_gb300 import fit
    rng = np.random.default_rng(11)
    ns, S, C = 4, 33, 64
    Y = torch.from_numpy(crand(rng, ns, S, C)).cuda().requires_grad_(True)
    k = rng.integers(0, C, ns)
    ref = fit.leakage_loss(Y, k)
    ref.backward()
    loss, gY = fit.leakage_loss_and_grad(Y.detach(), fit._inband(k, C, Y.device))
    assert abs(float(loss) - float(ref)) <= 1e-6 * abs(float(ref))
    assert oracle.rel_l2(gY.cpu().numpy(), Y.grad.cpu().numpy()) <= 1e-5


def _check_backward(ppf, C, T, S, ns, in_dtype, flags=0):
    """Both gradients of ppf_backward against the oracle's; returns them."""
    rng = np.random.default_rng(C + T + S + ns)
    sig = {"ci8": 16.0, "ci16": 2000.0, "cf32": 1.0}[in_dtype]
    h = synth.design_taps(C, T) + 0.01 * rng.standard_normal(C * T).astype(np.float32)
    xs = np.stack([synth.stream(C, S + T - 1, in_dtype, sig, 700 + i) for i in range(ns)])
    G = crand(rng, ns, S, C)
    with ppf.Plan(C, T, h, in_dtype, "c64") as plan:
        plan.set_debug_flags(flags)
        xd = torch.from_numpy(xs if ns > 1 else xs[0]).cuda()
        gx, gh = plan.backward(torch.from_numpy(G if ns > 1 else G[0]).cuda(), xd)
        torch.cuda.synchronize()
        plan.check_device()
    gx = gx.cpu().numpy().astype(np.complex128).reshape(ns, -1)
    gh = gh.cpu().numpy().astype(np.float64)
    ref_gx = np.stack([oracle.pfb_grad_input(G[i].astype(np.complex128), h, C, T) for i in range(ns)])
    ref_gh = sum(oracle.pfb_grad_taps(G[i].astype(np.complex128), xs[i], C, T) for i in range(ns))
    assert oracle.rel_l2(gx, ref_gx) <= 1e-5
    assert oracle.rel_l2(gh, ref_gh) <= 1e-4
    return gx, gh


@pytest.mark.parametrize("C,T,S,ns,in_dtype", [(512, 8, 300, 2, "cf32"), (512, 8, 1000, 1, "ci8"),
                                               (512, 5, 77, 3, "ci16"), (256, 16, 500, 2, "ci8"),
                                               (128, 4, 900, 1, "ci16"), (512, 1, 40, 1, "ci8")])
def test_backward_wide_channels_and_integer_input(mods, C, T, S, ns, in_dtype):
    """The fused adjoint at C = 512 (inverse DFT spread over the CTA) and with
    8/16-bit input (the input gradient is complex FP32 per input sample)."""
    _check_backward(mods[0], C, T, S, ns, in_dtype)


@pytest.mark.parametrize("C,T,S,ns,in_dtype", [(512, 32, 200, 2, "ci8"), (512, 16, 150, 1, "cf32"),
                                               (512, 64, 90, 1, "ci16"), (4096, 8, 40, 2, "ci16"),
                                               (1024, 5, 50, 1, "ci8"), (2048, 17, 30, 1, "cf32"),
                                               (32, 64, 100, 1, "cf32"), (32, 4, 1000, 3, "ci8"),
                                               (384, 3, 90, 2, "ci8"), (768, 16, 33, 3, "ci16"),
                                               (3072, 2, 20, 1, "cf32"), (256, 40, 1, 2, "ci8"),
                                               (64, 64, 2, 1, "ci16")])
def test_backward_three_pass_shapes(mods, C, T, S, ns, in_dtype):
    """Shapes outside the fused adjoint kernel (C = 32, C >= 1024, C = 3*2^k,
    T up to 64, T > 8 at C = 512): inverse DFT, grad_in and tap-correlation
    passes, against the oracle; ragged tiles, one spectrum, many taps."""
    _check_backward(mods[0], C, T, S, ns, in_dtype)


@pytest.mark.parametrize("C,T,S,ns,in_dtype", [(256, 16, 500, 2, "ci8"), (512, 8, 300, 1, "cf32"),
                                               (512, 8, 700, 2, "ci8"), (512, 3, 51, 3, "ci16"),
                                               (64, 1, 70, 3, "ci16")])
def test_three_pass_adjoint_matches_fused(mods, C, T, S, ns, in_dtype):
    """Where the fused kernel exists, the three-pass path (forced by the
    debug flag) gives the same gradients within FP32 rounding."""
    ppf = mods[0]
    gx_f, gh_f = _check_backward(ppf, C, T, S, ns, in_dtype)
    gx_u, gh_u = _check_backward(ppf, C, T, S, ns, in_dtype, flags=2)
    assert oracle.rel_l2(gx_u, gx_f) <= 1e-6
    assert oracle.rel_l2(gh_u, gh_f) <= 1e-5
