"""ppf_backward_noalloc: the backward pass for callers that cannot allocate.

Some users run the PFB where device allocation is not allowed (a processing
loop with a device-memory budget fixed at start-up, or code where a cudaMalloc
could synchronise the device or fail).  ppf_backward_noalloc keeps its
tap-gradient partial sums in a fixed array inside the library instead of
allocating them.  These tests call it through the C ABI, twice in a row with
different shapes, and compare each result with the FP64 oracle's gradients
and with ppf_backward, within the adjoint tests' tolerances (relative L2 1e-5
for the input gradient, 1e-4 for the tap gradient).  The file is named to be
collected last.
"""
import ctypes

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


def _call(ppf, fn, plan, G, x, S, ns):
    gx = torch.empty_like(x)
    gh = torch.empty(plan.C * plan.T, dtype=torch.float32, device="cuda")
    st = getattr(ppf.lib(), fn)(plan.handle, ctypes.c_void_p(G.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                ctypes.c_void_p(gx.data_ptr()), ctypes.c_void_p(gh.data_ptr()), S, ns,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    ppf.check(st)
    torch.cuda.synchronize()
    return gx, gh


def _oracle_grads(G, x, h, C, T):
    Gn = G.cpu().numpy().astype(np.complex128)
    xn = x.cpu().numpy().astype(np.complex128)
    gx = np.stack([oracle.pfb_grad_input(Gn[i], h, C, T) for i in range(Gn.shape[0])])
    gh = sum(oracle.pfb_grad_taps(Gn[i], xn[i], C, T) for i in range(Gn.shape[0]))
    return gx, gh


def test_noalloc_backward_matches_backward_twice(ppf):
    rng = np.random.default_rng(2024)
    C, T = 256, 16
    h = synth.design_taps(C, T)
    with ppf.Plan(C, T, h, "cf32", "c64") as plan:
        for S, ns in ((700, 3), (129, 1)):
            x = torch.from_numpy((rng.standard_normal((ns, C * (S + T - 1)))
                                  + 1j * rng.standard_normal((ns, C * (S + T - 1)))).astype(np.complex64)).cuda()
            G = torch.from_numpy((rng.standard_normal((ns, S, C))
                                  + 1j * rng.standard_normal((ns, S, C))).astype(np.complex64)).cuda()
            gx_n, gh_n = _call(ppf, "ppf_backward_noalloc", plan, G, x, S, ns)
            gx_r, gh_r = _call(ppf, "ppf_backward", plan, G, x, S, ns)
            plan.check_device()
            ref_gx, ref_gh = _oracle_grads(G, x, h, C, T)
            assert oracle.rel_l2(gx_n.cpu().numpy().reshape(ref_gx.shape), ref_gx) <= 1e-5
            assert oracle.rel_l2(gh_n.cpu().numpy(), ref_gh) <= 1e-4
            assert oracle.rel_l2(gx_n.cpu().numpy(), gx_r.cpu().numpy()) <= 1e-5
            assert oracle.rel_l2(gh_n.cpu().numpy(), gh_r.cpu().numpy()) <= 1e-4


def test_noalloc_grid_is_capped_by_the_fixed_array(ppf):
    """At C=512, T=8 the fixed array holds 524,288 / (8 * 512) = 128 rows of partial
    sums, fewer than the CTAs the plain call launches (one per SM): the capped grid
    still gives the oracle's gradients, twice in a row, with different inputs."""
    C, T, S = 512, 8, 2000
    assert torch.cuda.get_device_properties(0).multi_processor_count > (1 << 19) // (T * C)
    rng = np.random.default_rng(2026)
    h = synth.design_taps(C, T)
    with ppf.Plan(C, T, h, "ci8", "c64") as plan:
        for seed in (1, 2):
            x = synth.stream(C, S + T - 1, "ci8", 16.0, 900 + seed)
            xd = torch.from_numpy(x).cuda()
            G = torch.from_numpy((rng.standard_normal((S, C)) + 1j * rng.standard_normal((S, C))).astype(np.complex64)).cuda()
            gx = torch.empty(C * (S + T - 1), dtype=torch.complex64, device="cuda")
            gh = torch.empty(C * T, dtype=torch.float32, device="cuda")
            st = ppf.lib().ppf_backward_noalloc(plan.handle, ctypes.c_void_p(G.data_ptr()), ctypes.c_void_p(xd.data_ptr()),
                                                ctypes.c_void_p(gx.data_ptr()), ctypes.c_void_p(gh.data_ptr()), S, 1,
                                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            ppf.check(st)
            torch.cuda.synchronize()
            plan.check_device()
            Gn = G.cpu().numpy().astype(np.complex128)
            assert oracle.rel_l2(gx.cpu().numpy(), oracle.pfb_grad_input(Gn, h, C, T)) <= 1e-5
            assert oracle.rel_l2(gh.cpu().numpy(), oracle.pfb_grad_taps(Gn, x, C, T)) <= 1e-4


def test_noalloc_many_streams_match_backward(ppf):
    """CTAs share the batches of all streams, so any stream count fits the fixed array."""
    rng = np.random.default_rng(2025)
    C, T = 256, 16
    h = synth.design_taps(C, T)
    with ppf.Plan(C, T, h, "cf32", "c64") as plan:
        ns, S = 300, 3          # more streams than resident CTAs
        x = torch.from_numpy((rng.standard_normal((ns, C * (S + T - 1)))
                              + 1j * rng.standard_normal((ns, C * (S + T - 1)))).astype(np.complex64)).cuda()
        G = torch.from_numpy((rng.standard_normal((ns, S, C))
                              + 1j * rng.standard_normal((ns, S, C))).astype(np.complex64)).cuda()
        gx_n, gh_n = _call(ppf, "ppf_backward_noalloc", plan, G, x, S, ns)
        gx_r, gh_r = _call(ppf, "ppf_backward", plan, G, x, S, ns)
        plan.check_device()
        ref_gx, ref_gh = _oracle_grads(G, x, h, C, T)
        assert oracle.rel_l2(gx_n.cpu().numpy().reshape(ref_gx.shape), ref_gx) <= 1e-5
        assert oracle.rel_l2(gh_n.cpu().numpy(), ref_gh) <= 1e-4
        assert oracle.rel_l2(gx_n.cpu().numpy(), gx_r.cpu().numpy()) <= 1e-5
        assert oracle.rel_l2(gh_n.cpu().numpy(), gh_r.cpu().numpy()) <= 1e-4


def test_noalloc_rejects_shapes_outside_the_fused_kernel(ppf):
    """C = 512 with T = 16 needs ppf_backward's three-pass path (a g_y scratch):
    ppf_backward runs it, ppf_backward_noalloc returns UNSUPPORTED and
    allocates nothing."""
    C, T, S, ns = 512, 16, 20, 1
    rng = np.random.default_rng(5)
    h = synth.design_taps(C, T)
    with ppf.Plan(C, T, h, "cf32", "c64") as plan:
        x = torch.from_numpy((rng.standard_normal((ns, C * (S + T - 1)))
                              + 1j * rng.standard_normal((ns, C * (S + T - 1)))).astype(np.complex64)).cuda()
        G = torch.from_numpy((rng.standard_normal((ns, S, C))
                              + 1j * rng.standard_normal((ns, S, C))).astype(np.complex64)).cuda()
        gx_r, gh_r = _call(ppf, "ppf_backward", plan, G, x, S, ns)
        ref_gx, ref_gh = _oracle_grads(G, x, h, C, T)
        assert oracle.rel_l2(gx_r.cpu().numpy(), ref_gx) <= 1e-5
        assert oracle.rel_l2(gh_r.cpu().numpy(), ref_gh) <= 1e-4
        with pytest.raises(ppf.PPFError) as ei:
            _call(ppf, "ppf_backward_noalloc", plan, G, x, S, ns)
        assert ei.value.status == 2
