"""Many beams with uneven C, T and spectrum counts in one persistent launch."""
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
    from paper_1511_03599_gb300 import beams, ppf
    ppf.lib()
    return ppf, beams


BEAMS = [(64, 4, 3000), (128, 8, 700), (256, 16, 333), (512, 8, 517), (1024, 4, 99), (2048, 16, 40),
         (4096, 8, 13), (512, 3, 1), (64, 16, 5000), (256, 5, 250), (4096, 16, 7), (1024, 16, 64)]


def make_set(mods, beams_def, seed=0):
    ppf, beams = mods
    C = [b[0] for b in beams_def]
    T = [b[1] for b in beams_def]
    S = [b[2] for b in beams_def]
    taps = [synth.design_taps(c, t) for c, t in zip(C, T)]
    xs = [synth.stream(c, s + t - 1, "ci8", 16.0, seed + i) for i, (c, t, s) in enumerate(beams_def)]
    bs = beams.BeamSet(C, T, S, taps)
    ins = [torch.from_numpy(x).cuda() for x in xs]
    outs = [torch.empty((s, c), dtype=torch.complex64, device="cuda") for c, s in zip(C, S)]
    bs.bind(ins, outs)
    return bs, xs, taps, ins, outs


def test_beams_match_oracle(mods):
    ppf, _ = mods
    bs, xs, taps, ins, outs = make_set(mods, BEAMS)
    bs.execute()
    torch.cuda.synchronize()
    bs.check_device()
    for (c, t, s), x, h, y in zip(BEAMS, xs, taps, outs):
        assert oracle.rel_l2(y.cpu().numpy(), oracle.pfb(x, h, c, t)) <= 1e-5, (c, t, s)
    bs.close()


@pytest.mark.parametrize("tile_samples,ctas", [(1 << 12, 1), (1 << 16, 0), (1 << 24, 1)])
def test_beams_tiling_does_not_change_results(mods, tile_samples, ctas):
    bs, xs, taps, ins, outs = make_set(mods, BEAMS[:7], seed=50)
    bs.execute()
    ref = [y.clone() for y in outs]
    bs.set_tiling(tile_samples)
    for y in outs:
        y.zero_()
    bs.execute(ctas_per_sm=ctas)
    torch.cuda.synchronize()
    for a, b in zip(ref, outs):
        assert torch.equal(torch.view_as_real(a), torch.view_as_real(b))
    bs.close()


def test_beams_cuda_graph_replay(mods):
    bs, xs, taps, ins, outs = make_set(mods, BEAMS[:6], seed=80)
    bs.execute()
    torch.cuda.synchronize()
    ref = [y.clone() for y in outs]
    g = bs.capture_graph()
    for _ in range(2):
        for y in outs:
            y.zero_()
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(ref, outs):
            assert torch.equal(torch.view_as_real(a), torch.view_as_real(b))
    bs.close()


def test_beams_autotune_and_cache(mods, tmp_path):
    _, beams = mods
    bs, xs, taps, ins, outs = make_set(mods, BEAMS[:5], seed=90)
    cache = str(tmp_path / "tune.json")
    r1 = beams.autotune(bs, tile_candidates=(1 << 14, 1 << 18), cache_path=cache)
    assert not r1["cached"] and r1["tile_samples"] in (1 << 14, 1 << 18)
    r2 = beams.autotune(bs, tile_candidates=(1 << 14, 1 << 18), cache_path=cache)
    assert r2["cached"] and r2["tile_samples"] == r1["tile_samples"]
    bs.execute()
    torch.cuda.synchronize()
    for (c, t, s), x, h, y in zip(BEAMS[:5], xs, taps, outs):
        assert oracle.rel_l2(y.cpu().numpy(), oracle.pfb(x, h, c, t)) <= 1e-5
    bs.close()


def test_beams_reject_unsupported(mods):
    ppf, beams = mods
    with pytest.raises(ppf.PPFError):
        beams.BeamSet([32], [8], [10], [synth.design_taps(32, 8)])
    with pytest.raises(ppf.PPFError):
        beams.BeamSet([512], [32], [10], [synth.design_taps(512, 32)])


def test_beams_wide_and_narrow_tiles_in_one_launch(mods):
    """C >= 1024 beams run as wide tiles (the whole CTA) and C <= 512 beams as narrow
    tiles (half-CTA groups) of the same persistent launch.  The body at C = 1024 is
    the carry kernel's and at C = 4096 the generic kernel's, as ppf_execute picks
    them for int8 input, so those beams are bit-identical to ppf_execute."""
    ppf, _ = mods
    for beams_def in ([(2048, 8, 300), (4096, 4, 100), (512, 8, 200), (2048, 16, 57), (64, 4, 900)],
                      [(2048, 3, 129), (4096, 16, 64)], [(4096, 8, 1), (128, 16, 3)],
                      [(1024, 8, 700), (512, 16, 333), (1024, 3, 65), (512, 4, 1), (256, 8, 90)]):
        bs, xs, taps, ins, outs = make_set(mods, beams_def, seed=120)
        info = bs.info()
        assert bs.launches_per_execute() == 1
        assert info["wide_tiles"] >= 0 and info["tiles"] >= info["wide_tiles"]
        assert (info["wide_tiles"] > 0) == any(c >= 1024 for c, _, _ in beams_def)
        assert (info["tiles"] > info["wide_tiles"]) == any(c < 1024 for c, _, _ in beams_def)
        bs.execute()
        torch.cuda.synchronize()
        bs.check_device()
        for (c, t, s), x, h, xd, y in zip(beams_def, xs, taps, ins, outs):
            assert oracle.rel_l2(y.cpu().numpy(), oracle.pfb(x, h, c, t)) <= 1e-5, (c, t, s)
            if c in (1024, 4096):
                with ppf.Plan(c, t, h, "ci8", "c64") as plan:
                    ref = plan(xd)
                    torch.cuda.synchronize()
                assert torch.equal(torch.view_as_real(ref), torch.view_as_real(y)), (c, t, s)
        bs.close()
