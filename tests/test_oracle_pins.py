"""Pins of the FP64 oracle against things other than itself (CPU only).

Each check ties the oracle to the paper or to mathematics: brute force with an
explicit PFB matrix built by independent loops, the T=1 special case against
numpy's FFT, closed forms for an impulse and a bin-centred tone, linearity,
Parseval, the shift property, finite differences for the adjoint, and the
paper's worked FLOP example.  The mutation tests at the end plant plausible
mistakes in the oracle (on the CPU) and check that some pin catches each one.
"""
import cmath
import math
import os

import numpy as np
import pytest

import oracle
import oracle.fp64 as opfb
from paper_1511_03599_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_complex(rng, n):
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


# ----------------------------------------------------------------- checks ---

def check_bruteforce(C, T, S, seed=0):
    """P1: the PFB as an explicit (S*C) x (C*(S+T-1)) matrix, built entry by entry."""
    rng = np.random.default_rng(seed)
    h = rng.standard_normal(C * T)
    x = _rand_complex(rng, C * (S + T - 1))
    n_in = C * (S + T - 1)
    M = [[0j] * n_in for _ in range(S * C)]
    for s in range(S):
        for m in range(C):
            for r in range(S + T - 1):
                t = r - s                       # raw spectrum r feeds output s through tap r-s
                if 0 <= t < T:
                    for c in range(C):
                        M[s * C + m][r * C + c] += h[t * C + c] * cmath.exp(-2j * math.pi * c * m / C)
    ref = np.array(M) @ x
    got = oracle.pfb(x, h, C, T).reshape(-1)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def check_t1_fft(C, S, seed=1):
    """P2: T=1 and h=1 reduces the PFB to a batched DFT: numpy.fft.fft."""
    rng = np.random.default_rng(seed)
    x = _rand_complex(rng, C * S)
    got = oracle.pfb(x, np.ones(C), C, 1)
    ref = np.fft.fft(x.reshape(S, C), axis=1)
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def check_impulse(C, T, S, r, c0, seed=2):
    """P3: an impulse at (raw spectrum r, channel c0) traces polyphase branch c0 of h.

    Y[s][m] = h[(r-s)C + c0] * exp(-2 pi i c0 m / C) for r-T+1 <= s <= r, else 0.
    """
    rng = np.random.default_rng(seed)
    h = rng.standard_normal(C * T)
    x = np.zeros(C * (S + T - 1), dtype=np.complex128)
    x[r * C + c0] = 1.0
    got = oracle.pfb(x, h, C, T)
    ref = np.zeros((S, C), dtype=np.complex128)
    for s in range(S):
        t = r - s
        if 0 <= t < T:
            for m in range(C):
                ref[s, m] = h[t * C + c0] * cmath.exp(-2j * math.pi * ((c0 * m) % C) / C)
    assert np.max(np.abs(got - ref)) <= 1e-12


def check_tone(C, T, S, k0, A=0.75, seed=3):
    """P4: a tone at the centre of channel k0 makes every raw spectrum identical.

    Y[s][m] = A * sum_c g[c] exp(+2 pi i (k0 - m) c / C), g[c] = sum_t h[tC+c];
    with non-negative taps the peak is bin k0 with value A * sum_c g[c].
    """
    h = synth.design_taps(C, T).astype(np.float64)
    n = np.arange(C * (S + T - 1))
    x = A * np.exp(2j * np.pi * k0 * n / C)
    got = oracle.pfb(x, h, C, T)
    g = h.reshape(T, C).sum(axis=0)
    ref_row = np.array([A * sum(g[c] * cmath.exp(2j * math.pi * (k0 - m) * c / C) for c in range(C))
                        for m in range(C)])
    assert np.max(np.abs(got - ref_row[None, :])) <= 1e-9 * np.max(np.abs(ref_row))
    assert int(np.argmax(np.abs(got[0]))) == k0
    assert abs(got[0, k0] - A * g.sum()) <= 1e-9 * abs(A * g.sum())


def check_linearity(C, T, S, seed=4):
    """P5: linear in x and in h."""
    rng = np.random.default_rng(seed)
    h1, h2 = rng.standard_normal(C * T), rng.standard_normal(C * T)
    x1, x2 = _rand_complex(rng, C * (S + T - 1)), _rand_complex(rng, C * (S + T - 1))
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    lhs = oracle.pfb(a * x1 + b * x2, h1, C, T)
    rhs = a * oracle.pfb(x1, h1, C, T) + b * oracle.pfb(x2, h1, C, T)
    assert np.max(np.abs(lhs - rhs)) <= 1e-10 * np.max(np.abs(rhs))
    lhs = oracle.pfb(x1, 0.3 * h1 - 2.0 * h2, C, T)
    rhs = 0.3 * oracle.pfb(x1, h1, C, T) - 2.0 * oracle.pfb(x1, h2, C, T)
    assert np.max(np.abs(lhs - rhs)) <= 1e-10 * np.max(np.abs(rhs))


def check_parseval(C, T, S, seed=5):
    """P6: sum_m |Y[s][m]|^2 = C * sum_c |y[s][c]|^2 for every spectrum.

    y is computed here directly from Alg. 1's sum, not through the oracle's FIR.
    """
    rng = np.random.default_rng(seed)
    h = rng.standard_normal(C * T)
    x = _rand_complex(rng, C * (S + T - 1))
    Y = oracle.pfb(x, h, C, T)
    y = np.zeros((S, C), dtype=np.complex128)
    for s in range(S):
        for c in range(C):
            y[s, c] = sum(h[t * C + c] * x[(s + t) * C + c] for t in range(T))
    e_freq = np.sum(np.abs(Y) ** 2, axis=1)
    e_time = C * np.sum(np.abs(y) ** 2, axis=1)
    assert np.allclose(e_freq, e_time, rtol=1e-11, atol=0)


def check_shift(C, T, S, seed=6):
    """P7: dropping the first raw spectrum drops the first output spectrum."""
    rng = np.random.default_rng(seed)
    h = rng.standard_normal(C * T)
    x = _rand_complex(rng, C * (S + T - 1))
    full = oracle.pfb(x, h, C, T)
    tail = oracle.pfb(x[C:], h, C, T)
    assert tail.shape == (S - 1, C)
    assert np.max(np.abs(full[1:] - tail)) <= 1e-12 * np.max(np.abs(full))


def check_adjoint_fd(C, T, S, seed=7):
    """The hand-derived gradients against FP64 central finite differences.

    Loss L = Re(sum(conj(G) * Y)), so dL/dY* has the closed form G; the
    oracle's grad_x / grad_h must match numeric derivatives of L.
    """
    rng = np.random.default_rng(seed)
    h = rng.standard_normal(C * T)
    x = _rand_complex(rng, C * (S + T - 1))
    G = _rand_complex(rng, S * C).reshape(S, C)

    def loss(xx, hh):
        return float(np.real(np.sum(np.conj(G) * oracle.pfb(xx, hh, C, T))))

    gx = oracle.pfb_grad_input(G, h, C, T)
    gh = oracle.pfb_grad_taps(G, x, C, T)
    eps = 1e-6
    for i in range(0, C * (S + T - 1), max(1, (C * (S + T - 1)) // 7)):
        d = np.zeros_like(x)
        d[i] = eps
        fd_re = (loss(x + d, h) - loss(x - d, h)) / (2 * eps)
        fd_im = (loss(x + 1j * d, h) - loss(x - 1j * d, h)) / (2 * eps)
        assert abs(gx[i] - (fd_re + 1j * fd_im)) <= 1e-6 * max(1.0, abs(gx[i]))
    for i in range(0, C * T, max(1, (C * T) // 7)):
        d = np.zeros_like(h)
        d[i] = eps
        fd = (loss(x, h + d) - loss(x, h - d)) / (2 * eps)
        assert abs(gh[i] - fd) <= 1e-6 * max(1.0, abs(gh[i]))


def check_flop_example():
    """P8: the paper's worked FLOP example (Sec. 4.1), read from a golden file."""
    with open(os.path.join(GOLDEN, "fir_flops_example.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for T, C, S, t, flops in rows:
        got = oracle.fir_effective_flops(int(S), int(C), int(T)) / float(t)
        assert got == float(flops)


ALL_CHECKS = [
    lambda: check_bruteforce(4, 3, 3),
    lambda: check_t1_fft(16, 5),
    lambda: check_impulse(8, 3, 6, r=4, c0=5),
    lambda: check_tone(16, 4, 3, k0=5),
    lambda: check_linearity(8, 3, 5),
    lambda: check_parseval(8, 2, 3),
    lambda: check_shift(8, 3, 6),
    lambda: check_adjoint_fd(4, 2, 3),
]


# ------------------------------------------------------------------ tests ---

@pytest.mark.parametrize("C,T,S", [(2, 1, 4), (2, 3, 2), (4, 2, 3), (8, 3, 2), (8, 1, 1)])
def test_bruteforce_matrix(C, T, S):
    check_bruteforce(C, T, S)


@pytest.mark.parametrize("C,S", [(8, 3), (64, 7), (256, 2), (12, 4)])
def test_t1_is_batched_fft(C, S):
    check_t1_fft(C, S)


@pytest.mark.parametrize("C,T,S,r,c0", [(8, 3, 6, 4, 5), (16, 8, 12, 9, 0), (32, 4, 5, 0, 31), (8, 2, 3, 3, 7)])
def test_impulse_traces_polyphase_branch(C, T, S, r, c0):
    check_impulse(C, T, S, r, c0)


@pytest.mark.parametrize("C,T,k0", [(16, 4, 5), (32, 8, 0), (64, 2, 63)])
def test_tone_lands_in_its_bin(C, T, k0):
    check_tone(C, T, 3, k0)


def test_linearity():
    check_linearity(8, 3, 5)
    check_linearity(32, 4, 3)


def test_parseval():
    check_parseval(8, 2, 3)
    check_parseval(16, 3, 2)


def test_shift():
    check_shift(8, 3, 6)
    check_shift(32, 8, 4)


def test_adjoint_finite_differences():
    check_adjoint_fd(4, 2, 3)
    check_adjoint_fd(8, 3, 2)


def test_adjoint_inner_product_identity():
    """<A x, G> = <x, A^H G> for the FIR+DFT map and its oracle adjoint."""
    rng = np.random.default_rng(11)
    C, T, S = 16, 4, 5
    h = rng.standard_normal(C * T)
    x = _rand_complex(rng, C * (S + T - 1))
    G = _rand_complex(rng, S * C).reshape(S, C)
    lhs = np.vdot(G, oracle.pfb(x, h, C, T))
    rhs = np.vdot(oracle.pfb_grad_input(G, h, C, T), x)
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_flop_count_worked_example():
    check_flop_example()


def test_efficiency_limits():
    """epsilon = S/(S+T-1): 1 for T=1, -> 1 as S grows, 1/T for S=1 (Sec. 4.1)."""
    assert oracle.efficiency(10, 1) == 1.0
    assert oracle.efficiency(1, 8) == pytest.approx(1 / 8)
    assert oracle.efficiency(10 ** 7, 8) > 0.999999


def test_integer_inputs_are_exact_and_signed():
    """Interleaved int8 / int16 samples map to their integer values (incl. -128)."""
    raw = np.array([[-128, 127], [0, -1]], dtype=np.int8)
    z = oracle.as_complex(raw)
    assert z[0] == -128 + 127j and z[1] == -1j
    raw16 = np.array([[-32768, 32767]], dtype=np.int16)
    assert oracle.as_complex(raw16)[0] == -32768 + 32767j


def test_sampled_rows_match_full():
    rng = np.random.default_rng(12)
    C, T, S = 32, 4, 9
    h = rng.standard_normal(C * T).astype(np.float32)
    x = synth.stream(C, S + T - 1, "ci8", 16.0, 5)
    full = oracle.pfb(x, h, C, T)
    idx = [0, 3, 8]
    assert np.max(np.abs(oracle.pfb_spectra(x, h, C, T, idx) - full[idx])) <= 1e-9


def test_rel_l2():
    a = np.array([3 + 4j, 0])
    assert oracle.rel_l2(a, a) == 0.0
    assert oracle.rel_l2(np.array([3 + 4j, 1]), a) == pytest.approx(0.2)


def test_rel_l2_max_per_spectrum():
    # two spectra of two bins: errors 0.2 and 0.5 of their own norms
    ref = np.array([[3 + 4j, 0], [0, 2]])
    got = np.array([[3 + 4j, 1], [0, 2 + 1j]])
    assert oracle.rel_l2_max_per_spectrum(ref, ref) == 0.0
    assert oracle.rel_l2_max_per_spectrum(got, ref) == pytest.approx(0.5)
    # the whole-output ratio is smaller: sqrt(1 + 1) / sqrt(25 + 4)
    assert oracle.rel_l2(got, ref) == pytest.approx(np.sqrt(2 / 29))
    # an all-zero reference spectrum contributes its absolute error
    assert oracle.rel_l2_max_per_spectrum(np.array([[0, 3j]]), np.array([[0, 0]])) == pytest.approx(3.0)
    with pytest.raises(ValueError):
        oracle.rel_l2_max_per_spectrum(np.zeros((2, 3)), np.zeros((3, 2)))


# ------------------------------------------------------- mutation tests ---
# Each mutant is a plausible mistake planted in the oracle itself (via
# monkeypatch); at least one pin above must fail for it.

def _fir_reversed_taps(x, h, C, T):       # Eq. 1 read as a convolution
    return _orig_fir(x, np.asarray(h).reshape(T, C)[::-1].reshape(-1), C, T)


def _fir_dropped_last_tap(x, h, C, T):
    hh = np.array(h, dtype=np.float64).reshape(T, C)
    hh[-1] = 0
    return _orig_fir(x, hh.reshape(-1), C, T)


def _fir_transposed_taps(x, h, C, T):     # h[c*T + t] instead of h[t*C + c]
    return _orig_fir(x, np.asarray(h).reshape(C, T).T.reshape(-1), C, T)


def _fir_channel_off_by_one(x, h, C, T):
    return np.roll(_orig_fir(x, h, C, T), 1, axis=1)


def _dft_matrix_wrong_sign(C):
    return np.conj(_orig_dft_matrix(C))


def _dft_matrix_normalised(C):
    return _orig_dft_matrix(C) / C


def _dft_matrix_transposed_index(C):      # exp(-2 pi i c / C) ignoring m
    c = np.arange(C)
    return np.exp(-2j * np.pi * np.outer(c, np.ones(C, dtype=np.int64)) / C)


_orig_fir = opfb.fir
_orig_dft_matrix = opfb.dft_matrix

MUTANTS = [
    ("fir", _fir_reversed_taps),
    ("fir", _fir_dropped_last_tap),
    ("fir", _fir_transposed_taps),
    ("fir", _fir_channel_off_by_one),
    ("dft_matrix", _dft_matrix_wrong_sign),
    ("dft_matrix", _dft_matrix_normalised),
    ("dft_matrix", _dft_matrix_transposed_index),
]


@pytest.mark.parametrize("name,mutant", MUTANTS, ids=[m[1].__name__ for m in MUTANTS])
def test_pins_catch_planted_mistakes(monkeypatch, name, mutant):
    monkeypatch.setattr(opfb, name, mutant)
    monkeypatch.setattr(oracle, name, mutant, raising=False)
    failed = 0
    for chk in ALL_CHECKS:
        try:
            chk()
        except AssertionError:
            failed += 1
    assert failed >= 1, "no pin caught the planted mistake"


def test_pins_pass_unmutated():
    for chk in ALL_CHECKS:
        chk()


# ------------------------------------------------------------ generators ---

def test_taps_design_properties():
    """sinc x Hamming of length CT: symmetric, peak at the centre, branch sums near 1."""
    C, T = 512, 8
    h = synth.design_taps(C, T).astype(np.float64)
    assert h.dtype == np.float64 and h.shape == (C * T,)
    assert np.allclose(h, h[::-1], atol=1e-7)
    g = h.reshape(T, C).sum(axis=0)
    assert 0.99 < g.min() and g.max() < 1.001
    hn = synth.design_taps(4, 2, window="hanning")
    assert hn[0] == 0.0 and hn[-1] == 0.0


def test_stream_recipe():
    x = synth.stream(64, 100, "ci8", 16.0, 1, ((3, 32.0),))
    assert x.dtype == np.int8 and x.shape == (6400, 2)
    assert abs(x.astype(np.float64).std() - 16.0 * math.sqrt(1 + 0.5 * 4)) < 1.5
    x2 = synth.stream(64, 100, "ci8", 16.0, 1, ((3, 32.0),))
    assert np.array_equal(x, x2)
    xi = synth.stream(8, 10, "ci16", 2000.0, 2)
    assert xi.dtype == np.int16 and np.abs(xi.astype(np.int32)).max() <= 32767
