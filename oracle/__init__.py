"""FP64 CPU oracle of the polyphase filter bank -- test infrastructure only.

Imported by the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py``; never by the product package.
"""
from .fp64 import (as_complex, fir, dft, dft_matrix, pfb, pfb_spectra,  # noqa: F401
                  idft_unnormalised, pfb_grad_input, pfb_grad_taps,
                  fir_effective_flops, efficiency, rel_l2, rel_l2_max_per_spectrum)
