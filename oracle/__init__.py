"""FP64 CPU oracle for guided-filter non-blind deconvolution (arXiv 1609.01839).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library path
(``paper_1609_01839_gb300``) never imports it and shares no code with it.

Plain, slow, obviously-correct NumPy in float64.  ``numpy.fft`` serves as the
textbook DFT (a library primitive); every other step is the paper's formula
written out, each function citing the passage it follows.  Readings of places
where the paper is silent or garbled are marked "reading:".

Parity status: every function here is pinned by CPU tests against brute force,
closed forms or invariants (tests/test_oracle_*.py), except the end-to-end
ISNR against the paper's Tables 2-3, which is **parity unpinned**: the paper
prints no worked example and its test images are not available.
"""
from .gfdeconv import (  # noqa: F401
    embed_psf, psf_spectrum, grad_weight, rho_eq12, discrepancy_target,
    residual_norm2, f_lambda, solve_lambda, deblur, box_mean, box_mean_truncated, guided_filter,
    guided_filter_color, pad_symmetric, crop,
    isnr, iterate, solve, NONCONVERGED, LAMBDA_LO, LAMBDA_RTOL,
)
from . import adjoint  # noqa: F401  (gradient of the unrolled method, oracle/adjoint.py)
