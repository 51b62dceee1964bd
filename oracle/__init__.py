"""FP64 CPU oracle for the time-dependent weighting field H(x, t) and Eq. 1.

TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may import,
call, link or run this package; only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` do.  It shares no code with the CUDA
path.

The oracle is a plain, slow, direct restatement of the method: numpy/scipy in
float64, direct (non-FFT) spectral sums, library least squares (QR) and a
library symmetric-definite eigensolver.  The paper (arXiv 2605.13987) does not
print its equations beyond Eq. 1 and the column resistance formula of Sec. 5;
every step below is the reading of its Abstract / Sec. 1 / Sec. 3 sentences
listed in the module docstrings:

* ``greens``   band-limited periodic fundamental solution (Abstract; Sec. 3:
               spectra multiplied or divided by |k|^2), plus an independent
               Ewald lattice sum used only as a pin.
* ``geometry`` columns, point sources, collocation points, the resistive line
               (Sec. 5: R = 4 rho L / (pi d^2)).
* ``fit``      point-charge magnitudes fitted to the electrode boundary values
               (Abstract: fundamental solutions impose the boundary
               conditions; Sec. 3: charges adjusted in magnitude).
* ``relax``    the quasi-static relaxation in time (Abstract: third-order
               quasi-static PDE; Sec. 3: forward-Euler iteration, kept here as
               a cross-check of the exact modal exponential).
* ``extend``   pseudo-spectral extension of the potential/field into the bulk
               at each time sample (Abstract; Sec. 1: discrete Fourier
               transforms).
* ``eq1``      the Ramo-Shockley-Riegler convolution, Eq. 1.
* ``electronics`` CR-(RC)^n shaping of the currents (parameterised; the paper
               gives no transfer function).
* ``features`` signal-shape features of the currents (amplitude, peak time,
               charge, threshold and constant-fraction crossings) and their
               sensitivities, for the geometry scans of Sec. 5.

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``.
The brute-force finite-difference model (``bruteforce``) is pinned in its parts
(the Laplacian's spectrum, parallel plates, the Schur complement against its
definition); its agreement with the spectral fit is a loose consistency check
between two different discretisations (~4-9 % on the single cell), parity
unpinned for that one comparison.
"""
from . import greens, geometry, fit, relax, extend, eq1, bruteforce  # noqa: F401
from .pipeline import solve, Solution  # noqa: F401
