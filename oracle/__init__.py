"""FP64 CPU oracle for k-space-preconditioned PDHG (Ong, Uecker & Lustig, arXiv 1902.09657).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct
restatement of what the GPU library computes, written directly from the paper:
the multi-coil forward model (Sec. 2, Eq. model_i / model), its Kaiser-Bessel
NUFFT approximation (Sec. 6, "following Beatty et al.", oversampling 1.25,
width 4), the l2-optimised diagonal k-space preconditioners (Sec. 5, App. A,
Eq. sc_precond / mc_precond and the fast FFT/NUFFT route), the power method for
lambda_max(P A A^H) (Sec. 6), preconditioned PDHG with the accelerated step-size
schedule (Sec. 4.1) and the l2 / l1-Daubechies-4-wavelet proximal operators
(Sec. 2, Eq. obj).

Only the test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  It shares no code with
the CUDA path and never imports the product package.  NumPy's FFT, ``numpy.i0``
and dense linear algebra are used as library steps; everything else is written
out in the paper's order and notation, in float64.

Parity status per module: every public function is pinned by a ``-m "not gpu"``
test against brute force, closed forms or invariants (see ``tests/test_oracle_*.py``).
"""
from . import nufft, precond, wavelet, solvers  # noqa: F401
