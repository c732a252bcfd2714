"""Plain FP64 CPU oracle for the Fourier x Chebyshev generalized-tau IMEX step.

THIS PACKAGE IS TEST INFRASTRUCTURE.  It exists only to check the CUDA path.
Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or run it.  The product
package never imports it, and it never imports the product package: the two
share no code.  The single module both sides use is ``seeded_inputs`` (random
draws and workload sizes only, none of the method's arithmetic).

Everything here is written for a reader checking it against the paper by eye:
dense matrices in the plain Chebyshev-T basis, block-concatenated variables
(no interleaving, no Dirichlet recombination, no real-ification), explicit
stage formulas, numpy.fft for the Fourier axis and an explicit T_n(x_i)
matrix for the Chebyshev axis (no DCT).

Modules
-------
bases          Fourier / Chebyshev grids, transforms and operator matrices
               (Sec. "Fourier basis", "Chebyshev basis", "Scaled transforms &
               dealiasing", Appendix "Spectral operator matrices").
problem        generic first-order tau pencil assembly in the T basis
               (Sec. "Matrix construction", "A general sparse tau method").
rb             Rayleigh-Benard equations, nonlinear RHS, initial state
               (the workload; the paper does not write these equations).
timesteppers   IMEX Runge-Kutta and multistep (SBDF) steppers
               (Sec. "Timesteppers", Eqs. for B^n_p and B^i_p).

Parity status
-------------
Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
library routines used as independent definitions, brute force, or textbook
values, except the long nonlinear Rayleigh-Benard trajectories, whose only
check is the composition of pinned pieces: parity unpinned for
``rb.RBSystem`` runs beyond the linear regime.
"""
