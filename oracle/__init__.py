"""Plain FP64 CPU oracle for the ICWF time step (Albareda, Kelly, Rubio, arXiv 1805.11169).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``
may import or run it.  It shares no code with the CUDA library (the two meet only through the
seeded inputs built by ``workloads``, which hold none of the method's arithmetic).

Modules
-------
``icwf``     the ICWF ansatz step: Hermitian-CWF propagation, Bohmian velocities (Eq. v1/v2),
             matrix elements (Eq. Matrices) in the direct and the rank-k factorised form,
             the coefficient equation (Eq. coeff) by RK4, and grid observables.
``exact2d``  a split-operator solver of the full 2D TDSE (Eq. TDSE), the accuracy reference.
``sampler``  SplitMix64 and the inverse-CDF sampler of initial positions from |Psi0|^2.

Every function is written in complex128 / float64 from the paper's equations; library
primitives (FFT, SVD, Cholesky, triangular solve) serve as single steps.  Parity status of each
function is stated in its docstring; all of them are pinned by the ``-m "not gpu"`` tests
(closed forms, invariants, brute force), except where a docstring says "parity unpinned".
"""
