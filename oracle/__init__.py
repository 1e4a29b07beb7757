"""FP64 CPU oracle for the lattice Boltzmann stream-collide sweep.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, literal restatement
of the method of Bauer, Koestler & Ruede, "lbmpy: Automatic code generation
for efficient parallel lattice Boltzmann methods" (arXiv:2001.11806), used to
check the CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg and reference arm of ``bench.py`` may import it.  The
product package never imports it and shares no code, table or constant
generator with it.

Everything is numpy float64, vectorised over cells only; per-cell formulas are
written in the paper's notation.  Modules:

- ``lattice``   DdQq velocity sets and weights (Sec. III-A).
- ``moments``   moment polynomials, the automatic monomial basis, the
                shear/bulk split and weighted Gram-Schmidt in exact rationals
                (Sec. III-A "Moment Space"), Maxwellian moments (Eqs.
                cont_maxwellian / cont_moment_integral).
- ``collision`` equilibrium (Eq. discrete_eq), SRT (Eq. bgk), TRT, MRT
                (Eq. mrt), Guo forcing, the Smagorinsky model (Sec. III-C)
                and the entropic KBC operator (Eq. entropic_direct_omega_eq).
- ``cumulant``  cumulant collision from the generating function
                (Eq. cumulant_generating_function) in a truncated power-series
                ring.
- ``lbm``       pull streaming, boundaries (UBB listing, halfway bounce-back,
                equilibrium outlet), the time step, macroscopic output, FP64
                reductions and the boundary link mask.
- ``adjoint``   discrete adjoint of the time step by complex-step
                differentiation of the collision and the transposed streaming
                map, plus the kinetic-energy box loss.

Parity status per function is listed in each module header; every function
here is pinned by a ``-m "not gpu"`` test except where a header says
"parity unpinned".
"""
