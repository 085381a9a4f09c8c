"""FP64 CPU oracle for the non-orthogonal MRT pseudopotential lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct
reference that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  It shares no code with ``paper_2306_16274_gb300`` (the CUDA path) and
imports nothing from it; the only code both sides see is the seeded input
generator in ``workloads/``, which holds none of the method's arithmetic.

Everything is float64 numpy, written in the order and notation of
Fei et al., "Modeling realistic multiphase flows using a non-orthogonal
multiple-relaxation-time lattice Boltzmann method" (arXiv:2306.16274):

* ``lattice``        velocity sets (Eq. e1, App. C) and weights (text after Eq. e5)
* ``moments``        moment set (Eq. e11), M (Eq. "matrix"), exact M^-1, S (Eq. e12),
                     m^eq (Eq. e13), forcing moments (Eq. e14), D3Q19 extraction (App. C)
* ``eos``            Carnahan-Starling and piecewise-linear EOS (Eqs. e19-e21),
                     square-root pseudopotential (Sec. II C)
* ``lbm``            one time step: density, psi, F_int (Eq. e15), F_ads (Sec. III E),
                     Q (Eq. e18), collision in moment space (Eq. e8 with Eq. e17),
                     back-transform and streaming (Eq. e9), macroscopic update (Sec. II A)
* ``velocity_space`` independent velocity-space forms: Eq. e7 with a dense
                     Lambda = M^-1 S M, and SRT/BGK with Guo forcing (Eqs. e5, e6)

Parity status per function is stated in each module header.
"""
