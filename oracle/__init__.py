"""FP64 CPU oracle of the lattice method of arXiv:2006.15122.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import, call, link or execute anything in this
package.  The CUDA library never does, and nothing here imports it: the two
share no code, header, helper, table or constant generator.

What it computes (each function cites the passage it follows):
  core.py          ctypes front of lattice_oracle.c: scalar kernels, energies,
                   VV2/VVn (section 4.3.2), staggered leapfrog scheme III
                   (section 4.2.1), compact U(1) kernels, energies, Gauss law
                   and staggered leapfrog (sections 5.3, 5.4), compact U(1) VVn
                   (5.3.2, 5.3.3), prescribed fluid background (4.1), explicit
                   RK4 (4.3.1), Gauss-Legendre (3.4.2, 4.3.3), SU(2)-Higgs
                   kernels, energies, Gauss law and VVn (section 6), and the
                   SU(2) x U(1) doublet with a singlet (section 8.3)
  ic.py            initial conditions of section 7
  spectra.py       DFT convention and power spectra (sections 3.1, 4.4.2)
  philox.py        Philox4x32-10, the counter-based generator of the draws
  mlp.py           FP64 reference of the surrogate MLP (forward, loss, gradient)

Pins (tests/test_oracle_*.py, run with -m "not gpu") check it against closed
forms: exact per-mode dispersion of the free lattice field, the Jacobi-
elliptic homogeneous phi^4 solution, a high-accuracy ODE solve of the
expanding homogeneous mode, symplectic convergence orders, reversibility,
summation by parts, Parseval, the Gauss law to round-off, gauge invariance,
energy conservation and Philox known-answer vectors.
"""
from . import core, ic, mlp, philox, spectra  # noqa: F401
from .core import (VV2, VV4, VV6, VV8, VV10, ScalarLattice, ScalarModel, SU2Lattice,  # noqa: F401
                   SU2Model, SU2U1Lattice, SU2U1Model, U1Lattice, U1Model)
