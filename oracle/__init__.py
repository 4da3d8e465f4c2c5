"""FP64 CPU oracle for the staggered Dslash / CG / force path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, numpy code that states what the CUDA path must compute, written from the
paper's definitions (arXiv:1309.0551, Srinivasan, "Optimizing the performance of Lattice
Gauge Theory simulations with Streaming SIMD extensions") and, where the paper is silent,
from the readings listed per function.  Only the tests, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference arm may import it; the library never does, and the
oracle imports nothing from the library.  It shares no code with the CUDA path: the only
common module is ``synth`` (seeded random inputs, none of the method's arithmetic).

Modules
  geometry   lattice coordinates, parity, staggered phases, checkerboard <-> full maps
  su3        the fifteen SU(3) routines of Table 1 (Sec. 4), incl. Eq. (1.1)-(2.3)
  precision  storage rounding (bf16, fp16, fp32) and 12-real link compression
  dslash     stencil and dense staggered D, even/odd blocks, normal operator m^2 - D^2
  cg         FP64 conjugate gradient and the mixed-precision reliable-update CG
  force      action S = Re chi^dag (m^2 - D^2) chi, dS/dchi, dS/dU and its TA projection
  improved   improved staggered Dslash (one-hop fat + three-hop Naik links), long-link builder
  md         molecular-dynamics link and momentum updates (exp, reunitarisation, leapfrog)
  wilson     Wilson hopping term (DeGrand-Rossi gammas) and its half-spinor form (Table 1 hwvec)
  cxx        the FP64 C++ oracle (cpp/oracle.cpp: Dslash, M, CG, Table 1 products), plain loops
             parallel over sites, timed on the host cores by bench.py; pinned by the same
             brute-force, invariant and closed-form checks, and against this numpy code

Every function is pinned by a ``-m "not gpu"`` test against something other than itself
(brute force, closed forms, invariants, finite differences); see ``tests/test_oracle_*.py``.
"""
from . import geometry, su3, precision, dslash, cg, force, improved, md, wilson  # noqa: F401
