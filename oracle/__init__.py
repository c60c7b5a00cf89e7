"""CPU FP64 oracle for the EMSpice 3 EM/TM stress / void / IR-drop hot path.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow reference the CUDA
library is checked against.  Only the tests, __graft_entry__.smoke() and
bench.py's CPU-baseline leg may import it; the product path never does.  It
shares no code with the CUDA library: the two only consume the same seeded
inputs from ems_synth.

Modules:
  flow    tree extraction, temperature / kappa / forcing, IR solve, screen,
          void resistance, the coupled TTF loop (Sec. III, IV-A..D)
  krylov  constant-input block rational Krylov reduction (Sec. IV-E, Alg. 1)
  mlp     FP64 reference for the learned surrogate's MLP
"""
from . import flow  # noqa: F401
