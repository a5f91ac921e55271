"""GB300-native (sm_103a) solver for the P1 pressure system of the semi-implicit
hybrid FV/FE all-Mach scheme: A = M_alpha + dt^2 K_beta on the primal simplex
mesh, solved matrix-free by (preconditioned) conjugate gradient.

Submodules:
  pressure   -- binding of the C ABI in include/pressure.h (libpressure.so)
  synthetic  -- seeded synthetic meshes / coefficients / right-hand sides
  build      -- nvcc build of libpressure.so
The binding is imported lazily so that the input generator works on machines
without the compiled library.
"""
__version__ = "0.1.0"
