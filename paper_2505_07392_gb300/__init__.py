"""GB300-native IGR Euler stage solver.

One SSP-RK3 step of the 3D compressible Euler equations with information
geometric regularization: velocity gradients and IGR source, warm-started
Jacobi sweeps for the entropic pressure Sigma, 5th-order face
reconstruction, Lax-Friedrichs flux with p + Sigma, flux divergence and the
Runge-Kutta update, all in hand-written CUDA kernels for sm_103a behind the
C ABI declared in include/igr.h.

Submodules:
  inputs   seeded synthetic workloads (grids, jets, initial states)
  igr      ctypes binding of the C ABI (loads libigr.so; fails loudly if it
           is missing)
  build    compiles libigr.so with nvcc for sm_103a
"""
