// Compute kernels for highest MCSH order 0.
#include "gmp_inst.cuh"
GMP_DEFINE_LAUNCHER(0)
