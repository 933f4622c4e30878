// Compute kernels for highest MCSH order 1.
#include "gmp_inst.cuh"
GMP_DEFINE_LAUNCHER(1)
