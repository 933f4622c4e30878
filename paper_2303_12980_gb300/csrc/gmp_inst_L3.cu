// Compute kernels for highest MCSH order 3.
#include "gmp_inst.cuh"
GMP_DEFINE_LAUNCHER(3)
