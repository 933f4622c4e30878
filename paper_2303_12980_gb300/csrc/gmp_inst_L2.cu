// Compute kernels for highest MCSH order 2.
#include "gmp_inst.cuh"
GMP_DEFINE_LAUNCHER(2)
