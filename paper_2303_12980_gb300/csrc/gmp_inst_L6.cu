// Compute kernels for highest MCSH order 6.
#include "gmp_inst.cuh"
GMP_DEFINE_LAUNCHER(6)
