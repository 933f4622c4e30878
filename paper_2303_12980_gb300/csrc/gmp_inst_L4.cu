// Compute kernels for highest MCSH order 4.
#include "gmp_inst.cuh"
GMP_DEFINE_LAUNCHER(4)
