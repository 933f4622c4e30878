// Compute kernels for highest MCSH order 5.
#include "gmp_inst.cuh"
GMP_DEFINE_LAUNCHER(5)
