// Entry points of the per-order compute launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define GMP_KIND_FORWARD 0
#define GMP_KIND_VJP 1
#define GMP_KIND_JACOBIAN 2
#define GMP_KIND_BACKWARD 3

namespace gmpk {
struct KParams;
}

#define GMP_DECLARE_LAUNCHER(LV)                                                                \
  cudaError_t gmp_launch_compute_L##LV(int kind, int ns, const gmpk::KParams& K, cudaStream_t st, \
                                      int sm_count, int64_t* launches);
GMP_DECLARE_LAUNCHER(0)
GMP_DECLARE_LAUNCHER(1)
GMP_DECLARE_LAUNCHER(2)
GMP_DECLARE_LAUNCHER(3)
GMP_DECLARE_LAUNCHER(4)
GMP_DECLARE_LAUNCHER(5)
GMP_DECLARE_LAUNCHER(6)
