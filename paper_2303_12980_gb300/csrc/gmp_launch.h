// Entry points of the per-order compute launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define GMP_KIND_FORWARD 0
#define GMP_KIND_VJP 1
#define GMP_KIND_JACOBIAN 2
#define GMP_KIND_BACKWARD 3
#define GMP_KIND_BACKWARD_VIRIAL 4  // backward + per-structure strain derivative

namespace gmpk {
struct KParams;
}

// Launch shape of a compute kernel (chosen by the autotuner or defaults).
struct GmpShape {
  int tile;   // forward tile: 16 pairs (two lanes per pair) or 32 (one lane per pair)
  int warps;  // warps per CTA, 0 = largest that fits
};

#define GMP_DECLARE_LAUNCHER(LV)                                                                \
  cudaError_t gmp_launch_compute_L##LV(int kind, int ns, const gmpk::KParams& K, GmpShape shape,  \
                                      cudaStream_t st, int sm_count, int64_t* launches);
GMP_DECLARE_LAUNCHER(0)
GMP_DECLARE_LAUNCHER(1)
GMP_DECLARE_LAUNCHER(2)
GMP_DECLARE_LAUNCHER(3)
GMP_DECLARE_LAUNCHER(4)
GMP_DECLARE_LAUNCHER(5)
GMP_DECLARE_LAUNCHER(6)
