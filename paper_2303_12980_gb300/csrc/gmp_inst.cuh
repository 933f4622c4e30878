// Launchers for one highest order L (included by gmp_inst_L<L>.cu so the
// seven orders compile in parallel).
#pragma once

#include "gmp_kernels.cuh"
#include "gmp_launch.h"

namespace gmpk {

template <int L, int NS>
size_t smem_bytes(const GmpPass& P, int warps) {
  return sizeof(float) * (table_floats(P.n_el, NS, P.kmax) + (size_t)warps * Shape<L, NS>::WARP_FLOATS);
}

template <int L, int NS>
cudaError_t launch(int kind, const KParams& K, cudaStream_t st, int sm_count, int64_t* launches) {
  void (*fn)(KParams) = kind == GMP_KIND_FORWARD    ? k_forward<L, NS>
                        : kind == GMP_KIND_VJP      ? k_vjp<L, NS>
                        : kind == GMP_KIND_BACKWARD ? k_backward<L, NS>
                                                    : k_jacobian<L, NS>;
  // as many warps per CTA as the kernel allows (launch bounds) and 227 KB of
  // shared memory fit
  cudaFuncAttributes fa;
  cudaError_t ea = cudaFuncGetAttributes(&fa, fn);
  if (ea != cudaSuccess) return ea;
  int warps = fa.maxThreadsPerBlock / 32;
  if (warps > 16) warps = 16;
  while (warps > 1 && smem_bytes<L, NS>(K.pass, warps) > 227 * 1024) --warps;
  const size_t smem = smem_bytes<L, NS>(K.pass, warps);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t blocks = (int64_t)sm_count * per_sm;
  const int64_t need = (K.N + warps - 1) / warps;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  e = cudaMemsetAsync(K.counter, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)blocks, warps * 32, smem, st>>>(K);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace gmpk

#define GMP_DEFINE_LAUNCHER(LV)                                                                 \
  cudaError_t gmp_launch_compute_L##LV(int kind, int ns, const gmpk::KParams& K, cudaStream_t st, \
                                      int sm_count, int64_t* launches) {                       \
    switch (ns) {                                                                               \
      case 4: return gmpk::launch<LV, 4>(kind, K, st, sm_count, launches);                      \
      case 8: return gmpk::launch<LV, 8>(kind, K, st, sm_count, launches);                      \
      case 16: return gmpk::launch<LV, 16>(kind, K, st, sm_count, launches);                    \
      default: return cudaErrorInvalidValue;                                                    \
    }                                                                                           \
  }
