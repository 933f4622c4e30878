// Launchers for one highest order L (included by gmp_inst_L<L>.cu so the
// seven orders compile in parallel).
#pragma once

#include "gmp_kernels.cuh"
#include "gmp_launch.h"

namespace gmpk {

// The work counter of a launch over centers center0 .. N-1.
static __global__ void k_counter_start(int32_t* counter, int32_t v) { *counter = v; }

template <int L, int NS, int TILE>
size_t smem_bytes(const GmpPass& P, int warps, int extra_per_warp, bool pad = true) {
  return sizeof(float) * (table_floats(P.n_el, L, NS, P.kmax, pad) +
                          (size_t)warps * (Shape<L, NS, TILE>::WARP_FLOATS + extra_per_warp));
}

// shape.tile: 16 or 32 pairs per forward tile; shape.warps: warps per CTA
// (0 = as many as the launch bounds and 227 KB of shared memory allow).
template <int L, int NS>
cudaError_t launch(int kind, const KParams& K, GmpShape shape, cudaStream_t st, int sm_count,
                   int64_t* launches) {
  const int tile = (kind == GMP_KIND_FORWARD && shape.tile == 32) ? 32 : 16;
  void (*fn)(KParams) = kind == GMP_KIND_FORWARD    ? (tile == 32 ? k_forward<L, NS, 32> : k_forward<L, NS, 16>)
                        : kind == GMP_KIND_VJP      ? k_vjp<L, NS>
                        : kind == GMP_KIND_BACKWARD
                            ? (K.pass.mixed_sign ? k_backward<L, NS, false, true> : k_backward<L, NS, false, false>)
                        : kind == GMP_KIND_BACKWARD_VIRIAL
                            ? (K.pass.mixed_sign ? k_backward<L, NS, true, true> : k_backward<L, NS, true, false>)
                            : k_jacobian<L, NS>;
  const int extra = kind == GMP_KIND_BACKWARD_VIRIAL ? virial_extra_floats<L, NS>() : 0;
  auto smem_of = [&](int w) {
    const bool pad = kind != GMP_KIND_BACKWARD && kind != GMP_KIND_JACOBIAN;  // these two: unpadded table
    return tile == 32 ? smem_bytes<L, NS, 32>(K.pass, w, 0) : smem_bytes<L, NS, 16>(K.pass, w, extra, pad);
  };
  cudaFuncAttributes fa;
  cudaError_t ea = cudaFuncGetAttributes(&fa, fn);
  if (ea != cudaSuccess) return ea;
  int warps = fa.maxThreadsPerBlock / 32;
  if (warps > 16) warps = 16;
  if (shape.warps > 0 && shape.warps < warps) warps = shape.warps;
  while (warps > 1 && smem_of(warps) > 227 * 1024) --warps;
  cudaError_t e = cudaSuccess;
  if (kind == GMP_KIND_JACOBIAN && shape.warps <= 0) {
    // untuned Jacobian launch: the CTA size with the most resident warps
    // (at order 6 the kernel takes 165 registers: one 8-warp CTA per SM,
    // or three 4-warp CTAs)
    int best_w = warps, best_res = 0;
    for (int w = warps; w >= 1; w >>= 1) {
      if (smem_of(w) > 227 * 1024) continue;
      e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_of(w));
      if (e != cudaSuccess) return e;
      int ps = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, fn, w * 32, smem_of(w));
      if (e != cudaSuccess) return e;
      if (ps * w > best_res) { best_res = ps * w; best_w = w; }
    }
    warps = best_w;
  }
  const size_t smem = smem_of(warps);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t blocks = (int64_t)sm_count * per_sm;
  const int64_t need = (K.N - K.center0 + warps - 1) / warps;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  if (K.center0 == 0) {
    e = cudaMemsetAsync(K.counter, 0, sizeof(int32_t), st);
  } else {
    k_counter_start<<<1, 1, 0, st>>>(K.counter, (int32_t)K.center0);
    ++*launches;
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)blocks, warps * 32, smem, st>>>(K);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace gmpk

#define GMP_DEFINE_LAUNCHER(LV)                                                                      \
  cudaError_t gmp_launch_compute_L##LV(int kind, int ns, const gmpk::KParams& K, GmpShape shape,      \
                                      cudaStream_t st, int sm_count, int64_t* launches) {             \
    switch (ns) {                                                                                    \
      case 4: return gmpk::launch<LV, 4>(kind, K, shape, st, sm_count, launches);                    \
      case 8: return gmpk::launch<LV, 8>(kind, K, shape, st, sm_count, launches);                    \
      case 16: return gmpk::launch<LV, 16>(kind, K, shape, st, sm_count, launches);                  \
      default: return cudaErrorInvalidValue;                                                         \
    }                                                                                                \
  }
