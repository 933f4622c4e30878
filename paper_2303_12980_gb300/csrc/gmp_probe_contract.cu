// Measured evaluation of a tensor-core recast of the moment contraction
// (the forward kernel's phase 2): per center and 16-pair tile,
//   mu[s][c] += sum_p R_{l(c)}[p][s] S[p][c]
// for 16 sigmas s and the 64 component slots c of orders 0..6 (16 chunks
// of 4 slots, chunk_l(chunk) = order), on shared-memory tiles laid out as
// the forward kernel lays them out (R [pair][order][sigma], S [pair][slot]).
// The versions run on the same tiles:
//   fp32   the forward kernel's scheme: lane = (4 sigmas) x (one chunk),
//          packed FP32-pair FMAs over the tile's 16 pairs, the partial
//          folded into a (hi, lo) pair by TwoSum;
//   tf32x3 mma.sync m16n8k8 with TF32 operands (rows = the 16 sigmas,
//          k = pairs, n = 8 slots: two chunks of one order), each operand
//          split as hi + lo (hi = TF32 rounding, lo = TF32 rounding of the
//          rest) and multiplied as hi*hi + hi*lo + lo*hi (three MMAs per
//          product tile), the FP32 accumulators folded by TwoSum per tile;
//          at two register budgets, and on tiles stored pre-split.
// The 5th-generation MMA (tcgen05) needs M = 64 or 128 rows per CTA; a
// center has 16 (its sigmas) and centers share no pairs, so it would have
// to run block-diagonal products of 4 to 8 centers (75-88% zero work); the
// warp-level m16n8k8 shape is the one that fits a center.
// Only for the throughput/accuracy probe below: the library's kernels do
// not call this.
#include "gmp.h"
#include "gmp_internal.cuh"
#include "gmp_kernels.cuh"

#include <cmath>
#include <cstdint>
#include <vector>

namespace {

using PSH = gmpk::Shape<6, 16, 16>;
constexpr int kNS = 16;
constexpr int kTiles = 3;        // distinct tiles in shared memory, cycled
constexpr int kWarps = 16;       // warps per CTA (the forward kernel's 16 per SM)
constexpr int kRTile = 16 * PSH::RSTR;
constexpr int kSTile = 16 * PSH::SSTR;
constexpr int kNTiles = 10;      // n-tiles of 8 slots: orders 0..6 have 1,1,2,2,3,3,4 chunks

// n-tile j: order, first chunk, second chunk (-1: none, slots 4..7 are zero)
__host__ __device__ constexpr int ntile_l(int j) {
  int t = 0;
  for (int l = 0; l <= 6; ++l) {
    const int n = (gmpk::chunks_of_order(l) + 1) / 2;
    if (j < t + n) return l;
    t += n;
  }
  return -1;
}
__host__ __device__ constexpr int ntile_c0(int j) {
  int t = 0, cs = 0;
  for (int l = 0; l <= 6; ++l) {
    const int nch = gmpk::chunks_of_order(l), n = (nch + 1) / 2;
    if (j < t + n) return cs + 2 * (j - t);
    t += n;
    cs += nch;
  }
  return -1;
}
__host__ __device__ constexpr int ntile_c1(int j) {
  int t = 0, cs = 0;
  for (int l = 0; l <= 6; ++l) {
    const int nch = gmpk::chunks_of_order(l), n = (nch + 1) / 2;
    if (j < t + n) return 2 * (j - t) + 1 < nch ? cs + 2 * (j - t) + 1 : -1;
    t += n;
    cs += nch;
  }
  return -1;
}
static_assert(ntile_l(kNTiles - 1) == 6 && ntile_l(kNTiles) == -1, "n-tile count of orders 0..6");

__device__ __forceinline__ uint32_t tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_round(x);
  lo = tf32_round(__fsub_rn(x, __uint_as_float(hi)));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void two_sum_into(float& hi, float& lo, float x) {
  const gmp_f2 s = gmp_two_sum(hi, x);
  hi = s.hi;
  lo = __fadd_rn(lo, s.lo);
}

// Tiles: R [kTiles][16 pairs][RSTR], S [kTiles][16 pairs][SSTR] from global.
__device__ __forceinline__ void load_probe_tiles(const float* __restrict__ Rg, const float* __restrict__ Sg,
                                                 float* Rs, float* Ss) {
  for (int t = threadIdx.x; t < kTiles * kRTile; t += blockDim.x) Rs[t] = Rg[t];
  for (int t = threadIdx.x; t < kTiles * kSTile; t += blockDim.x) Ss[t] = Sg[t];
}

// out [warps][16][64]: each warp's sums (hi + lo), slot order of S.
__global__ void __launch_bounds__(kWarps * 32) k_contract_fp32(const float* __restrict__ Rg,
                                                               const float* __restrict__ Sg, int reps,
                                                               float* __restrict__ out) {
  __shared__ __align__(16) float Rs[kTiles * kRTile];
  __shared__ __align__(16) float Ss[kTiles * kSTile];
  load_probe_tiles(Rg, Sg, Rs, Ss);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  float hi[PSH::Q][16], lo[PSH::Q][16];
  int it_sb[PSH::Q], it_ch[PSH::Q], it_l[PSH::Q];
#pragma unroll
  for (int q = 0; q < PSH::Q; ++q) {
    const int item = lane + 32 * q;  // NITEM = 64: every item valid
    it_sb[q] = item % PSH::NSB;
    it_ch[q] = item / PSH::NSB;
    it_l[q] = gmpk::chunk_l(it_ch[q]);
#pragma unroll
    for (int v = 0; v < 16; ++v) hi[q][v] = lo[q][v] = 0.0f;
  }
  for (int rep = 0; rep < reps; ++rep) {
    for (int tile = 0; tile < kTiles; ++tile) {
      const float* Rt = Rs + tile * kRTile;
      const float* St = Ss + tile * kSTile;
#pragma unroll
      for (int q = 0; q < PSH::Q; ++q) {
        const float* rp = Rt + it_l[q] * kNS + 4 * it_sb[q];
        const float* sp = St + 4 * it_ch[q];
        float2 acc2[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) acc2[v] = make_float2(0.0f, 0.0f);
#pragma unroll 4
        for (int pp = 0; pp < 16; ++pp) {
          const float4 r = *reinterpret_cast<const float4*>(rp + pp * PSH::RSTR);
          const float4 s = *reinterpret_cast<const float4*>(sp + pp * PSH::SSTR);
          const float rv[4] = {r.x, r.y, r.z, r.w};
          const float2 s01 = make_float2(s.x, s.y), s23 = make_float2(s.z, s.w);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 ru = make_float2(rv[u], rv[u]);
            acc2[2 * u] = gmp_fma2(ru, s01, acc2[2 * u]);
            acc2[2 * u + 1] = gmp_fma2(ru, s23, acc2[2 * u + 1]);
          }
        }
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          float2 l2 = make_float2(lo[q][2 * v], lo[q][2 * v + 1]);
          const float2 sm = gmp_two_sum2(make_float2(hi[q][2 * v], hi[q][2 * v + 1]), acc2[v], l2);
          hi[q][2 * v] = sm.x;
          hi[q][2 * v + 1] = sm.y;
          lo[q][2 * v] = l2.x;
          lo[q][2 * v + 1] = l2.y;
        }
      }
    }
  }
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  float* o = out + (int64_t)warp * kNS * 64;
#pragma unroll
  for (int q = 0; q < PSH::Q; ++q)
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v)
        o[(4 * it_sb[q] + u) * 64 + 4 * it_ch[q] + v] = __fadd_rn(hi[q][4 * u + v], lo[q][4 * u + v]);
}

// WARPS per CTA sets the register budget: 16 (one CTA per SM, 128
// registers, the forward kernel's occupancy) or 8 (up to 255 registers).
// PRESPLIT: the tiles are stored already split (TF32 hi and lo words, as a
// producer could write them), which leaves the loop only the fragment loads
// and the MMAs -- the best case for the tensor cores, at twice the shared
// memory.  Dynamic shared memory: [R | S] floats, or [Rh | Rl | Sh | Sl].
template <int WARPS, bool PRESPLIT>
__global__ void __launch_bounds__(WARPS * 32) k_contract_tf32x3(const float* __restrict__ Rg,
                                                                const float* __restrict__ Sg, int reps,
                                                                float* __restrict__ out) {
  extern __shared__ __align__(16) uint32_t sm_tf[];
  constexpr int NR = kTiles * kRTile, NSL = kTiles * kSTile;
  uint32_t* Rh = sm_tf;
  uint32_t* Rl = sm_tf + NR;
  uint32_t* Sh = PRESPLIT ? sm_tf + 2 * NR : sm_tf + NR;
  uint32_t* Sl = Sh + NSL;
  if constexpr (PRESPLIT) {
    for (int t = threadIdx.x; t < NR; t += blockDim.x) tf32_split(Rg[t], Rh[t], Rl[t]);
    for (int t = threadIdx.x; t < NSL; t += blockDim.x) tf32_split(Sg[t], Sh[t], Sl[t]);
  } else {
    load_probe_tiles(Rg, Sg, reinterpret_cast<float*>(Rh), reinterpret_cast<float*>(Sh));
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  auto split_at = [&](const uint32_t* H, const uint32_t* Lw, int idx, uint32_t& h, uint32_t& l) {
    if constexpr (PRESPLIT) {
      h = H[idx];
      l = Lw[idx];
    } else {
      tf32_split(__uint_as_float(H[idx]), h, l);
    }
  };
  float hi[kNTiles][4], lo[kNTiles][4];
#pragma unroll
  for (int j = 0; j < kNTiles; ++j)
#pragma unroll
    for (int v = 0; v < 4; ++v) hi[j][v] = lo[j][v] = 0.0f;
  for (int rep = 0; rep < reps; ++rep) {
    for (int tile = 0; tile < kTiles; ++tile) {
      const int rb = tile * kRTile, sb = tile * kSTile;
      float acc[kNTiles][4];
#pragma unroll
      for (int j = 0; j < kNTiles; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[j][v] = 0.0f;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const int p0 = 8 * kk + t, p1 = p0 + 4;
        gmpk::static_for<7>([&](auto ll) {
          constexpr int l = decltype(ll)::value;
          // A (16 sigmas x 8 pairs): a0 = (g, p0), a1 = (g+8, p0), a2 = (g, p1), a3 = (g+8, p1)
          uint32_t ah[4], al[4];
          split_at(Rh, Rl, rb + p0 * PSH::RSTR + l * kNS + g, ah[0], al[0]);
          split_at(Rh, Rl, rb + p0 * PSH::RSTR + l * kNS + g + 8, ah[1], al[1]);
          split_at(Rh, Rl, rb + p1 * PSH::RSTR + l * kNS + g, ah[2], al[2]);
          split_at(Rh, Rl, rb + p1 * PSH::RSTR + l * kNS + g + 8, ah[3], al[3]);
          gmpk::static_for<kNTiles>([&](auto jj) {
            constexpr int j = decltype(jj)::value;
            if constexpr (ntile_l(j) == l) {
              constexpr int c0 = ntile_c0(j), c1 = ntile_c1(j);
              // B (8 pairs x 8 slots): b0 = (p0, n = g), b1 = (p1, n = g)
              const bool ok = g < 4 || c1 >= 0;
              const int col = g < 4 ? 4 * c0 + g : 4 * (c1 >= 0 ? c1 : 0) + g - 4;
              uint32_t bh0, bl0, bh1, bl1;
              split_at(Sh, Sl, sb + p0 * PSH::SSTR + col, bh0, bl0);
              split_at(Sh, Sl, sb + p1 * PSH::SSTR + col, bh1, bl1);
              if (!ok) bh0 = bl0 = bh1 = bl1 = 0u;
              mma_tf32(acc[j], ah, bh0, bh1);
              mma_tf32(acc[j], ah, bl0, bl1);
              mma_tf32(acc[j], al, bh0, bh1);
            }
          });
        });
      }
#pragma unroll
      for (int j = 0; j < kNTiles; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) two_sum_into(hi[j][v], lo[j][v], acc[j][v]);
    }
  }
  // D fragment: d0 = (g, 2t), d1 = (g, 2t+1), d2 = (g+8, 2t), d3 = (g+8, 2t+1)
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  float* o = out + (int64_t)warp * kNS * 64;
  gmpk::static_for<kNTiles>([&](auto jj) {
    constexpr int j = decltype(jj)::value;
    constexpr int c0 = ntile_c0(j), c1 = ntile_c1(j);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int n = 2 * t + (v & 1), s = g + (v >> 1) * 8;
      if (n >= 4 && c1 < 0) continue;
      const int col = n < 4 ? 4 * c0 + n : 4 * c1 + n - 4;
      o[s * 64 + col] = __fadd_rn(hi[j][v], lo[j][v]);
    }
  });
}

}  // namespace

extern "C" gmp_status gmp_probe_contraction(int device, double* result, int32_t n_result) {
  if (!result || n_result < GMP_PROBE_CONTRACT_N) return GMP_ERR_INVALID_ARG;
  for (int k = 0; k < GMP_PROBE_CONTRACT_N; ++k) result[k] = 0.0;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return GMP_ERR_CUDA;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    return GMP_ERR_CUDA;
  }
  // seeded tiles (a 64-bit LCG): R > 0 as for non-negative densities, S of
  // either sign; slots of an order's last chunk past its 2l+1 components
  // hold values too (the forward kernel keeps r^l there)
  std::vector<float> R((size_t)kTiles * kRTile, 0.0f), S((size_t)kTiles * kSTile, 0.0f);
  uint64_t st = 0x9E3779B97F4A7C15ull;
  auto uni = [&st]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(st >> 11) * (1.0 / 9007199254740992.0);
  };
  for (int tile = 0; tile < kTiles; ++tile)
    for (int p = 0; p < 16; ++p) {
      for (int l = 0; l <= 6; ++l)
        for (int s = 0; s < kNS; ++s) R[(size_t)tile * kRTile + p * PSH::RSTR + l * kNS + s] = (float)uni();
      for (int c = 0; c < 64; ++c) S[(size_t)tile * kSTile + p * PSH::SSTR + c] = (float)(2.0 * uni() - 1.0);
    }
  const int reps_check = 3;  // 3 x 3 tiles = 144 pairs, about one slab center
  // FP64 sums and their cancellation-free scales for the check
  std::vector<double> ref((size_t)kNS * 64, 0.0), scale((size_t)kNS * 64, 0.0);
  for (int rep = 0; rep < reps_check; ++rep)
    for (int tile = 0; tile < kTiles; ++tile)
      for (int p = 0; p < 16; ++p)
        for (int s = 0; s < kNS; ++s)
          for (int c = 0; c < 64; ++c) {
            const double r = R[(size_t)tile * kRTile + p * PSH::RSTR + gmpk::chunk_l(c / 4) * kNS + s];
            const double x = r * (double)S[(size_t)tile * kSTile + p * PSH::SSTR + c];
            ref[s * 64 + c] += x;
            scale[s * 64 + c] += std::fabs(x);
          }
  const int blocks = prop.multiProcessorCount;  // one CTA per SM
  const int64_t max_warps = (int64_t)blocks * kWarps;
  float *dR = nullptr, *dS = nullptr, *dout = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  gmp_status res = GMP_OK;
  std::vector<float> h((size_t)kNS * 64);
  auto fail = [&](cudaError_t e) {
    if (e != cudaSuccess && res == GMP_OK) {
      cudaGetLastError();
      res = e == cudaErrorMemoryAllocation ? GMP_ERR_OOM : GMP_ERR_CUDA;
    }
    return res != GMP_OK;
  };
  if (fail(cudaMalloc(&dR, R.size() * sizeof(float))) || fail(cudaMalloc(&dS, S.size() * sizeof(float))) ||
      fail(cudaMalloc(&dout, (size_t)max_warps * kNS * 64 * sizeof(float))) ||
      fail(cudaMemcpy(dR, R.data(), R.size() * sizeof(float), cudaMemcpyHostToDevice)) ||
      fail(cudaMemcpy(dS, S.data(), S.size() * sizeof(float), cudaMemcpyHostToDevice)) ||
      fail(cudaEventCreate(&e0)) || fail(cudaEventCreate(&e1))) {
  } else {
    // versions: FP32 (16 warps per SM), TF32x3 (16 warps), TF32x3 (8
    // warps), TF32x3 on pre-split tiles (16 warps)
    constexpr int NV = 4;
    void (*const kern[NV])(const float*, const float*, int, float*) = {
        k_contract_fp32, k_contract_tf32x3<16, false>, k_contract_tf32x3<8, false>, k_contract_tf32x3<16, true>};
    const int warps[NV] = {kWarps, 16, 8, 16};
    const size_t tile_bytes = sizeof(float) * (size_t)kTiles * (kRTile + kSTile);
    const size_t smem[NV] = {0, tile_bytes, tile_bytes, 2 * tile_bytes};
    const int reps_time = 2000;
    for (int v = 0; v < NV && res == GMP_OK; ++v) {
      if (smem[v] > 48 * 1024 &&
          fail(cudaFuncSetAttribute(kern[v], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem[v])))
        break;
      cudaFuncAttributes fa;
      if (fail(cudaFuncGetAttributes(&fa, kern[v]))) break;
      result[2 * NV + v] = fa.numRegs;
      // accuracy: warp 0's sums over reps_check x kTiles tiles
      kern[v]<<<blocks, warps[v] * 32, smem[v]>>>(dR, dS, reps_check, dout);
      if (fail(cudaGetLastError()) || fail(cudaMemcpy(h.data(), dout, h.size() * sizeof(float),
                                                      cudaMemcpyDeviceToHost)))
        break;
      double worst = 0.0;
      for (size_t k = 0; k < h.size(); ++k)
        worst = std::fmax(worst, std::fabs((double)h[k] - ref[k]) / std::fmax(scale[k], 1e-300));
      result[NV + v] = worst;
      // throughput: warm-up, then a timed launch
      kern[v]<<<blocks, warps[v] * 32, smem[v]>>>(dR, dS, 50, dout);
      if (fail(cudaEventRecord(e0))) break;
      kern[v]<<<blocks, warps[v] * 32, smem[v]>>>(dR, dS, reps_time, dout);
      if (fail(cudaEventRecord(e1)) || fail(cudaEventSynchronize(e1))) break;
      float ms = 0.0f;
      if (fail(cudaEventElapsedTime(&ms, e0, e1))) break;
      const double pairs = (double)blocks * warps[v] * reps_time * kTiles * 16;
      result[v] = pairs / (ms * 1e-3) / 1e9;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(dR);
  cudaFree(dS);
  cudaFree(dout);
  return res;
}
