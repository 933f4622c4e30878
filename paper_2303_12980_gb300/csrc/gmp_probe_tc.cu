// Measured evaluation of a 5th-generation tensor-core (tcgen05) recast of
// the backward kernel's per-pair adjoint contraction.  For every neighbor
// pair p of a center, with the center's adjoints Lam[s][k] (16 sigmas s,
// the 49 independent MCSH components k of orders 0..6) and the pair's
// radial factors R[p][s][l] (orders l = 0..7):
//   lam[p][k]  = sum_s Lam[s][k] R[p][s][l(k)]
//   lamd[p][k] = sum_s Lam[s][k] (-beta_s) R[p][s][l(k)+1]     (dR_l/dr^2)
// i.e. per order l a product (pairs x sigmas) . (sigmas x components):
//   D_l[p][0..15]  = sum_s R[p][s][l] B_l[s][0..15],  B_l = Lam of order l,
//   D_l[p][16..31] = ..., B_l = -beta_s Lam of order l-1.
// The versions run on the same seeded data:
//   fp32     the backward kernel's scheme: lane = pair, the adjoint rows read
//            from shared memory as float4 broadcasts, scalar FMAs (1568 per
//            pair), 12 warps per SM;
//   tcgen05  M = 128 pairs per tile (one per TMEM lane), K = 16 sigmas, N =
//            32 columns per order, 8 orders: kind::tf32 MMAs issued by one
//            thread with operands in shared memory (no swizzle, K-major
//            core matrices) and FP32 accumulators in tensor memory, each
//            operand split as hi + lo (hi = TF32 rounding, lo = TF32
//            rounding of the rest; hi*hi + lo*hi + hi*lo: 48 MMAs per tile);
//            the threads write the radial factors into the A tiles, wait on
//            an mbarrier for the MMAs and read their rows back with
//            tcgen05.ld.  Every wait is bounded: a wait that runs out sets a
//            flag in the result and the kernel skips to its end, where it
//            frees its tensor memory.
// Only for the throughput/accuracy probe below: the library's kernels do
// not call this.
#include "gmp.h"
#include "gmp_internal.cuh"

#include <cmath>
#include <cstdint>
#include <vector>

namespace {

constexpr int kNS = 16;          // sigmas (K)
constexpr int kOrders = 8;       // radial orders 0..7 (A tiles)
constexpr int kNInd = 49;        // independent components of orders 0..6
constexpr int kNIndP = 52;       // padded row of adjoints
constexpr int kRows = 128;       // pairs per tile (M)
constexpr int kN = 32;           // columns per order (N)
constexpr int kSrcPairs = 512;   // distinct pairs in the source array (cycled)

__host__ __device__ constexpr int order_of(int k) {
  int l = 0;
  while ((l + 1) * (l + 1) <= k) ++l;
  return l;
}

// Shared-memory operand layout (K-major, no swizzle): for k-step t (K
// elements 8t .. 8t+7) a 4 KB (A: 128 rows) or 1 KB (B: 32 rows) block of
// core matrices [row group of 8][K half of 4][8 rows][4 elements]; LBO (K
// neighbour core matrix) = 128 B, SBO (next 8-row group) = 256 B.
__host__ __device__ constexpr int op_offset(int row, int k, int rows) {
  return (k >> 3) * (rows * 32) + (row >> 3) * 256 + ((k >> 2) & 1) * 128 + (row & 7) * 16 + (k & 3) * 4;
}
constexpr int kABytes = kRows * kNS * 4;          // one order, one split part: 8 KB
constexpr int kBBytes = kN * kNS * 4;             // 2 KB
constexpr int kSmemA = 2 * kOrders * kABytes;     // hi, lo: 128 KB
constexpr int kSmemB = 2 * kOrders * kBBytes;     // 32 KB
constexpr int kSmemTotal = kSmemA + kSmemB + 64;  // + mbarrier, TMEM address

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);           // start address
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;      // leading byte offset (K)
  d |= (uint64_t)((256u >> 4) & 0x3FFFu) << 32;      // stride byte offset (8-row groups)
  d |= (uint64_t)1 << 46;                            // descriptor version (sm_100 family)
  return d;                                          // base offset 0, no swizzle
}

// Instruction descriptor: D F32, A and B TF32, both K-major, N = 32, M = 128.
constexpr uint32_t kIDesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kRows >> 4) << 24);

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIDesc), "r"(accumulate));
}

// Adjoint rows Lam[s][k] and -beta_s, seeded on the host; per-sigma radial
// bases and ratios for the generated radial factors.
struct Src {
  const float* rad;   // [kNS][2]: base b_s, ratio q_s
  const float* Lam;   // [kNS][kNIndP]
  const float* nbeta; // [kNS]
};

// The pair's radial factors, generated in registers as the backward kernel
// has them (there from exponentials; here R[s][l] = b_s (1 + p / 512) q_s^l
// by FP32 products, p the pair's index mod 512), the same on host and device.
__host__ __device__ inline float gen_radial(float b, float q, int p, int l) {
  float r = b * (1.0f + (float)(p & (kSrcPairs - 1)) * (1.0f / 512.0f));
  for (int k = 0; k < l; ++k) r = r * q;
  return r;
}

// ---------------------------------------------------------------- fp32
// lane = pair; lam and lamd of the pair accumulated over the 16 sigmas with
// scalar FMAs, the adjoint rows read as float4 broadcasts; the pair's rows
// are summed into a checksum (and, for the first tile, written out).
__global__ void __launch_bounds__(384) k_bwd_contract_fp32(Src src, int reps, float* out, float* check) {
  __shared__ __align__(16) float s_lam[kNS * kNIndP];
  for (int t = threadIdx.x; t < kNS * kNIndP; t += blockDim.x) s_lam[t] = src.Lam[t];
  __syncthreads();
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  float sum = 0.0f;
  for (int rep = 0; rep < reps; ++rep) {
    const int p = (gtid + rep * 97) % kSrcPairs;
    float lam[kNInd], lamd[kNInd];
#pragma unroll
    for (int k = 0; k < kNInd; ++k) lam[k] = lamd[k] = 0.0f;
#pragma unroll 1
    for (int sg = 0; sg < kNS / 4; ++sg) {
      float R[4][kOrders];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float b = src.rad[2 * (4 * sg + u)], q = src.rad[2 * (4 * sg + u) + 1];
        R[u][0] = b * (1.0f + (float)(p & (kSrcPairs - 1)) * (1.0f / 512.0f));
#pragma unroll
        for (int l = 1; l < kOrders; ++l) R[u][l] = R[u][l - 1] * q;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float nb = src.nbeta[4 * sg + u];
        float Rd[kOrders - 1];
#pragma unroll
        for (int l = 0; l < kOrders - 1; ++l) Rd[l] = __fmul_rn(nb, R[u][l + 1]);
        const float* lrow = s_lam + (4 * sg + u) * kNIndP;
#pragma unroll
        for (int c4 = 0; c4 < kNIndP / 4; ++c4) {
          const float4 lv4 = *reinterpret_cast<const float4*>(lrow + 4 * c4);
          const float lv[4] = {lv4.x, lv4.y, lv4.z, lv4.w};
#pragma unroll
          for (int tt = 0; tt < 4; ++tt) {
            const int k = 4 * c4 + tt;
            if (k < kNInd) {
              lam[k] = __fmaf_rn(lv[tt], R[u][order_of(k)], lam[k]);
              lamd[k] = __fmaf_rn(lv[tt], Rd[order_of(k)], lamd[k]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kNInd; ++k) sum += lam[k] + lamd[k];
    if (rep == 0 && check && gtid < kRows)
#pragma unroll
      for (int k = 0; k < kNInd; ++k) {
        check[gtid * 2 * kNInd + k] = lam[k];
        check[gtid * 2 * kNInd + kNInd + k] = lamd[k];
      }
  }
  out[gtid] = sum;
}

// ---------------------------------------------------------------- tcgen05
// One CTA of 4 warps per SM (thread = pair = TMEM lane); 256 TMEM columns
// (8 orders x 32).
__global__ void __launch_bounds__(128, 1) k_bwd_contract_tc(Src src, int reps, float* out, float* check,
                                                          unsigned* flags) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;                       // [part][order] 8 KB tiles
  unsigned char* sB = smem + kSmemA;              // [part][order] 2 KB tiles
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kSmemA + kSmemB);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kSmemA + kSmemB + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // B tiles: order l: columns 0..15 the adjoints of order l, 16..31 the
  // adjoints of order l-1 times -beta; rows (columns of D) beyond an
  // order's components are zero
  for (int t = tid; t < kOrders * kN * kNS; t += blockDim.x) {
    const int l = t / (kN * kNS), n = (t / kNS) % kN, s = t % kNS;
    float v = 0.0f;
    if (n < 16) {
      const int k = l * l + n;
      if (l <= 6 && n < 2 * l + 1) v = src.Lam[s * kNIndP + k];
    } else {
      const int lm = l - 1, k = lm * lm + (n - 16);
      if (lm >= 0 && n - 16 < 2 * lm + 1) v = src.nbeta[s] * src.Lam[s * kNIndP + k];
    }
    const float hi = tf32_round(v), lo = tf32_round(v - hi);
    *reinterpret_cast<float*>(sB + l * kBBytes + op_offset(n, s, kN)) = hi;
    *reinterpret_cast<float*>(sB + (kOrders + l) * kBBytes + op_offset(n, s, kN)) = lo;
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);  // this warp's lanes
  uint32_t phase = 0;
  bool ok = true;
  float sum = 0.0f;
  for (int rep = 0; rep < reps && ok; ++rep) {
    // A tiles: this pair's radial factors, split hi / lo
    const int p = (blockIdx.x * kRows + tid + rep * 97) % kSrcPairs;
#pragma unroll
    for (int s4 = 0; s4 < kNS / 4; ++s4) {
      float R[4][kOrders];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float b = src.rad[2 * (4 * s4 + u)], q = src.rad[2 * (4 * s4 + u) + 1];
        R[u][0] = b * (1.0f + (float)(p & (kSrcPairs - 1)) * (1.0f / 512.0f));
#pragma unroll
        for (int l = 1; l < kOrders; ++l) R[u][l] = R[u][l - 1] * q;
      }
#pragma unroll
      for (int l = 0; l < kOrders; ++l) {
        const float4 r = make_float4(R[0][l], R[1][l], R[2][l], R[3][l]);
        const float4 h = make_float4(tf32_round(r.x), tf32_round(r.y), tf32_round(r.z), tf32_round(r.w));
        const float4 q = make_float4(tf32_round(r.x - h.x), tf32_round(r.y - h.y), tf32_round(r.z - h.z),
                                     tf32_round(r.w - h.w));
        *reinterpret_cast<float4*>(sA + l * kABytes + op_offset(tid, 4 * s4, kRows)) = h;
        *reinterpret_cast<float4*>(sA + (kOrders + l) * kABytes + op_offset(tid, 4 * s4, kRows)) = q;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int l = 0; l < kOrders; ++l) {
        const uint32_t d = tmem + (uint32_t)(l * kN);
        for (int ks = 0; ks < 2; ++ks) {
          const uint64_t ahi = smem_desc(smem_u32(sA + l * kABytes + ks * (kRows * 32)));
          const uint64_t alo = smem_desc(smem_u32(sA + (kOrders + l) * kABytes + ks * (kRows * 32)));
          const uint64_t bhi = smem_desc(smem_u32(sB + l * kBBytes + ks * (kN * 32)));
          const uint64_t blo = smem_desc(smem_u32(sB + (kOrders + l) * kBBytes + ks * (kN * 32)));
          mma_tf32(d, ahi, bhi, ks > 0 ? 1u : 0u);
          mma_tf32(d, alo, bhi, 1u);
          mma_tf32(d, ahi, blo, 1u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar)));
    }
    // bounded wait for the MMAs of this tile
    uint32_t done = 0;
    for (int it = 0; it < (1 << 22) && !done; ++it)
      asm volatile(
          "{\n\t.reg .pred q;\n\t"
          "mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, q;\n\t}\n"
          : "=r"(done)
          : "r"(smem_u32(mbar)), "r"(phase));
    if (!__all_sync(0xffffffffu, done)) {
      if (lane == 0) atomicOr(flags, 1u);
      ok = false;
    }
    ok = __syncthreads_and(ok);
    if (!ok) break;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // this pair's rows of the 8 orders' results
    for (int l = 0; l < kOrders; ++l) {
      uint32_t r[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr + (uint32_t)(l * kN)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int c = 0; c < kN; ++c) sum += __uint_as_float(r[c]);
      if (rep == 0 && check && blockIdx.x == 0) {
        for (int c = 0; c < 16; ++c)
          if (l <= 6 && c < 2 * l + 1) check[tid * 2 * kNInd + l * l + c] = __uint_as_float(r[c]);
        for (int c = 0; c < 16; ++c)
          if (l >= 1 && c < 2 * (l - 1) + 1) check[tid * 2 * kNInd + kNInd + (l - 1) * (l - 1) + c] = __uint_as_float(r[16 + c]);
      }
    }
    // every lane is done with the accumulators before the next tile's MMAs
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  out[blockIdx.x * kRows + tid] = sum;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
  }
}

}  // namespace

extern "C" gmp_status gmp_probe_backward_contraction(int device, double* result, int32_t n_result) {
  if (!result || n_result < GMP_PROBE_BWD_CONTRACT_N) return GMP_ERR_INVALID_ARG;
  for (int k = 0; k < GMP_PROBE_BWD_CONTRACT_N; ++k) result[k] = 0.0;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return GMP_ERR_CUDA;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    return GMP_ERR_CUDA;
  }
  // seeded data (64-bit LCG): radial factors > 0, adjoints of either sign,
  // -beta of the slab's sigmas (0.05 .. 1.5 A, log-spaced)
  std::vector<float> rad(2 * kNS), Lam((size_t)kNS * kNIndP, 0.0f), nb(kNS);
  uint64_t st = 0x2545F4914F6CDD1Dull;
  auto uni = [&st]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(st >> 11) * (1.0 / 9007199254740992.0);
  };
  for (int s = 0; s < kNS; ++s) {
    rad[2 * s] = (float)(0.5 + uni());
    rad[2 * s + 1] = (float)(0.3 + 0.6 * uni());
  }
  for (int s = 0; s < kNS; ++s)
    for (int k = 0; k < kNInd; ++k) Lam[s * kNIndP + k] = (float)(2.0 * uni() - 1.0);
  for (int s = 0; s < kNS; ++s) {
    const double sig = 0.05 * std::pow(30.0, s / 15.0);
    nb[s] = (float)(-1.0 / (2.0 * sig * sig));
  }
  // FP64 results of the first tile's 128 pairs and their cancellation-free scales
  std::vector<double> ref((size_t)kRows * 2 * kNInd, 0.0), scale((size_t)kRows * 2 * kNInd, 0.0);
  // (pair p of the first tile: fp32 thread p of CTA 0, tcgen05 row p of CTA 0; both p < 512)
  for (int p = 0; p < kRows; ++p)
    for (int k = 0; k < kNInd; ++k) {
      const int l = order_of(k);
      for (int s = 0; s < kNS; ++s) {
        const double a = (double)Lam[s * kNIndP + k] * gen_radial(rad[2 * s], rad[2 * s + 1], p, l);
        const double b = (double)Lam[s * kNIndP + k] * nb[s] * gen_radial(rad[2 * s], rad[2 * s + 1], p, l + 1);
        ref[p * 2 * kNInd + k] += a;
        scale[p * 2 * kNInd + k] += std::fabs(a);
        ref[p * 2 * kNInd + kNInd + k] += b;
        scale[p * 2 * kNInd + kNInd + k] += std::fabs(b);
      }
    }
  const int sms = prop.multiProcessorCount;
  float *drad = nullptr, *dLam = nullptr, *dnb = nullptr, *dout = nullptr, *dcheck = nullptr;
  unsigned* dflags = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  gmp_status res = GMP_OK;
  auto fail = [&](cudaError_t e) {
    if (e != cudaSuccess && res == GMP_OK) {
      cudaGetLastError();
      res = e == cudaErrorMemoryAllocation ? GMP_ERR_OOM : GMP_ERR_CUDA;
    }
    return res != GMP_OK;
  };
  const int fp32_threads = 384, tc_threads = kRows;
  const size_t n_out = (size_t)sms * fp32_threads;
  std::vector<float> h((size_t)kRows * 2 * kNInd);
  if (fail(cudaMalloc(&drad, rad.size() * 4)) || fail(cudaMalloc(&dLam, Lam.size() * 4)) ||
      fail(cudaMalloc(&dnb, nb.size() * 4)) || fail(cudaMalloc(&dout, n_out * 4)) ||
      fail(cudaMalloc(&dcheck, h.size() * 4)) || fail(cudaMalloc(&dflags, 4)) ||
      fail(cudaMemcpy(drad, rad.data(), rad.size() * 4, cudaMemcpyHostToDevice)) ||
      fail(cudaMemcpy(dLam, Lam.data(), Lam.size() * 4, cudaMemcpyHostToDevice)) ||
      fail(cudaMemcpy(dnb, nb.data(), nb.size() * 4, cudaMemcpyHostToDevice)) ||
      fail(cudaMemset(dflags, 0, 4)) || fail(cudaEventCreate(&e0)) || fail(cudaEventCreate(&e1))) {
  } else {
    const Src src{drad, dLam, dnb};
    auto check_err = [&](double* lam_err, double* lamd_err) {
      if (fail(cudaMemcpy(h.data(), dcheck, h.size() * 4, cudaMemcpyDeviceToHost))) return;
      double a = 0.0, b = 0.0;
      for (int p = 0; p < kRows; ++p)
        for (int k = 0; k < kNInd; ++k) {
          const size_t i = (size_t)p * 2 * kNInd + k, j = i + kNInd;
          a = std::fmax(a, std::fabs(h[i] - ref[i]) / std::fmax(scale[i], 1e-300));
          b = std::fmax(b, std::fabs(h[j] - ref[j]) / std::fmax(scale[j], 1e-300));
        }
      *lam_err = a;
      *lamd_err = b;
    };
    cudaFuncAttributes fa;
    // fp32 scheme
    if (!fail(cudaFuncGetAttributes(&fa, k_bwd_contract_fp32))) {
      result[6] = fa.numRegs;
      if (!fail(cudaMemset(dcheck, 0, h.size() * 4))) {
        k_bwd_contract_fp32<<<sms, fp32_threads>>>(src, 1, dout, dcheck);
        if (!fail(cudaGetLastError())) check_err(&result[2], &result[3]);
      }
      const int reps = 400;
      k_bwd_contract_fp32<<<sms, fp32_threads>>>(src, 20, dout, nullptr);
      if (!fail(cudaEventRecord(e0))) {
        k_bwd_contract_fp32<<<sms, fp32_threads>>>(src, reps, dout, nullptr);
        float ms = 0.0f;
        if (!fail(cudaEventRecord(e1)) && !fail(cudaEventSynchronize(e1)) && !fail(cudaEventElapsedTime(&ms, e0, e1)))
          result[0] = (double)sms * fp32_threads * reps / (ms * 1e-3) / 1e9;
      }
    }
    // tcgen05 scheme
    if (res == GMP_OK && !fail(cudaFuncSetAttribute(k_bwd_contract_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    kSmemTotal)) &&
        !fail(cudaFuncGetAttributes(&fa, k_bwd_contract_tc))) {
      result[7] = fa.numRegs;
      if (!fail(cudaMemset(dcheck, 0, h.size() * 4))) {
        k_bwd_contract_tc<<<sms, tc_threads, kSmemTotal>>>(src, 1, dout, dcheck, dflags);
        if (!fail(cudaGetLastError())) check_err(&result[4], &result[5]);
      }
      const int reps = 400;
      k_bwd_contract_tc<<<sms, tc_threads, kSmemTotal>>>(src, 20, dout, nullptr, dflags);
      if (!fail(cudaEventRecord(e0))) {
        k_bwd_contract_tc<<<sms, tc_threads, kSmemTotal>>>(src, reps, dout, nullptr, dflags);
        float ms = 0.0f;
        if (!fail(cudaEventRecord(e1)) && !fail(cudaEventSynchronize(e1)) && !fail(cudaEventElapsedTime(&ms, e0, e1)))
          result[1] = (double)sms * kRows * reps / (ms * 1e-3) / 1e9;
      }
      unsigned fl = 0;
      if (!fail(cudaMemcpy(&fl, dflags, 4, cudaMemcpyDeviceToHost))) result[8] = fl;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(drad);
  cudaFree(dLam);
  cudaFree(dnb);
  cudaFree(dout);
  cudaFree(dcheck);
  cudaFree(dflags);
  return res;
}
