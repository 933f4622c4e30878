// Double-float recomputation of features that FP32 cannot resolve.
//
// A feature f_{l,s} = sum_c w_c mu_c^2 whose value is tiny compared with the
// cancellation-free scale of its moments (near-symmetric environments make
// l >= 1 moments cancel) loses relative accuracy in FP32 in proportion to
// sqrt(scale / f).  The forward kernels queue such (center, order, sigma)
// entries; this kernel recomputes each of them in double-float arithmetic
// (pairs of FP32 words, about 2^-44 relative per operation), which FP32
// hardware runs far faster than FP64: the displacement from the
// double-float split of the positions (the atoms, or the reference points of
// gmp_featurize_points), the radial factor with a double-float exponential,
// the MCSH components by the same recurrences, and the invariant.  When a
// derivative kernel follows, the recomputed moments also replace the FP32
// moments it reads: the adjoints of a cancelling moment group would
// otherwise carry its FP32 rounding, which is relative to the group's
// cancellation-free scale rather than to the moments themselves.
#include "gmp_internal.cuh"
#include "mcsh_gen.cuh"


namespace {

// Sigmas recomputed together: the displacement and the MCSH components of a
// pair serve all of them, the radial factor is per sigma.  Only orders 4
// and 5 take pairs of sigmas.  Below order 4 the components are cheap and
// a group only takes parallelism from the few flagged features of a
// typical batch (random alloy slab: refinement 0.30 ms with single sigmas,
// 0.40 ms with groups of 4); at order 6 a second sigma's accumulators do
// not fit the kernel's 128 registers (two 256-thread CTAs per SM; at 168
// registers it ran at half the resident warps and slower, grouping or
// not).  Perfect FCC crystal (orders 4 and 6 flagged at the widest
// sigmas): 24.9 ms single, 21.5 ms with pairs at orders 4-5.
template <int L>
constexpr int refine_group() { return (L == 4 || L == 5) ? 2 : 1; }

// Moments of order L (2L+1 independent components) of one center for the
// ng <= G sigmas sig[0 .. ng-1] over its pairs, lane-strided, in
// double-float arithmetic.
template <int L, int G>
__device__ __forceinline__ void refine_moments(int lane, const float4& xhi, const float4& xli,
                                               const GmpStruct& st, const int64_t p0, const int64_t p1,
                                               const GmpPair* __restrict__ pairs,
                                               const float4* __restrict__ atom_xh, const float4* __restrict__ atom_xl,
                                               const float* __restrict__ ktab, int nsig_total, const int (&sig)[G],
                                               int ng, int kmax, const float2* __restrict__ exp_tab,
                                               gmp_f2 (&mu)[G][2 * L + 1]) {
  for (int64_t p = p0 + lane; p < p1; p += 32) {
    const GmpPair pr = pairs[p];
    int nn[3];
    gmp_unpack_shift(pr.shift, nn);
    gmp_f2 d[3], r2;
    float mag;
    gmp_df_disp(xhi, xli, atom_xh[pr.j], atom_xl[pr.j], st, nn, d, r2, mag);
    gmp_f2 Sd[(L + 1) * (L + 1)];
    gmp_mcsh_indep_df(L, d[0], d[1], d[2], r2, Sd);
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if (g >= ng) break;
      // radial factor: sum_q A_{q,L} exp(-b_q r^2); table entry (b, A_0 .. A_6) as double-floats
      gmp_f2 R{0.0f, 0.0f};
      const float* te = ktab + ((size_t)pr.e * nsig_total + sig[g]) * kmax * 16;  // [element][sigma][primitive]
      for (int q = 0; q < kmax; ++q) {
        const float* ent = te + q * 16;
        const gmp_f2 E = gmp_df_exp_neg(gmp_df_mul(gmp_f2{ent[0], ent[1]}, r2), exp_tab);
        R = gmp_df_add(R, gmp_df_mul(gmp_f2{ent[2 + 2 * L], ent[3 + 2 * L]}, E));
      }
#pragma unroll
      for (int k = 0; k <= 2 * L; ++k) mu[g][k] = gmp_df_add(mu[g][k], gmp_df_mul(R, Sd[L * L + k]));
    }
  }
}

// The flagged features of order LO of one task: center i, the order's
// first column c0 (col_info[c0] = (order << 16) | global sigma of that
// column) and a mask of flagged sigmas, recomputed by the whole warp G
// sigmas at a time (entries of other orders are left to that order's
// launch).  Moments over the center's pairs (lane-strided), warp-reduced,
// and the invariant, all double-float; the feature is rounded to FP32.  With
// mu_out, the 2L+1 moments of a sigma of the pass rounded to FP32 overwrite
// its FP32 moments.
template <int LO>
__device__ __forceinline__ void refine_entry(int lane, const GmpRefine& A, int64_t i, int c0, unsigned mask) {
  constexpr int G = refine_group<LO>();
  const int info = c0 < A.F ? A.col_info[c0] : -1;
  if (info < 0 || (info >> 16) != LO) return;
  const int sig0 = info & 0xffff;
  const GmpStruct& st = A.structs[A.center_struct[i]];
  const float4 xhi = A.center_xh[i], xli = A.center_xl[i];
  const int64_t p0 = A.nbr_beg[i], p1 = A.nbr_end[i];
  while (mask) {  // warp-uniform
    int sig[G], col[G], ng = 0;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      sig[g] = sig0;
      col[g] = c0;
      if (mask) {
        const int b = __ffs(mask) - 1;
        mask &= mask - 1;
        sig[g] = sig0 + b;
        col[g] = c0 + b;
        ng = g + 1;
      }
    }
    gmp_f2 mu[G][2 * LO + 1];
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
      for (int k = 0; k <= 2 * LO; ++k) mu[g][k] = gmp_f2{0.0f, 0.0f};
    refine_moments<LO, G>(lane, xhi, xli, st, p0, p1, A.pairs, A.atom_xh, A.atom_xl, A.ktab, A.nsig_total, sig, ng,
                          A.kmax, A.exp_tab, mu);
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if (g >= ng) break;
#pragma unroll
      for (int k = 0; k <= 2 * LO; ++k)
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          const gmp_f2 other{__shfl_xor_sync(0xffffffffu, mu[g][k].hi, o),
                             __shfl_xor_sync(0xffffffffu, mu[g][k].lo, o)};
          mu[g][k] = gmp_df_add(mu[g][k], other);
        }
      if (A.mu_out && sig[g] >= A.mu_sig0 && sig[g] < A.mu_sig0 + A.mu_nsig && lane == 0) {
        float* mu_dst = A.mu_out + (i * A.mu_nsig + (sig[g] - A.mu_sig0)) * (int64_t)A.mu_nind + LO * LO;
#pragma unroll
        for (int k = 0; k <= 2 * LO; ++k) mu_dst[k] = mu[g][k].hi + mu[g][k].lo;
      }
      const gmp_f2 f = gmp_mcsh_invariant_df(LO, mu[g]);
      if (lane == 0) A.features[i * A.F + col[g]] = f.hi + f.lo;
    }
  }
}

// Flagged features of order LO (one launch per order, so that every warp of
// a launch runs the same instantiation: the per-order code is large, and
// warps mixing orders thrash the instruction cache).  The order's queue
// entries (center << 32 | first column of the order << 16 | mask of up to
// 16 sigmas) are cut into tasks of one group of G flagged sigmas each,
// numbered group-major (all entries' first groups, then their second
// groups, ...; empty groups cost a load and a count), so that a center with
// many flagged sigmas is spread over as many warps as it has groups instead
// of one warp taking them in turn.
template <int LO>
__global__ void __launch_bounds__(256, 2) k_refine(const GmpRefine A) {
  constexpr int G = refine_group<LO>();
  constexpr int S = (16 + G - 1) / G;
  const int qi = A.qidx[LO];
  if (qi < 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned long long n = A.count[qi];
  const int64_t nq = n < (unsigned long long)A.cap ? (int64_t)n : A.cap;
  const unsigned long long* queue = A.queue + qi * A.cap;
  // task v = g * nq + t: group g of entry t, so that the groups of one
  // entry fall to different warps
  for (int64_t v = warp; v < S * nq; v += nw) {
    const int g = (int)(v / nq);
    const int64_t t = v - (int64_t)g * nq;
    const unsigned long long e = queue[t];
    unsigned mask = (unsigned)(e & 0xffffu);
    if (__popc(mask) <= g * G) continue;
    for (int k = 0; k < g * G; ++k) mask &= mask - 1;  // the groups before this one
    unsigned grp = 0;
    for (int k = 0; k < G && mask; ++k) {
      grp |= mask & (0u - mask);
      mask &= mask - 1;
    }
    refine_entry<LO>(lane, A, (int64_t)(e >> 32), (int)((e >> 16) & 0xffffu), grp);
  }
}

}  // namespace

cudaError_t gmp_launch_refine(const GmpRefine& A, unsigned order_mask, int sm_count, cudaStream_t stream,
                              int64_t* launches) {
  if (A.n_centers <= 0) return cudaSuccess;
  void (*const kernels[7])(GmpRefine) = {k_refine<0>, k_refine<1>, k_refine<2>, k_refine<3>,
                                         k_refine<4>, k_refine<5>, k_refine<6>};
  for (int l = 0; l < 7; ++l) {
    if (!(order_mask & (1u << l))) continue;
    // as many CTAs as can be resident: the warps take fixed strides of the
    // flagged entries, so a second partial wave would leave most of each
    // SM idle while it runs
    int per_sm = 0;
    const cudaError_t eo = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernels[l], 256, 0);
    if (eo != cudaSuccess) return eo;
    if (per_sm < 1) per_sm = 1;
    // order 6: one CTA (8 warps) per SM.  Its pair loop is bound by
    // instruction fetch, and fewer warps at different points of that code
    // fetch less: perfect FCC 262k refinement 21.5 -> 20.4 ms against two
    // CTAs (12 warps in two 6-warp CTAs: 22.9 ms; 4 warps: 30.6 ms; one CTA
    // per SM for orders 4 and 5 as well: 21.3 ms)
    if (l == 6) per_sm = 1;
    kernels[l]<<<(unsigned)(sm_count * per_sm), 256, 0, stream>>>(A);
    ++*launches;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
