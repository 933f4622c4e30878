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

// exp(-x) for a double-float x >= 0 to about 1e-13 relative, in FP32
// arithmetic, by table-driven reduction (Tang's method):
// x = k ln2/64 + r with |r| <= ln2/128 (ln2/64 as a double-float), so that
// exp(-x) = 2^-(k div 64) * 2^-((k mod 64)/64) * exp(-r); the middle factor
// is a double-float table entry (tab[j] = 2^(-j/64)) and
// exp(-r) = 1 - r + r^2 w, w = 1/2 + r t, t = -1/6 + r/24 - r^2/120, where
// |r t| < 1e-3 lets t be FP32 (the omitted r^6/720 term is below 3e-17).
// Results below the FP32 normal range (x > 87) are returned as 0.
__device__ __forceinline__ gmp_f2 df_exp_neg(gmp_f2 x, const float2* __restrict__ tab) {
  if (!(x.hi <= 87.0f)) return gmp_f2{0.0f, 0.0f};
  const float C_HI = 0.010830424726009369f, C_LO = -2.976022206446771e-11f;  // ln2/64
  const float k = rintf(__fmul_rn(x.hi, 92.33248261689366f));                  // x * 64/ln2
  const gmp_f2 kc = gmp_df_add(gmp_two_prod(k, C_HI), gmp_two_prod(k, C_LO));
  const gmp_f2 r = gmp_df_add(x, gmp_df_neg(kc));
  const float t = __fmaf_rn(r.hi, __fmaf_rn(r.hi, -0.008333333767950535f, 0.0416666679084301f),
                            -0.1666666716337204f);
  const gmp_f2 rt = gmp_two_prod(r.hi, t);
  gmp_f2 w = gmp_fast_two_sum(0.5f, rt.hi);
  w = gmp_fast_two_sum(w.hi, __fadd_rn(w.lo, rt.lo));
  const gmp_f2 q = gmp_df_mul(gmp_df_mul(r, r), w);
  gmp_f2 e = gmp_df_add(gmp_df_add(gmp_f2{1.0f, 0.0f}, gmp_df_neg(r)), q);
  const int ki = (int)k;
  const float2 T = __ldg(tab + (ki & 63));
  e = gmp_df_mul(e, gmp_f2{T.x, T.y});
  return gmp_f2{ldexpf(e.hi, -(ki >> 6)), ldexpf(e.lo, -(ki >> 6))};
}

// Moments of order L (2L+1 independent components) of one center and one
// sigma over its pairs, lane-strided, in double-float arithmetic.
template <int L>
__device__ __forceinline__ void refine_moments(int lane, const float4& xhi, const float4& xli,
                                               const GmpStruct& st, const int64_t p0, const int64_t p1,
                                               const GmpPair* __restrict__ pairs,
                                               const float4* __restrict__ atom_xh, const float4* __restrict__ atom_xl,
                                               const float* __restrict__ ktab, int nsig_total, int sig, int kmax,
                                               const float2* __restrict__ exp_tab, gmp_f2 (&mu)[2 * L + 1]) {
  for (int64_t p = p0 + lane; p < p1; p += 32) {
    const GmpPair pr = pairs[p];
    int nn[3];
    gmp_unpack_shift(pr.shift, nn);
    gmp_f2 d[3], r2;
    float mag;
    gmp_df_disp(xhi, xli, atom_xh[pr.j], atom_xl[pr.j], st, nn, d, r2, mag);
    // radial factor: sum_q A_{q,L} exp(-b_q r^2); table entry (b, A_0 .. A_6) as double-floats
    gmp_f2 R{0.0f, 0.0f};
    const float* te = ktab + ((size_t)pr.e * nsig_total + sig) * kmax * 16;  // [element][sigma][primitive]
    for (int q = 0; q < kmax; ++q) {
      const float* ent = te + q * 16;
      const gmp_f2 E = df_exp_neg(gmp_df_mul(gmp_f2{ent[0], ent[1]}, r2), exp_tab);
      R = gmp_df_add(R, gmp_df_mul(gmp_f2{ent[2 + 2 * L], ent[3 + 2 * L]}, E));
    }
    gmp_f2 Sd[(L + 1) * (L + 1)];
    gmp_mcsh_indep_df(L, d[0], d[1], d[2], r2, Sd);
#pragma unroll
    for (int k = 0; k <= 2 * L; ++k) mu[k] = gmp_df_add(mu[k], gmp_df_mul(R, Sd[L * L + k]));
  }
}

// One flagged feature f_{L,sigma} of one center: moments over the center's
// pairs (lane-strided), warp-reduced, and the invariant, all double-float;
// the result (rounded to FP32) is valid in every lane.  mu_dst (optional)
// receives the 2L+1 moments rounded to FP32.
template <int L>
__device__ __forceinline__ float refine_feature(int lane, const GmpRefine& A, const float4& xhi, const float4& xli,
                                                const GmpStruct& st, int64_t p0, int64_t p1, int sig,
                                                float* mu_dst) {
  gmp_f2 mu[2 * L + 1];
#pragma unroll
  for (int k = 0; k <= 2 * L; ++k) mu[k] = gmp_f2{0.0f, 0.0f};
  refine_moments<L>(lane, xhi, xli, st, p0, p1, A.pairs, A.atom_xh, A.atom_xl, A.ktab, A.nsig_total, sig, A.kmax,
                    A.exp_tab, mu);
#pragma unroll
  for (int k = 0; k <= 2 * L; ++k)
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const gmp_f2 other{__shfl_xor_sync(0xffffffffu, mu[k].hi, o), __shfl_xor_sync(0xffffffffu, mu[k].lo, o)};
      mu[k] = gmp_df_add(mu[k], other);
    }
  if (mu_dst && lane == 0) {
#pragma unroll
    for (int k = 0; k <= 2 * L; ++k) mu_dst[k] = mu[k].hi + mu[k].lo;
  }
  const gmp_f2 f = gmp_mcsh_invariant_df(L, mu);
  return f.hi + f.lo;
}

// One flagged feature (center i, column col) of order LO recomputed by the
// whole warp (entries of other orders are left to that order's launch);
// col_info[col] = (order << 16) | global sigma.
template <int LO>
__device__ __forceinline__ void refine_entry(int lane, const GmpRefine& A, int64_t i, int col) {
  const int info = col < A.F ? A.col_info[col] : -1;
  if (info < 0 || (info >> 16) != LO) return;
  const int sig = info & 0xffff;
  const GmpStruct& st = A.structs[A.center_struct[i]];
  const float4 xhi = A.center_xh[i], xli = A.center_xl[i];
  const int64_t p0 = A.nbr_beg[i], p1 = A.nbr_end[i];
  float* mu_dst = nullptr;
  if (A.mu_out && sig >= A.mu_sig0 && sig < A.mu_sig0 + A.mu_nsig)
    mu_dst = A.mu_out + (i * A.mu_nsig + (sig - A.mu_sig0)) * (int64_t)A.mu_nind + LO * LO;
  const float f = refine_feature<LO>(lane, A, xhi, xli, st, p0, p1, sig, mu_dst);
  if (lane == 0) A.features[i * A.F + col] = f;
}

// Flagged features of order LO (one launch per order, so that every warp of
// a launch runs the same instantiation: the per-order code is large, and
// warps mixing orders thrash the instruction cache).  First the queue
// (entries center << 16 | column, spread over the warps one entry each);
// when it overflowed, the rest are the set bits of the bitmask (bit
// col % 32 of word i * FW + col / 32), which each warp reads 32 words at a
// time (lane = word).
template <int LO>
__global__ void k_refine(const GmpRefine A) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned long long n = *A.count;
  const int64_t nq = n < (unsigned long long)A.cap ? (int64_t)n : A.cap;
  for (int64_t t = warp; t < nq; t += nw) {
    const unsigned long long e = A.queue[t];
    refine_entry<LO>(lane, A, (int64_t)(e >> 16), (int)(e & 0xffffu));
  }
  if (n <= (unsigned long long)A.cap) return;
  const int64_t n_words = A.n_centers * A.flag_words;
  for (int64_t base = warp * 32; base < n_words; base += nw * 32) {
    const uint32_t word = base + lane < n_words ? A.bits[base + lane] : 0u;
    unsigned live = __ballot_sync(0xffffffffu, word != 0u);
    while (live) {  // warp-uniform from here on
      const int src = __ffs(live) - 1;
      live &= live - 1;
      uint32_t wv = __shfl_sync(0xffffffffu, word, src);
      const int64_t tw = base + src;
      const int64_t i = tw / A.flag_words;
      const int cbase = (int)(tw - i * A.flag_words) * 32;
      while (wv) {
        const int col = cbase + __ffs(wv) - 1;
        wv &= wv - 1;
        refine_entry<LO>(lane, A, i, col);
      }
    }
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
    kernels[l]<<<(unsigned)(sm_count * per_sm), 256, 0, stream>>>(A);
    ++*launches;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
