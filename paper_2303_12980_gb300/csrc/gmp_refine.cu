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
// the MCSH components by the same recurrences, and the invariant.
#include "gmp_internal.cuh"
#include "mcsh_gen.cuh"

namespace {

// Moments of order L (2L+1 independent components) of one center and one
// sigma over its pairs, lane-strided, in double-float arithmetic.
template <int L>
__device__ __forceinline__ void refine_moments(int lane, const float4& xhi, const float4& xli,
                                               const GmpStruct& st, const int64_t p0, const int64_t p1,
                                               const GmpPair* __restrict__ pairs,
                                               const float4* __restrict__ atom_xh, const float4* __restrict__ atom_xl,
                                               const float* __restrict__ ktab, int nsig_total, int sig, int kmax,
                                               gmp_f2 (&mu)[13]) {
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
      const gmp_f2 E = gmp_df_exp_neg(gmp_df_mul(gmp_f2{ent[0], ent[1]}, r2));
      R = gmp_df_add(R, gmp_df_mul(gmp_f2{ent[2 + 2 * L], ent[3 + 2 * L]}, E));
    }
    gmp_f2 Sd[(L + 1) * (L + 1)];
    gmp_mcsh_indep_df(L, d[0], d[1], d[2], r2, Sd);
#pragma unroll
    for (int k = 0; k <= 2 * L; ++k) mu[k] = gmp_df_add(mu[k], gmp_df_mul(R, Sd[L * L + k]));
  }
}

__global__ void k_refine(const unsigned long long* __restrict__ flags, const int32_t* __restrict__ count,
                         int64_t cap, float* __restrict__ features, int F, const float4* __restrict__ atom_xh,
                         const float4* __restrict__ atom_xl, const float4* __restrict__ cxh,
                         const float4* __restrict__ cxl, const int32_t* __restrict__ cstruct,
                         const GmpStruct* __restrict__ S, const int64_t* __restrict__ nbr_beg,
                         const int64_t* __restrict__ nbr_end, const GmpPair* __restrict__ pairs,
                         const float* __restrict__ ktab, int nsig_total, int kmax, uint32_t* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t n = *count;
  if (n > cap) {
    if (warp == 0 && lane == 0) atomicOr(err, GMP_DEV_CAPACITY);
    n = cap;
  }
  for (int64_t t = warp; t < n; t += nw) {
    const unsigned long long e = flags[t];
    const int64_t i = (int64_t)(e >> 28);
    const int l = (int)((e >> 24) & 15);
    const int sig = (int)((e >> 12) & 4095);
    const int col = (int)(e & 4095);
    const GmpStruct& st = S[cstruct[i]];
    const float4 xhi = cxh[i], xli = cxl[i];
    gmp_f2 mu[13];
    for (int k = 0; k < 13; ++k) mu[k] = gmp_f2{0.0f, 0.0f};
    const int64_t p0 = nbr_beg[i], p1 = nbr_end[i];
    switch (l) {  // warp-uniform: every lane works on the same entry
      case 0: refine_moments<0>(lane, xhi, xli, st, p0, p1, pairs, atom_xh, atom_xl, ktab, nsig_total, sig, kmax, mu); break;
      case 1: refine_moments<1>(lane, xhi, xli, st, p0, p1, pairs, atom_xh, atom_xl, ktab, nsig_total, sig, kmax, mu); break;
      case 2: refine_moments<2>(lane, xhi, xli, st, p0, p1, pairs, atom_xh, atom_xl, ktab, nsig_total, sig, kmax, mu); break;
      case 3: refine_moments<3>(lane, xhi, xli, st, p0, p1, pairs, atom_xh, atom_xl, ktab, nsig_total, sig, kmax, mu); break;
      case 4: refine_moments<4>(lane, xhi, xli, st, p0, p1, pairs, atom_xh, atom_xl, ktab, nsig_total, sig, kmax, mu); break;
      case 5: refine_moments<5>(lane, xhi, xli, st, p0, p1, pairs, atom_xh, atom_xl, ktab, nsig_total, sig, kmax, mu); break;
      case 6: refine_moments<6>(lane, xhi, xli, st, p0, p1, pairs, atom_xh, atom_xl, ktab, nsig_total, sig, kmax, mu); break;
      default: break;
    }
    for (int k = 0; k <= 2 * l; ++k)
      for (int o = 16; o; o >>= 1) {
        const gmp_f2 other{__shfl_xor_sync(0xffffffffu, mu[k].hi, o), __shfl_xor_sync(0xffffffffu, mu[k].lo, o)};
        mu[k] = gmp_df_add(mu[k], other);
      }
    if (lane == 0) {
      const gmp_f2 f = gmp_mcsh_invariant_df(l, mu);
      features[i * F + col] = f.hi + f.lo;
    }
  }
}

}  // namespace

cudaError_t gmp_launch_refine(const unsigned long long* flags, const int32_t* count, int64_t cap,
                              float* features, int F, const float4* atom_xh, const float4* atom_xl,
                              const float4* center_xh, const float4* center_xl, const int32_t* center_struct,
                              const GmpStruct* structs, const int64_t* nbr_beg, const int64_t* nbr_end,
                              const GmpPair* pairs, const float* ktab, int nsig_total, int kmax, uint32_t* err,
                              int sm_count, cudaStream_t stream, int64_t* launches) {
  k_refine<<<sm_count * 4, 256, 0, stream>>>(flags, count, cap, features, F, atom_xh, atom_xl, center_xh, center_xl,
                                             center_struct, structs, nbr_beg, nbr_end, pairs, ktab, nsig_total, kmax,
                                             err);
  ++*launches;
  return cudaGetLastError();
}
