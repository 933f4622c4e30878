// FP64 recomputation of features that FP32 cannot resolve.
//
// A feature f_{l,s} = sum_c w_c mu_c^2 whose value is tiny compared with the
// cancellation-free scale of its moments (near-symmetric environments make
// l >= 1 moments cancel) loses relative accuracy in FP32 in proportion to
// sqrt(scale / f).  The forward kernels queue such (center, order, sigma)
// entries; this kernel recomputes each of them from the FP64 positions
// (center_pos: the atoms, or the reference points of gmp_featurize_points):
// the displacement by the neighbor definition's own FP64 expression, the
// Gaussian overlap radial factor with FP64 exp, the MCSH components by the
// same recurrences in double, and the invariant in double.
#include "gmp_internal.cuh"
#include "mcsh_gen.cuh"

namespace {

__global__ void k_refine(const unsigned long long* __restrict__ flags, const int32_t* __restrict__ count,
                         int64_t cap, float* __restrict__ features, int F, const double* __restrict__ pos,
                         const double* __restrict__ cpos, const int32_t* __restrict__ cstruct,
                         const GmpStruct* __restrict__ S,
                         const int64_t* __restrict__ nbr_beg, const int64_t* __restrict__ nbr_end,
                         const GmpPair* __restrict__ pairs,
                         const double* __restrict__ ktab, int nsig_total, int kmax, uint32_t* __restrict__ err) {
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
    double mu[13];
    for (int k = 0; k < 13; ++k) mu[k] = 0.0;
    const int64_t p0 = nbr_beg[i], p1 = nbr_end[i];
    for (int64_t p = p0 + lane; p < p1; p += 32) {
      const GmpPair pr = pairs[p];
      int nn[3];
      gmp_unpack_shift(pr.shift, nn);
      double d[3];
      for (int c = 0; c < 3; ++c) {
        const double sh = __dadd_rn(__dadd_rn(__dmul_rn((double)nn[0], st.A[c]), __dmul_rn((double)nn[1], st.A[3 + c])),
                                    __dmul_rn((double)nn[2], st.A[6 + c]));
        d[c] = __dadd_rn(__dsub_rn(pos[3 * (int64_t)pr.j + c], cpos[3 * i + c]), sh);
      }
      const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
      // radial factor: sum_q Kd (alpha/gamma)^l exp(-(alpha beta / gamma) r^2)
      double R = 0.0;
      const double* tq = ktab + ((size_t)pr.e * nsig_total + sig) * kmax * 3;
      for (int q = 0; q < kmax; ++q) {
        double a = tq[3 * q];
        for (int m = 0; m < l; ++m) a = __dmul_rn(a, tq[3 * q + 1]);
        R = __fma_rn(a, exp(-__dmul_rn(tq[3 * q + 2], r2)), R);
      }
      double Sd[49];
      gmp_mcsh_indep_d(l, d[0], d[1], d[2], r2, Sd);
      for (int k = 0; k <= 2 * l; ++k) mu[k] = __fma_rn(R, Sd[l * l + k], mu[k]);
    }
    for (int k = 0; k <= 2 * l; ++k)
      for (int o = 16; o; o >>= 1) mu[k] = __dadd_rn(mu[k], __shfl_xor_sync(0xffffffffu, mu[k], o));
    if (lane == 0) features[i * F + col] = (float)gmp_mcsh_invariant_d(l, mu);
  }
}

}  // namespace

cudaError_t gmp_launch_refine(const unsigned long long* flags, const int32_t* count, int64_t cap,
                              float* features, int F, const double* pos, const double* center_pos,
                              const int32_t* center_struct, const GmpStruct* structs, const int64_t* nbr_beg,
                              const int64_t* nbr_end, const GmpPair* pairs,
                              const double* ktab, int nsig_total, int kmax, uint32_t* err, int sm_count,
                              cudaStream_t stream, int64_t* launches) {
  k_refine<<<sm_count * 4, 256, 0, stream>>>(flags, count, cap, features, F, pos, center_pos, center_struct, structs, nbr_beg, nbr_end,
                                             pairs, ktab, nsig_total, kmax, err);
  ++*launches;
  return cudaGetLastError();
}
