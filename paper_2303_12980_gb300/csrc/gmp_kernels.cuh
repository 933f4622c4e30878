// GMP moment, feature, VJP and Jacobian kernels (templates on the highest
// MCSH order L and the padded sigma count NS).
//
// Per center i the moments are (GMP-Featurizer, Statement of Needs: the
// local density as a multipole expansion; Examples: MCSH orders x sigmas)
//   mu_{l,s,k}(i) = sum over neighbor images p of R_{l,s}(r_p^2) S_k(d_p)
// with S_k the MCSH polynomial of component k and the radial factor
//   R_{l,s}(r^2) = sum_q c_q N_s (pi/g)^(3/2) (alpha_q/g)^l exp(-(alpha_q beta_s/g) r^2),
//   beta_s = 1/(2 s^2), g = alpha_q + beta_s, N_s = (2 pi s^2)^(-3/2).
// This factorised form is the Gaussian overlap integral of the density
// primitive c_q exp(-alpha_q |r - d|^2) with the probe N_s S_k(r) exp(-beta_s r^2):
// the Gaussian product theorem moves the product to a Gaussian centred at
// (alpha/g) d, and the Gaussian average of a harmonic polynomial equals its
// value at the centre, so the integral is K S_k((alpha/g) d) = K (alpha/g)^l S_k(d).
// Feature f_{l,s} = sum over all components of l!/(a!b!c!) mu^2 (the
// rotation invariant of the group).  Only the 2l+1 independent components
// (a <= 1) are accumulated; the rest follow from tracelessness.
//
// Layout: one warp per center (persistent warps take centers from an atomic
// counter).  The forward kernel walks its center's neighbor list in tiles of
// 16 pairs (two lanes per pair) or 32 (one lane per pair):
//   phase 1, lane = pair (and half of its sigma groups): exps and radial
//            factors R[l][s] (double-float exponent argument, four sigmas per
//            16-byte table load, packed FP32 pairs), MCSH values S[k] ->
//            shared-memory tiles;
//   phase 2, lane = block of 4 sigmas x 4 components: packed FP32 FMAs over
//            the tile, the partial of every 16 pairs folded into a (hi, lo)
//            pair by TwoSum (blocked compensated summation over neighbors).
// The backward kernel takes one pair per lane and recomputes its radial
// factors (one order more: dR_l/dr^2 = -beta R_{l+1}) and MCSH values to
// apply the adjoints of the center's features.
#pragma once

#include "gmp_internal.cuh"
#include "mcsh_gen.cuh"

#include <utility>

namespace gmpk {

// Compile-time loop: f(std::integral_constant<int, 0>), ..., f(<N-1>).
template <typename F, int... Cs>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Cs...>) {
  (f(std::integral_constant<int, Cs>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

__host__ __device__ constexpr int chunks_of_order(int l) { return (l + 2) / 2; }  // ceil((2l+1)/4)
__host__ __device__ constexpr int nchunks(int L) {
  int n = 0;
  for (int l = 0; l <= L; ++l) n += chunks_of_order(l);
  return n;
}
__host__ __device__ constexpr int chunk_l(int c) {
  int l = 0;
  while (c >= chunks_of_order(l)) { c -= chunks_of_order(l); ++l; }
  return l;
}
__host__ __device__ constexpr int chunk_k0(int c) {
  int l = 0;
  while (c >= chunks_of_order(l)) { c -= chunks_of_order(l); ++l; }
  return l * l + 4 * c;
}
// chunk holding the last independent components of order l
__host__ __device__ constexpr int last_chunk(int l) {
  int c = 0;
  for (int m = 0; m <= l; ++m) c += chunks_of_order(m);
  return c - 1;
}
// order l of flat independent component k (k in [l^2, (l+1)^2))
__host__ __device__ constexpr int order_of(int k) {
  int l = 0;
  while ((l + 1) * (l + 1) <= k) ++l;
  return l;
}
// The same for a chunk width cw of 4 (above) or 2.  With cw = 2 an order l
// takes l + 1 chunks: its 2l + 1 components and, in the last slot, r^l.
__host__ __device__ constexpr int chunks_of_order_w(int l, int cw) { return cw == 4 ? (l + 2) / 2 : l + 1; }
__host__ __device__ constexpr int nchunks_w(int L, int cw) {
  int n = 0;
  for (int l = 0; l <= L; ++l) n += chunks_of_order_w(l, cw);
  return n;
}
__host__ __device__ constexpr int chunk_l_w(int c, int cw) {
  int l = 0;
  while (c >= chunks_of_order_w(l, cw)) { c -= chunks_of_order_w(l, cw); ++l; }
  return l;
}
__host__ __device__ constexpr int chunk_k0_w(int c, int cw) {
  int l = 0;
  while (c >= chunks_of_order_w(l, cw)) { c -= chunks_of_order_w(l, cw); ++l; }
  return l * l + cw * c;
}
// Chunk width of the moment contraction for orders 0..L and NS sigmas: the
// one with fewer warp instructions per pair (items of 4 sigmas x cw
// components, 32 per warp pass; an item issues 2 cw packed FMAs and two
// shared loads per pair), 2 on a tie (fewer accumulator registers).
__host__ __device__ constexpr int pick_cw(int L, int NS) {
  const int q4 = ((NS / 4) * nchunks_w(L, 4) + 31) / 32, q2 = ((NS / 4) * nchunks_w(L, 2) + 31) / 32;
  return q4 * 10 < q2 * 6 ? 4 : 2;
}
// smallest m >= n with m / 2 odd (conflict-free 8-byte stores by 16
// consecutive lanes at a stride of m floats)
__host__ __device__ constexpr int odd2(int n) {
  int h = (n + 1) / 2;
  if ((h & 1) == 0) ++h;
  return 2 * h;
}

// float count rounded to a multiple of 4 holding an odd number of float4s
// (conflict-free 16-byte stores by 8 consecutive lanes)
__host__ __device__ constexpr int odd4(int n) {
  int q = (n + 3) / 4;
  if ((q & 1) == 0) ++q;
  return 4 * q;
}

template <int L, int NS, int TILE_ = 16>
struct Shape {
  static constexpr int NIND = (L + 1) * (L + 1);   // independent components, orders 0..L
  static constexpr int NIND1 = (L + 2) * (L + 2);  // ... orders 0..L+1
  static constexpr int NINDP = (NIND + 3) / 4 * 4; // padded row of per-sigma vectors
  static constexpr int NSB = NS / 4;
  static constexpr int CW = pick_cw(L, NS);        // components per contraction item
  static constexpr int NCH = nchunks_w(L, CW);
  static constexpr int NITEM = NSB * NCH;
  static constexpr int Q = (NITEM + 31) / 32;
  // cw = 4: r^l, l = 0..L, after the S chunks (mixed signs); cw = 2 keeps
  // r^l in the last slot of every order
  static constexpr int RL4 = CW == 4 ? (L + 1 + 3) / 4 * 4 : 0;
  static constexpr int RSTR = odd4((L + 1) * NS);
  static constexpr int TILE = TILE_;               // pairs staged per tile: 16 (2 lanes per pair) or 32
  static constexpr int SSTR = CW == 4 ? odd4(NCH * 4 + RL4)
                                      : odd2(NCH * 2 > (NS * NINDP + TILE_ - 1) / TILE_ ? NCH * 2
                                                                                        : (NS * NINDP + TILE_ - 1) / TILE_);
  static constexpr int FOLD = 16;                  // pairs per FP32 partial before the TwoSum fold
  static_assert(TILE_ == 16 || TILE_ == 32, "tile of 16 or 32 pairs");
  static constexpr int WARP_FLOATS = TILE * RSTR + TILE * SSTR;
  static_assert(NS * NIND + NS * (L + 1) <= TILE * RSTR, "moments and bounds must fit the R tile");
  static_assert(NS * NINDP <= TILE * SSTR, "adjoints must fit the S tile");
};

// Per-warp shared floats of the backward kernel's strain-derivative sums
// ([9][32]: one column per lane).  They reuse the moment block of the
// warp's region (dead once the adjoints are formed) when it is large
// enough, else they take extra space after the region.
constexpr int kVirialFloats = 9 * 32;
template <int L, int NS>
constexpr int virial_extra_floats() {
  return Shape<L, NS>::TILE * Shape<L, NS>::RSTR >= kVirialFloats ? 0 : kVirialFloats;
}

// Strides of the shared-memory radial table: within an element, the
// blocks of its 4-sigma groups (kmax primitives x gmp_rad_block(L) float4s
// each) an odd number of float4s apart (pad), so that lanes reading two
// groups of one element at once hit different banks; the elements an odd
// number of float4s apart, for lanes reading different elements.  The
// plain backward and the Jacobian kernels keep the groups unpadded: the
// padded stride costs each a register it does not have.
__host__ __device__ inline int rad_sg_stride(int L, int kmax, bool pad = true) {
  return pad ? (kmax * gmp_rad_block(L)) | 1 : kmax * gmp_rad_block(L);
}
__host__ __device__ inline int rad_elem_stride(int L, int NS, int kmax, bool pad = true) {
  int q = (NS / 4) * rad_sg_stride(L, kmax, pad);
  if ((q & 1) == 0) ++q;
  return 4 * q;
}
__host__ __device__ inline int dens_elem_stride(int kmax) {
  int q = kmax * (GMP_DENS_STRIDE / 4);
  if ((q & 1) == 0) ++q;
  return 4 * q;
}

struct KParams {
  GmpPass pass;
  int64_t N;
  const int64_t* nbr_beg;  // pairs of center i: nbr_beg[i] .. nbr_end[i]-1 (CSR: end = beg + 1)
  const int64_t* nbr_end;
  const GmpPair* pairs;
  float* features;        // [N, F] or null
  float* mu_out;          // [N, nsig, NIND] or null
  const float* grad_feat; // [N, F] (vjp)
  double* grad_acc;       // [N, 3] (vjp)
  const int64_t* jac_off; // [N+1] (jacobian)
  const int32_t* jac_row; // [P] row of each pair within its center (jacobian)
  int32_t* jac_j;
  float* jac;             // [nnz, F, 3]
  int32_t* counter;
  int64_t center0;        // centers center0 .. N-1 (the work counter starts there);
                          // jac_off row 0 belongs to center center0 (jacobian)
  const int32_t* center_struct;  // [N] structure of each center (virial)
  double* virial;                // [S, 3, 3] strain derivative accumulators (virial)
  // features too ill-conditioned for FP32 (recomputed in double-float
  // afterwards): one queue entry per (center, order) of the pass,
  // center << 32 | first column of the order << 16 | mask of the sigmas,
  // in the queue of the order's slot o (flags + o * flag_cap, count
  // flag_count[o])
  unsigned long long* flags;
  unsigned long long* flag_count;
  int64_t flag_cap;
  int64_t pair_cap;           // pairs buffer capacity: centers beyond it are skipped
  int sig0;                   // global index of this pass's first sigma
  float flag_tau;             // flag when flag_low * l! (2l-1)!! B^2 / 3^l <= f < flag_tau * l! (2l-1)!! B^2
  float flag_low;
  // VJP without float atomics: the gradient of each pair onto its neighbor
  // atom j is added exactly, as an integer, into one of kGradBins
  // fixed-point bins of (j, component) (gbins, see bin_add); each center's
  // own term goes to own[3 i + v] and its strain-derivative sums to
  // vir_c[9 i + v].  gmp_launch_grad_bins_finish then forms the gradient.
  unsigned long long* gbins;
  double* own;
  double* vir_c;
};

// l! (2l-1)!!: with B = sum_pairs |R_{l,s}| r^l, the cancellation-free scale
// F_abs = sum_c w_c (sum_pairs |R S_c|)^2 is the squared weighted norm of a
// sum over pairs of non-negative vectors, so by the triangle inequality
// F_abs <= (sum_pairs |R| sqrt(sum_c w_c S_c^2))^2 = l! (2l-1)!! B^2, using
// sum_c w_c S_c^2 = l! (2l-1)!! r^(2l).
__host__ __device__ constexpr float flag_scale(int l) {
  return l == 0 ? 1.0f : l == 1 ? 1.0f : l == 2 ? 6.0f : l == 3 ? 90.0f : l == 4 ? 2520.0f
       : l == 5 ? 113400.0f : 7484400.0f;
}
// 3^-l.  From below, F_abs >= l! (2l-1)!! B^2 / 3^l: by Cauchy-Schwarz over
// the components, F_abs >= (sum_c w_c A_c)^2 / sum_c w_c with sum_c w_c =
// 3^l, and sum_c w_c A_c = sum_pairs |R| sum_c w_c |S_c| >= sum_pairs |R|
// sqrt(sum_c w_c S_c^2) = sqrt(l! (2l-1)!!) B, since w_c >= 1.
__host__ __device__ constexpr float inv_pow3(int l) {
  return l == 0 ? 1.0f : l == 1 ? 1.0f / 3.0f : l == 2 ? 1.0f / 9.0f : l == 3 ? 1.0f / 27.0f : l == 4 ? 1.0f / 81.0f
       : l == 5 ? 1.0f / 243.0f : 1.0f / 729.0f;
}

__device__ __forceinline__ void load_pair(const GmpPair* __restrict__ pairs, int64_t idx, float& dx,
                                          float& dy, float& dz, float& r2h, float& r2l, int& e,
                                          int& j) {
  const float4* p4 = reinterpret_cast<const float4*>(pairs + idx);
  const float4 a = __ldg(p4);
  const float4 b = __ldg(p4 + 1);
  dx = a.x; dy = a.y; dz = a.z; r2h = a.w;
  r2l = b.x;
  e = __float_as_int(b.y);
  j = __float_as_int(b.z);
}

// r^2 fed to the MCSH recurrences: formed from the FP32 components
// themselves, so that the recurrences evaluate the harmonic polynomials of
// (dx, dy, dz) exactly as written.  The pair record's r^2 (that of the
// exact displacement, which the exponent arguments use) differs from
// dx^2 + dy^2 + dz^2 of the rounded components by ~2^-24 relative; with it
// the recurrences would mix a non-harmonic part of that relative size into
// every component, and their integer coefficients amplify it: a Jacobian
// entry then carried ~5 units of 2^-24 of its cancellation-free scale
// instead of ~1.5.
__device__ __forceinline__ float mcsh_r2(float dx, float dy, float dz) {
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Exact, order-independent accumulation of FP32 values.  A finite value is
// m 2^(e - 150) with m its 24-bit significand and e its biased exponent (1
// for subnormals).  Bin b = (e - 1) / 24 (0..10) counts in units of
// 2^(24 b - 149): the value is m << ((e - 1) % 24) < 2^47 of them, an exact
// integer added with a 64-bit integer atomic, so the bin's total does not
// depend on the order of the additions; up to 2^16 values per bin stay
// below 2^63.  Bin 11 collects flags of non-finite values (1 NaN, 2 +inf,
// 4 -inf).  The bins are combined in a fixed order afterwards.
constexpr int kGradBins = 12;
__device__ __forceinline__ void bin_add(unsigned long long* bins, float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned eb = (u >> 23) & 0xffu;
  if (eb == 0xffu) {
    atomicOr(bins + 11, (u & 0x7fffffu) ? 1ull : ((u >> 31) ? 4ull : 2ull));
    return;
  }
  const unsigned long long m = eb ? ((u & 0x7fffffu) | 0x800000u) : (u & 0x7fffffu);
  if (!m) return;
  const unsigned e = eb ? eb - 1u : 0u;
  const unsigned b = e / 24u;
  const unsigned long long x = m << (e - 24u * b);
  atomicAdd(bins + b, (u >> 31) ? (~x + 1ull) : x);
}

// Pulls the cache line of a pair record into L1 ahead of its use (no registers held).
__device__ __forceinline__ void prefetch_pair(const GmpPair* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Radial factors of one pair for a group of 4 sigmas, orders 0..NL-1 (the
// forward needs L+1 orders; the backward one more, for the derivative
// dR_l/dr^2 = -beta R_{l+1}).  Each 16-byte table load serves the four
// sigmas of the group.
// Radial factors with the exponent argument B r^2 as a double-float (about
// 1e-7 relative: the features), computed on packed FP32 pairs (sigmas
// (0,1) and (2,3) of the group) with the rounding of the scalar form.
template <int L, int NL = L + 2>
__device__ __forceinline__ void radial4d(const float* __restrict__ tab_e, int kmax, int sg, float r2h,
                                         float r2l, float (&R)[4][NL]) {
  constexpr int RB = gmp_rad_block(L);
  // sigma pairs (0,1) and (2,3) of the group as packed FP32 pairs
  float2 Rp[2][NL];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int l = 0; l < NL; ++l) Rp[h][l] = make_float2(0.0f, 0.0f);
  const float2 nr2h = make_float2(-r2h, -r2h), r2h2 = make_float2(r2h, r2h), r2l2 = make_float2(r2l, r2l);
#pragma unroll 1
  for (int q = 0; q < kmax; ++q) {
    const float4* blk = reinterpret_cast<const float4*>(tab_e) + sg * rad_sg_stride(L, kmax) + q * RB;
    const float4 bh = blk[0];
    const float4 bl = blk[1];
    float2 E[2];
    E[0] = gmp_exp_neg2(make_float2(bh.x, bh.y), make_float2(bl.x, bl.y), nr2h, r2h2, r2l2);
    E[1] = gmp_exp_neg2(make_float2(bh.z, bh.w), make_float2(bl.z, bl.w), nr2h, r2h2, r2l2);
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const float4 a = blk[2 + l];
      Rp[0][l] = gmp_fma2(make_float2(a.x, a.y), E[0], Rp[0][l]);
      Rp[1][l] = gmp_fma2(make_float2(a.z, a.w), E[1], Rp[1][l]);
    }
  }
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    R[0][l] = Rp[0][l].x;
    R[1][l] = Rp[0][l].y;
    R[2][l] = Rp[1][l].x;
    R[3][l] = Rp[1][l].y;
  }
}

// Radial factors scaled by 2^32 for the backward, with scalar FP32
// operations (the backward kernel keeps its 168-register budget with these;
// packed pairs need aligned register pairs and spill there).  The exponent
// argument 32 - B r^2 is one FMA, rounded once: an absolute error of at most
// 2^-18 while the scaled factor is normal (|32 - B r^2| < 128), so each
// exponential is within ~2e-6 relative: ample for derivatives, checked to
// 1e-4.  The offset keeps the factors normal (not flushed to zero by the SFU)
// down to exp(-B r^2) = 2^-158, with room for the amplitudes (alpha/gamma)^l
// of the higher orders: a gradient term of a far pair, multiplied by large
// adjoints, keeps its digits; the kernel scales its sums back by 2^-32.
template <int L, int NL = L + 2, bool PADG = true>
__device__ __forceinline__ void radial4s(const float* __restrict__ tab_e, int kmax, int sg, float r2h,
                                         float (&R)[4][NL]) {
  constexpr int RB = gmp_rad_block(L);
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int l = 0; l < NL; ++l) R[u][l] = 0.0f;
#pragma unroll 1
  for (int q = 0; q < kmax; ++q) {
    const float4* blk = reinterpret_cast<const float4*>(tab_e) + sg * rad_sg_stride(L, kmax, PADG) + q * RB;
    const float4 bh = blk[0];
    float E[4];
    E[0] = gmp_ex2(__fmaf_rn(bh.x, -r2h, GMP_EXP_SHIFT));
    E[1] = gmp_ex2(__fmaf_rn(bh.y, -r2h, GMP_EXP_SHIFT));
    E[2] = gmp_ex2(__fmaf_rn(bh.z, -r2h, GMP_EXP_SHIFT));
    E[3] = gmp_ex2(__fmaf_rn(bh.w, -r2h, GMP_EXP_SHIFT));
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const float4 a = blk[2 + l];
      const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) R[u][l] = __fmaf_rn(av[u], E[u], R[u][l]);
    }
  }
}

// The same scaled radial factors with the exact offset and the double-float
// exponent argument (gmp_exp_neg_shifted), for tables with coefficients of
// both signs: there the radial factor of an element can cancel within the
// pair, and the exponentials' errors count against sum_q |A_q| E_q rather
// than against the factor.  (A separate instantiation of the backward
// kernel: a runtime branch would raise the register count of every one.)
template <int L, int NL = L + 2, bool PADG = true>
__device__ __forceinline__ void radial4x(const float* __restrict__ tab_e, int kmax, int sg, float r2h,
                                         float r2l, float (&R)[4][NL]) {
  constexpr int RB = gmp_rad_block(L);
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int l = 0; l < NL; ++l) R[u][l] = 0.0f;
#pragma unroll 1
  for (int q = 0; q < kmax; ++q) {
    const float4* blk = reinterpret_cast<const float4*>(tab_e) + sg * rad_sg_stride(L, kmax, PADG) + q * RB;
    const float4 bh = blk[0], bl = blk[1];
    float E[4];
    E[0] = gmp_exp_neg_shifted(bh.x, bl.x, r2h, r2l);
    E[1] = gmp_exp_neg_shifted(bh.y, bl.y, r2h, r2l);
    E[2] = gmp_exp_neg_shifted(bh.z, bl.z, r2h, r2l);
    E[3] = gmp_exp_neg_shifted(bh.w, bl.w, r2h, r2l);
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const float4 a = blk[2 + l];
      const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) R[u][l] = __fmaf_rn(av[u], E[u], R[u][l]);
    }
  }
}

// The scaled radial factors of radial4s on packed FP32 pairs, sigmas (0,1)
// and (2,3) of the group: bit-identical to the scalar form, half the issue
// slots.
template <int L, int NL = L + 2, bool PADG = true>
__device__ __forceinline__ void radial4p(const float* __restrict__ tab_e, int kmax, int sg, float r2h,
                                         float (&R)[4][NL]) {
  constexpr int RB = gmp_rad_block(L);
  float2 Rp[2][NL];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int l = 0; l < NL; ++l) Rp[h][l] = make_float2(0.0f, 0.0f);
  const float2 nr2 = make_float2(-r2h, -r2h), sh = make_float2(GMP_EXP_SHIFT, GMP_EXP_SHIFT);
#pragma unroll 1
  for (int q = 0; q < kmax; ++q) {
    const float4* blk = reinterpret_cast<const float4*>(tab_e) + sg * rad_sg_stride(L, kmax, PADG) + q * RB;
    const float4 bh = blk[0];
    const float2 x0 = gmp_fma2(make_float2(bh.x, bh.y), nr2, sh), x1 = gmp_fma2(make_float2(bh.z, bh.w), nr2, sh);
    const float2 E0 = make_float2(gmp_ex2(x0.x), gmp_ex2(x0.y)), E1 = make_float2(gmp_ex2(x1.x), gmp_ex2(x1.y));
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const float4 a = blk[2 + l];
      Rp[0][l] = gmp_fma2(make_float2(a.x, a.y), E0, Rp[0][l]);
      Rp[1][l] = gmp_fma2(make_float2(a.z, a.w), E1, Rp[1][l]);
    }
  }
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    R[0][l] = Rp[0][l].x;
    R[1][l] = Rp[0][l].y;
    R[2][l] = Rp[1][l].x;
    R[3][l] = Rp[1][l].y;
  }
}

// Density at the center from one pair, sum_q c_q exp(-alpha_q r^2), and its
// derivative in r^2, both scaled by 2^32 (a density of a point far from
// every atom, or one row of a far pair, is linear in the exponentials: it
// keeps its digits down to exp = 2^-158).
__device__ __forceinline__ float density_term(const float* __restrict__ dens_e, int kmax, float r2h,
                                              float r2l, float* deriv) {
  float rho = 0.0f, drho = 0.0f;
  for (int q = 0; q < kmax; ++q) {
    const float4 h = *reinterpret_cast<const float4*>(dens_e + q * GMP_DENS_STRIDE);
    const float t = __fmul_rn(h.w, gmp_exp_neg_shifted(h.x, h.y, r2h, r2l));
    rho = __fadd_rn(rho, t);
    drho = __fmaf_rn(-h.z, t, drho);
  }
  if (deriv) *deriv = drho;
  return rho;
}

// The same density term in double-float arithmetic, scaled by 2^32, for
// tables with coefficients of both signs: there the primitives of one
// element can cancel, and FP32 terms (exponentials within 2 ulp, FP32
// coefficients) would leave errors relative to sum_q |c_q| exp(-alpha_q
// r^2) rather than to the density.  Each exponential comes from the
// double-float argument alpha r^2 - 32 ln 2 (gmp_df_exp_neg, ~1e-13), each
// coefficient is a double-float, and the terms are summed in double-float.
// (Out of line: it runs only for such tables and its registers would
// otherwise count against every forward kernel.)
static __device__ __noinline__ gmp_f2 density_term_df(const float* __restrict__ dens_e, int kmax, float r2h,
                                                      float r2l, const float2* __restrict__ exp_tab) {
  const gmp_f2 r2{r2h, r2l}, nshift{-22.180709838867188f, 6.094893478802987e-08f};  // -32 ln 2
  gmp_f2 rho{0.0f, 0.0f};
  for (int q = 0; q < kmax; ++q) {
    const float4 h0 = *reinterpret_cast<const float4*>(dens_e + q * GMP_DENS_STRIDE);
    const float4 h1 = *reinterpret_cast<const float4*>(dens_e + q * GMP_DENS_STRIDE + 4);
    const gmp_f2 E = gmp_df_exp_neg(gmp_df_add(gmp_df_mul(gmp_f2{h0.z, h1.x}, r2), nshift), exp_tab);
    rho = gmp_df_add(rho, gmp_df_mul(gmp_f2{h0.w, h1.y}, E));
  }
  return rho;
}

// Tables with coefficients of both signs: the radial factor R = sum_q A_q
// E_q of an element whose primitives differ in sign cancels within the
// pair, and its FP32 rounding is relative to sum_q |A_q| E_q, not to |R|.
// The refinement bound then takes B_{l,s} = sum_pairs sum_q |A_{l,q,s}| E_q
// r^l: recomputed here over the center's pairs (lanes = sigma x pair
// stream, FP32; a bound) and written over the slots that forward_sweep
// filled from |R|.  The streams are reduced in a fixed order, so the bound,
// and with it the refinement flags, are the same in every kernel.
template <int L, int NS>
__device__ __noinline__ void mixed_sign_bound(const GmpPass& P, const float* __restrict__ s_rad,
                                              const GmpPair* __restrict__ pairs, int64_t p0, int M,
                                              float* Mu) {
  constexpr int RB = gmp_rad_block(L);
  constexpr int NIND = (L + 1) * (L + 1);
  constexpr int STREAMS = 32 / NS;
  const int lane = threadIdx.x & 31;
  const int s = lane % NS, h = lane / NS;
  float B[L + 1];
#pragma unroll
  for (int l = 0; l <= L; ++l) B[l] = 0.0f;
  if (s < P.nsig) {
    for (int pp = h; pp < M; pp += STREAMS) {
      float dx, dy, dz, r2h, r2l;
      int e, j;
      load_pair(pairs, p0 + pp, dx, dy, dz, r2h, r2l, e, j);
      const float* tab_e = s_rad + (size_t)e * rad_elem_stride(L, NS, P.kmax);
      float Ra[L + 1];
#pragma unroll
      for (int l = 0; l <= L; ++l) Ra[l] = 0.0f;
      for (int q = 0; q < P.kmax; ++q) {
        const float* ent = tab_e + ((size_t)(s / 4) * rad_sg_stride(L, P.kmax) + (size_t)q * RB) * 4 + (s % 4);
        const float E = gmp_ex2(-__fmul_rn(ent[0], r2h));
#pragma unroll
        for (int l = 0; l <= L; ++l) Ra[l] = __fmaf_rn(fabsf(ent[4 * (2 + l)]), E, Ra[l]);
      }
      const float r = __fsqrt_rn(r2h);
      float rp = 1.0f;
#pragma unroll
      for (int l = 0; l <= L; ++l) {
        B[l] = __fmaf_rn(Ra[l], rp, B[l]);
        rp = __fmul_rn(rp, r);
      }
    }
  }
#pragma unroll
  for (int o = NS; o < 32; o <<= 1)
#pragma unroll
    for (int l = 0; l <= L; ++l) B[l] = __fadd_rn(B[l], __shfl_xor_sync(0xffffffffu, B[l], o));
  __syncwarp();
  if (h == 0 && s < P.nsig)
#pragma unroll
    for (int l = 0; l <= L; ++l) Mu[NS * NIND + s * (L + 1) + l] = B[l];
  __syncwarp();
}

// Shared memory: tables first (radial then density), then one region per warp.


__host__ __device__ inline size_t table_floats(int n_el, int L, int NS, int kmax, bool pad = true) {
  return (size_t)n_el * rad_elem_stride(L, NS, kmax, pad) + (size_t)n_el * dens_elem_stride(kmax);
}

// Copies the radial and density tables to shared memory, padding each
// element's and each sigma group's block to its bank-spreading stride.
template <int L, bool PADG = true>
__device__ __forceinline__ void load_tables(const GmpPass& P, int NS, float* s_rad, float* s_dens) {
  const int blk = P.kmax * gmp_rad_block(L);  // float4s per sigma group in global memory
  const int per = (NS / 4) * blk;             // ... per element
  const int es = rad_elem_stride(L, NS, P.kmax, PADG) / 4, gs = rad_sg_stride(L, P.kmax, PADG);
  for (int t = threadIdx.x; t < P.n_el * per; t += blockDim.x) {
    const int e = t / per, r = t - e * per, g = r / blk;
    reinterpret_cast<float4*>(s_rad)[e * es + g * gs + (r - g * blk)] =
        __ldg(reinterpret_cast<const float4*>(P.rad) + t);
  }
  if (P.want_density) {
    const int dper = P.kmax * (GMP_DENS_STRIDE / 4);
    const int ds = dens_elem_stride(P.kmax) / 4;
    for (int t = threadIdx.x; t < P.n_el * dper; t += blockDim.x) {
      const int e = t / dper, r = t - e * dper;
      reinterpret_cast<float4*>(s_dens)[e * ds + r] = __ldg(reinterpret_cast<const float4*>(P.dens) + t);
    }
  }
}

// ------------------------------------------------------------------------
// Forward sweep over one center's pairs: leaves mu (FP32, rounded from the
// compensated pair) in Mu[s * NIND + k] and the conditioning bound
// B_{l,s} = sum_pairs |R_{l,s}| r^l in Mu[NS * NIND + s * (L+1) + l]
// (with coefficients of both signs, sum over pairs and primitives of
// |A_q E_q| r^l: mixed_sign_bound)
// (warp-private shared memory), and returns the density (all lanes).
// The contraction runs over items of 4 sigmas x CW components (CW = 4 or
// 2, whichever the shape fills the warp's lanes with in fewer
// instructions).  The last chunk of every order has a free last slot (2l+1
// is odd); with non-negative density coefficients (R >= 0) that slot of the
// S row holds r^l, so the moment accumulator of the slot is B itself.  With
// mixed signs B is accumulated from |R| explicitly (CW = 4: the slot holds 0
// and a separate loop reads r^l after the chunks; CW = 2: the slot holds r^l
// and its accumulator takes |R|).
template <int L, int NS, int TILE = 16>
__device__ __forceinline__ float forward_sweep(const GmpPass& P, const float* __restrict__ s_rad,
                                               const float* __restrict__ s_dens,
                                               const GmpPair* __restrict__ pairs, int64_t p0,
                                               int M, float* Rt, float* St,
                                               float* Mu, const int (&it_l)[Shape<L, NS>::Q],
                                               const int (&it_sb)[Shape<L, NS>::Q],
                                               const int (&it_ch)[Shape<L, NS>::Q],
                                               const bool (&it_ok)[Shape<L, NS>::Q]) {
  using SH = Shape<L, NS, TILE>;
  constexpr int CW = SH::CW;
  const int lane = threadIdx.x & 31;
  float hi[SH::Q][4 * CW], lo[SH::Q][4 * CW];
#pragma unroll
  for (int q = 0; q < SH::Q; ++q)
#pragma unroll
    for (int v = 0; v < 4 * CW; ++v) { hi[q][v] = 0.0f; lo[q][v] = 0.0f; }
  float rho_hi = 0.0f, rho_lo = 0.0f;
  const bool mixed = P.mixed_sign != 0;

  constexpr int LPP = 32 / TILE;      // phase 1: lanes per pair (2 or 1)
  const int half = LPP == 2 ? (lane >> 4) : 0;
  const int pl = LPP == 2 ? (lane & 15) : lane;
  constexpr int SG_LO = LPP == 2 ? (SH::NSB + 1) / 2 : SH::NSB;  // sigma groups of half 0: [0, SG_LO)
  const int sg0 = half ? SG_LO : 0, sg1 = half ? SH::NSB : SG_LO;
  for (int base = 0; base < M; base += SH::TILE) {
    const int np = min(SH::TILE, M - base);
    // ---- phase 1: lanes (pair, half); both halves evaluate S and store
    // alternate chunks, each half computes the radial factors of half the
    // sigma groups
    if (pl < np) {
      float dx, dy, dz, r2h, r2l;
      int e, j;
      load_pair(pairs, p0 + base + pl, dx, dy, dz, r2h, r2l, e, j);
      if (half == 0 && base + SH::TILE + pl < M) prefetch_pair(pairs + p0 + base + SH::TILE + pl);
      float* srow = St + pl * SH::SSTR;
      if constexpr (CW == 2) {
        if (half == 0) {  // MCSH components, then r^l in the last slot of each order
          float S[SH::NIND];
          GmpMcsh<L>::eval(dx, dy, dz, mcsh_r2(dx, dy, dz), S);
          const float r = __fsqrt_rn(r2h);
          float rpow = 1.0f;
          static_for<L + 1>([&](auto ll) {
            constexpr int l = decltype(ll)::value;
            static_for<l + 1>([&](auto cc) {
              constexpr int c = decltype(cc)::value;
              constexpr int k = l * l + 2 * c;
              *reinterpret_cast<float2*>(srow + l * (l + 1) + 2 * c) =
                  make_float2(S[k], c == l ? rpow : S[c == l ? k : k + 1]);
            });
            rpow = __fmul_rn(rpow, r);
          });
        }
      } else {
        if (half == 0) {  // MCSH components; r^l in the free slot of each order's last chunk
          float S[SH::NIND];
          GmpMcsh<L>::eval(dx, dy, dz, mcsh_r2(dx, dy, dz), S);
          static_for<SH::NCH>([&](auto cc) {
            constexpr int c = decltype(cc)::value;
            constexpr int k0 = chunk_k0(c);
            constexpr int kend = (chunk_l(c) + 1) * (chunk_l(c) + 1);
            if constexpr (k0 + 4 < kend + 1 && k0 + 3 < kend) {  // full chunk
              *reinterpret_cast<float4*>(srow + 4 * c) = make_float4(S[k0], S[k0 + 1], S[k0 + 2], S[k0 + 3]);
            } else if constexpr (k0 + 1 == kend) {  // last chunk, one component: .y = 0
              *reinterpret_cast<float2*>(srow + 4 * c) = make_float2(S[k0], 0.0f);
            } else {  // last chunk, three components
              *reinterpret_cast<float2*>(srow + 4 * c) = make_float2(S[k0], S[(k0 + 1 < kend) ? k0 + 1 : k0]);
              srow[4 * c + 2] = S[(k0 + 2 < kend) ? k0 + 2 : k0];
            }
          });
        }
        if (LPP == 1 || half == 1) {  // free slots of the last chunks: r^l (0 with mixed signs)
          const float r = __fsqrt_rn(r2h);
          float rpow = mixed ? 0.0f : 1.0f;
          static_for<L + 1>([&](auto ll) {
            constexpr int l = decltype(ll)::value;
            constexpr int c = last_chunk(l);
            if constexpr (chunk_k0(c) + 1 == (l + 1) * (l + 1))
              *reinterpret_cast<float2*>(srow + 4 * c + 2) = make_float2(0.0f, rpow);
            else
              srow[4 * c + 3] = rpow;
            rpow = __fmul_rn(rpow, r);
          });
        }
        if (mixed && (LPP == 1 || half == 1)) {  // r^l for the explicit |R| bound
          const float r = __fsqrt_rn(r2h);
          float rl[SH::RL4];
          rl[0] = 1.0f;
#pragma unroll
          for (int l = 1; l < SH::RL4; ++l) rl[l] = __fmul_rn(rl[l - 1], r);
#pragma unroll
          for (int c = 0; c < SH::RL4 / 4; ++c)
            *reinterpret_cast<float4*>(srow + 4 * SH::NCH + 4 * c) =
                make_float4(rl[4 * c], rl[4 * c + 1], rl[4 * c + 2], rl[4 * c + 3]);
        }
      }
      const float* tab_e = s_rad + (size_t)e * rad_elem_stride(L, NS, P.kmax);
      float* rrow = Rt + pl * SH::RSTR;
      for (int sg = sg0; sg < sg1; ++sg) {
        float R[4][L + 1];
        radial4d<L, L + 1>(tab_e, P.kmax, sg, r2h, r2l, R);
#pragma unroll
        for (int l = 0; l <= L; ++l)
          *reinterpret_cast<float4*>(rrow + l * NS + 4 * sg) = make_float4(R[0][l], R[1][l], R[2][l], R[3][l]);
      }
      if (P.want_density && half == 0) {
        const float* dens_e = s_dens + (size_t)e * dens_elem_stride(P.kmax);
        if (mixed) {
          const gmp_f2 t = density_term_df(dens_e, P.kmax, r2h, r2l, P.exp_tab);
          const gmp_f2 s2 = gmp_two_sum(rho_hi, t.hi);
          rho_hi = s2.hi;
          rho_lo = __fadd_rn(rho_lo, __fadd_rn(s2.lo, t.lo));
        } else {
          const float t = density_term(dens_e, P.kmax, r2h, r2l, nullptr);
          const gmp_f2 s2 = gmp_two_sum(rho_hi, t);
          rho_hi = s2.hi;
          rho_lo += s2.lo;
        }
      }
    }
    __syncwarp();
    // ---- phase 2: lane = (4 sigmas) x (CW components) blocks; FP32 partials
    // over FOLD pairs, folded into (hi, lo) by TwoSum
#pragma unroll
    for (int q = 0; q < SH::Q; ++q) {
      if (!it_ok[q]) continue;
      const float* rp = Rt + it_l[q] * NS + 4 * it_sb[q];
      const float* sp = St + CW * it_ch[q];
      // mixed signs, last chunk of order l: its last slot sums the bound B from |R|
      const bool mixed_last = mixed && chunk_k0_w(it_ch[q], CW) + CW >= (it_l[q] + 1) * (it_l[q] + 1);
      if constexpr (CW == 4) {
        if (mixed_last) {
          // the free slot holds 0: B from |R| r^l, r^l read after the chunks
          const float* rlp = St + 4 * SH::NCH + it_l[q];
          for (int pp = 0; pp < np; ++pp) {
            const float4 r = *reinterpret_cast<const float4*>(rp + pp * SH::RSTR);
            const float rl = rlp[pp * SH::SSTR];
            hi[q][3] = __fmaf_rn(fabsf(r.x), rl, hi[q][3]);
            hi[q][7] = __fmaf_rn(fabsf(r.y), rl, hi[q][7]);
            hi[q][11] = __fmaf_rn(fabsf(r.z), rl, hi[q][11]);
            hi[q][15] = __fmaf_rn(fabsf(r.w), rl, hi[q][15]);
          }
        }
      }
      for (int b0 = 0; b0 < np; b0 += SH::FOLD) {
        const int b1 = min(np, b0 + SH::FOLD);
        // acc2[v]: components (2h, 2h+1) of sigma u as a packed pair, v = (CW / 2) u + h
        float2 acc2[2 * CW];
#pragma unroll
        for (int v = 0; v < 2 * CW; ++v) acc2[v] = make_float2(0.0f, 0.0f);
        if constexpr (CW == 4) {
#pragma unroll 8
          for (int pp = b0; pp < b1; ++pp) {
            const float4 r = *reinterpret_cast<const float4*>(rp + pp * SH::RSTR);
            const float4 s = *reinterpret_cast<const float4*>(sp + pp * SH::SSTR);
            const float rv[4] = {r.x, r.y, r.z, r.w};
            const float2 s01 = make_float2(s.x, s.y), s23 = make_float2(s.z, s.w);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float2 ru = make_float2(rv[u], rv[u]);
              acc2[2 * u] = gmp_fma2(ru, s01, acc2[2 * u]);
              acc2[2 * u + 1] = gmp_fma2(ru, s23, acc2[2 * u + 1]);
            }
          }
        } else if (!mixed_last) {
#pragma unroll 8
          for (int pp = b0; pp < b1; ++pp) {
            const float4 r = *reinterpret_cast<const float4*>(rp + pp * SH::RSTR);
            const float2 s = *reinterpret_cast<const float2*>(sp + pp * SH::SSTR);
            const float rv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) acc2[u] = gmp_fma2(make_float2(rv[u], rv[u]), s, acc2[u]);
          }
        } else {  // the r^l slot takes |R|, so that it sums B
          for (int pp = b0; pp < b1; ++pp) {
            const float4 r = *reinterpret_cast<const float4*>(rp + pp * SH::RSTR);
            const float2 s = *reinterpret_cast<const float2*>(sp + pp * SH::SSTR);
            const float rv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              acc2[u].x = __fmaf_rn(rv[u], s.x, acc2[u].x);
              acc2[u].y = __fmaf_rn(fabsf(rv[u]), s.y, acc2[u].y);
            }
          }
        }
#pragma unroll
        for (int v = 0; v < 2 * CW; ++v) {
          float2 l2 = make_float2(lo[q][2 * v], lo[q][2 * v + 1]);
          const float2 sm = gmp_two_sum2(make_float2(hi[q][2 * v], hi[q][2 * v + 1]), acc2[v], l2);
          hi[q][2 * v] = sm.x;
          hi[q][2 * v + 1] = sm.y;
          lo[q][2 * v] = l2.x;
          lo[q][2 * v + 1] = l2.y;
        }
      }
    }
    __syncwarp();
  }
  // ---- moments to shared memory
#pragma unroll
  for (int q = 0; q < SH::Q; ++q) {
    if (!it_ok[q]) continue;
    const int l = it_l[q];
    const int kend = (l + 1) * (l + 1);
    const int kbase = chunk_k0_w(it_ch[q], CW);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < CW; ++c)
        if (kbase + c < kend)
          Mu[(4 * it_sb[q] + u) * SH::NIND + kbase + c] = __fadd_rn(hi[q][CW * u + c], lo[q][CW * u + c]);
    if (kbase + CW >= kend)  // last chunk: the last slot holds B
#pragma unroll
      for (int u = 0; u < 4; ++u)
        Mu[NS * SH::NIND + (4 * it_sb[q] + u) * (L + 1) + l] =
            __fadd_rn(hi[q][CW * u + CW - 1], lo[q][CW * u + CW - 1]);
  }
  if (mixed) mixed_sign_bound<L, NS>(P, s_rad, pairs, p0, M, Mu);
  // density: warp total (double-float with coefficients of both signs,
  // whose lane sums may cancel)
  float rho;
  if (mixed) {
    gmp_f2 t{rho_hi, rho_lo};
#pragma unroll
    for (int o = 16; o; o >>= 1)
      t = gmp_df_add(t, gmp_f2{__shfl_xor_sync(0xffffffffu, t.hi, o), __shfl_xor_sync(0xffffffffu, t.lo, o)});
    rho = __fadd_rn(t.hi, t.lo);
  } else {
    rho = __fadd_rn(rho_hi, rho_lo);
#pragma unroll
    for (int o = 16; o; o >>= 1) rho = __fadd_rn(rho, __shfl_xor_sync(0xffffffffu, rho, o));
  }
  __syncwarp();
  return __fmul_rn(rho, GMP_EXP_UNSHIFT);
}

template <int L, int NS>
__device__ __forceinline__ void setup_items(int (&it_l)[Shape<L, NS>::Q], int (&it_sb)[Shape<L, NS>::Q],
                                            int (&it_ch)[Shape<L, NS>::Q], bool (&it_ok)[Shape<L, NS>::Q]) {
  using SH = Shape<L, NS>;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < SH::Q; ++q) {
    const int item = lane + 32 * q;
    it_ok[q] = item < SH::NITEM;
    const int it = it_ok[q] ? item : 0;
    // sigma-block major within a chunk group: consecutive lanes share a chunk
    // of S values across sigma blocks -> broadcast-friendly loads
    it_sb[q] = it % SH::NSB;
    it_ch[q] = it / SH::NSB;
    it_l[q] = chunk_l_w(it_ch[q], SH::CW);
  }
}

__device__ __forceinline__ int64_t next_center(int32_t* counter) {
  int64_t c = 0;
  if ((threadIdx.x & 31) == 0) c = atomicAdd(counter, 1);
  return __shfl_sync(0xffffffffu, (int)c, 0);
}

// Features of center i from Mu; features whose value is below the FP32
// resolution bound are queued for the double-float refinement kernel.
template <int L, int NS>
__device__ __forceinline__ void write_features(const KParams& K, int64_t i, const float* Mu, float rho) {
  using SH = Shape<L, NS>;
  const GmpPass& P = K.pass;
  const int lane = threadIdx.x & 31;
  float* frow = K.features + i * P.F;
  const int nf = P.n_ord * P.nsig;
  unsigned omask = 0;  // lane o: the sigmas of order o (this pass) to refine
  for (int t0 = 0; t0 < nf; t0 += 32) {
    const int t = t0 + lane;
    const int o = t < nf ? t / P.nsig : -1, s = t - o * P.nsig;
    bool flag = false;
    if (t < nf) {
      const int l = P.ord_l[o];
      const float f = gmp_mcsh_invariant(l, Mu + s * SH::NIND + l * l);
      frow[P.ord_col[o] + s] = f;
      // Refined: the band where FP32 moments (errors of a few 2^-24 of their
      // cancellation-free scales A_c) cannot hold the relative bound.  Below
      // it the feature is so small against F_abs that its FP32 value is
      // already within the absolute floor 1e-11 F_abs: with moment errors
      // eps A_c and a computed f below t F_abs, the true f is below
      // (sqrt(t) + eps)^2 F_abs and the computed one off by at most
      // (2 sqrt(t) eps + 3 eps^2) F_abs, 6.3e-12 F_abs for t = 1e-10 and
      // eps = 3e-7 (5 units of 2^-24).  Features that vanish by symmetry
      // (perfect crystals) land there and are not refined.
      const float B = Mu[NS * SH::NIND + s * (L + 1) + l];
      const float U = __fmul_rn(flag_scale(l), __fmul_rn(B, B));  // >= F_abs
      flag = K.flags && f < __fmul_rn(K.flag_tau, U) && !(f < __fmul_rn(__fmul_rn(K.flag_low, inv_pow3(l)), U));
    }
    // the orders these 32 features belong to, each gathered into its lane
    const int o_hi = min(P.n_ord - 1, (t0 + 31) / P.nsig);
    for (int oo = t0 / P.nsig; oo <= o_hi; ++oo) {
      const unsigned m = __reduce_or_sync(0xffffffffu, (flag && o == oo) ? 1u << s : 0u);
      if (lane == oo) omask |= m;
    }
  }
  // one entry per (center, order) with flagged sigmas, in the order's own
  // queue: center << 32 | first column of the order << 16 | sigma mask.  A
  // pass has at most one entry per (center, order), and a queue holds that
  // many.
  if (lane < P.n_ord && omask) {
    const unsigned long long slot = atomicAdd(K.flag_count + lane, 1ull);
    if (slot < (unsigned long long)K.flag_cap)
      K.flags[lane * K.flag_cap + slot] =
          ((unsigned long long)i << 32) | ((unsigned long long)P.ord_col[lane] << 16) | omask;
  }
  if (P.want_density && lane == 0) frow[P.dens_col] = rho;
}

// ------------------------------------------------------------------------
template <int L, int NS, int TILE>
__global__ void __launch_bounds__(512) k_forward(KParams K) {
  using SH = Shape<L, NS, TILE>;
  extern __shared__ __align__(16) float smem[];
  const GmpPass& P = K.pass;
  float* s_rad = smem;
  float* s_dens = s_rad + (size_t)P.n_el * rad_elem_stride(L, NS, P.kmax);
  float* s_warp = s_dens + (size_t)P.n_el * dens_elem_stride(P.kmax);
  load_tables<L>(P, NS, s_rad, s_dens);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* Rt = s_warp + (size_t)wib * SH::WARP_FLOATS;
  float* St = Rt + SH::TILE * SH::RSTR;
  float* Mu = Rt;  // reused after the sweep
  int it_l[SH::Q], it_sb[SH::Q], it_ch[SH::Q];
  bool it_ok[SH::Q];
  setup_items<L, NS>(it_l, it_sb, it_ch, it_ok);
  for (int64_t i = next_center(K.counter); i < K.N; i = next_center(K.counter)) {
    const int64_t p0 = K.nbr_beg[i], p1 = K.nbr_end[i];
    if (p1 > K.pair_cap) continue;  // over capacity: flagged by the fill pass
    const int M = (int)(p1 - p0);
    const float rho = forward_sweep<L, NS, TILE>(P, s_rad, s_dens, K.pairs, p0, M, Rt, St, Mu, it_l, it_sb, it_ch,
                                                 it_ok);
    write_features<L, NS>(K, i, Mu, rho);
    if (K.mu_out) {
      float* mrow = K.mu_out + i * (int64_t)P.nsig * SH::NIND;
      for (int t = lane; t < P.nsig * SH::NIND; t += 32) mrow[t] = Mu[t];
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------
// Adjoints lam[s][k] = sum over requested orders of g_{l,s} d f_{l,s} / d mu_{l,s,k}
// into Lam (warp-private shared memory, NS rows of NINDP floats).
template <int L, int NS>
__device__ __forceinline__ void adjoints(const GmpPass& P, const float* __restrict__ Mu,
                                         const float* __restrict__ grow, float* __restrict__ Lam) {
  using SH = Shape<L, NS>;
  const int lane = threadIdx.x & 31;
  for (int t = lane; t < NS * SH::NINDP; t += 32) Lam[t] = 0.0f;
  __syncwarp();
  const int nf = P.n_ord * P.nsig;
  for (int t = lane; t < nf; t += 32) {
    const int o = t / P.nsig, s = t - o * P.nsig;
    const int l = P.ord_l[o];
    const float g = grow ? grow[P.ord_col[o] + s] : 1.0f;
    gmp_mcsh_invariant_adjoint(l, Mu + s * SH::NIND + l * l, g, Lam + s * SH::NINDP + l * l);
  }
  __syncwarp();
}

// d/dd of sum_k lam_k R(r^2) S_k(d) for one pair, from
//   A = sum_k lamd_k S_k (lamd carries dR/dr^2), B = sum_k (2l_k+1) lam_k S_k,
//   V = sum_k lam_k S_{k+e}:   grad = d (2 A + B / r^2) - V / r^2   (r^2 > 0)
// where lam already carries R.  At d = 0 only order 1 has a gradient:
// (lam_x, lam_y, lam_z).  S1 holds the MCSH values of orders 0..L+1.
template <int L>
__device__ __forceinline__ void pair_gradient(const float* lam, float A, float dx, float dy, float dz, float r2,
                                              const float* S1, float* g) {
  float B = 0.0f;
#pragma unroll
  for (int l = 0; l <= L; ++l) {
    float b = 0.0f;
#pragma unroll
    for (int k = l * l; k < (l + 1) * (l + 1); ++k) b = __fmaf_rn(lam[k], S1[k], b);
    B = __fmaf_rn((float)(2 * l + 1), b, B);
  }
  float V[3];
  GmpMcsh<L>::shift_contract(lam, S1, V);
  if (r2 > 0.0f) {
    const float inv = 1.0f / r2;
    const float c = 2.0f * A + B * inv;
    g[0] = dx * c - V[0] * inv;
    g[1] = dy * c - V[1] * inv;
    g[2] = dz * c - V[2] * inv;
  } else if (L >= 1) {
    // independent order-1 components: (0,1,0), (0,0,1), (1,0,0) at flat 1, 2, 3
    g[0] = lam[3]; g[1] = lam[1]; g[2] = lam[2];
  } else {
    g[0] = g[1] = g[2] = 0.0f;
  }
}

// ------------------------------------------------------------------------
// Backward only: moments come from the forward kernel (K.mu_out, read), the
// per-pair terms are recomputed.  Lane = pair.  With VIRIAL, also the
// strain derivative of the structure: sum over pairs of (dL/dd)_a d_b
// (positions and lattice vectors strained alike move every d to (I+eps) d),
// each lane's partial sums kept in its column of Wv ([9][32] floats of
// warp-private shared memory) rather than in registers.
// PACKED: radial factors on packed FP32 pairs (same results, fewer issue
// slots; the plain backward kernel uses them, the strain-derivative variant
// would spill at the 168 registers of the 12-warp launch).
template <int L, int NS, bool VIRIAL = false, bool PACKED = false, bool PADG = true, bool MIXED = false>
__device__ __forceinline__ void backward_sweep(const KParams& K, const float* __restrict__ s_rad,
                                               const float* __restrict__ s_dens, int64_t i, int64_t p0, int M,
                                               const float* __restrict__ Lam, float gd, float* Wv = nullptr) {
  using SH = Shape<L, NS>;
  const GmpPass& P = K.pass;
  const int lane = threadIdx.x & 31;
  float own[3] = {0.0f, 0.0f, 0.0f};
  if constexpr (VIRIAL) {
#pragma unroll
    for (int v = 0; v < 9; ++v) Wv[32 * v + lane] = 0.0f;
  }
  for (int pp = lane; pp < M; pp += 32) {
    float dx, dy, dz, r2h, r2l;
    int e, j;
    load_pair(K.pairs, p0 + pp, dx, dy, dz, r2h, r2l, e, j);
    if (pp + 32 < M) prefetch_pair(K.pairs + p0 + pp + 32);
    // MCSH values of orders 0..L first (order L+1 after the sigma loop):
    // the sigma loop then contracts them directly, so that only the
    // radial-weighted adjoints lam (not their derivative counterparts) are
    // live beside them
    const float r2c = mcsh_r2(dx, dy, dz);
    float S[SH::NIND1];
    GmpMcsh<L>::eval(dx, dy, dz, r2c, S);
    float lam[SH::NIND];
#pragma unroll
    for (int k = 0; k < SH::NIND; ++k) lam[k] = 0.0f;
    float A = 0.0f;  // sum over sigma and order of dR_l/dr^2 * sum_{k in l} Lam_k S_k
    const float* tab_e = s_rad + (size_t)e * rad_elem_stride(L, NS, P.kmax, PADG);
    for (int sg = 0; sg < SH::NSB; ++sg) {
      float R[4][L + 2];
      if constexpr (MIXED)
        radial4x<L, L + 2, PADG>(tab_e, P.kmax, sg, r2h, r2l, R);
      else if constexpr (PACKED)
        radial4p<L, L + 2, PADG>(tab_e, P.kmax, sg, r2h, R);
      else
        radial4s<L, L + 2, PADG>(tab_e, P.kmax, sg, r2h, R);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float nb = P.nbeta[4 * sg + u];
        const float* lrow = Lam + (4 * sg + u) * SH::NINDP;
        float pl[L + 1];
#pragma unroll
        for (int l = 0; l <= L; ++l) pl[l] = 0.0f;
        static_for<SH::NINDP / 4>([&](auto cq) {
          constexpr int c4 = decltype(cq)::value;
          const float4 lv4 = *reinterpret_cast<const float4*>(lrow + 4 * c4);
          const float lv[4] = {lv4.x, lv4.y, lv4.z, lv4.w};
          static_for<4>([&](auto tt) {
            constexpr int k = 4 * c4 + decltype(tt)::value;
            if constexpr (k < SH::NIND) {
              constexpr int l = order_of(k);
              lam[k] = __fmaf_rn(lv[decltype(tt)::value], R[u][l], lam[k]);
              pl[l] = __fmaf_rn(lv[decltype(tt)::value], S[k], pl[l]);
            }
          });
        });
        // dR_l/dr^2 = -beta R_{l+1}: A += -beta sum_l R_{l+1} pl_l
        float a = 0.0f;
#pragma unroll
        for (int l = 0; l <= L; ++l) a = __fmaf_rn(R[u][l + 1], pl[l], a);
        A = __fmaf_rn(nb, a, A);
      }
    }
    GmpMcsh<L + 1>::eval_top(dx, dy, dz, r2c, S);
    float g[3];
    pair_gradient<L>(lam, A, dx, dy, dz, r2c, S, g);
    // the radial factors carried 2^32
    g[0] = __fmul_rn(g[0], GMP_EXP_UNSHIFT);
    g[1] = __fmul_rn(g[1], GMP_EXP_UNSHIFT);
    g[2] = __fmul_rn(g[2], GMP_EXP_UNSHIFT);
    if (P.want_density && gd != 0.0f) {
      float drho;  // scaled by 2^32
      density_term(s_dens + (size_t)e * dens_elem_stride(P.kmax), P.kmax, r2h, r2l, &drho);
      const float c = __fmul_rn(__fmul_rn(__fmul_rn(gd, 2.0f), drho), GMP_EXP_UNSHIFT);
      g[0] = __fmaf_rn(c, dx, g[0]);
      g[1] = __fmaf_rn(c, dy, g[1]);
      g[2] = __fmaf_rn(c, dz, g[2]);
    }
    if (j != (int32_t)i) {  // images of the center itself do not move relative to it
      if (K.gbins) {
        bin_add(K.gbins + (3 * (int64_t)j + 0) * kGradBins, g[0]);
        bin_add(K.gbins + (3 * (int64_t)j + 1) * kGradBins, g[1]);
        bin_add(K.gbins + (3 * (int64_t)j + 2) * kGradBins, g[2]);
      }
      own[0] -= g[0];
      own[1] -= g[1];
      own[2] -= g[2];
    }
    if constexpr (VIRIAL) {
      const float d[3] = {dx, dy, dz};
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Wv[32 * (3 * a + b) + lane] = __fmaf_rn(g[a], d[b], Wv[32 * (3 * a + b) + lane]);
    }
  }
  if constexpr (VIRIAL) {
#pragma unroll
    for (int v = 0; v < 9; ++v) {
      double o = (double)Wv[32 * v + lane];
#pragma unroll
      for (int s = 16; s; s >>= 1) o += __shfl_xor_sync(0xffffffffu, o, s);
      if (lane == 0 && K.vir_c) K.vir_c[9 * i + v] = o;
    }
  }
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    double o = (double)own[v];
#pragma unroll
    for (int s = 16; s; s >>= 1) o += __shfl_xor_sync(0xffffffffu, o, s);
    if (lane == 0 && K.own) K.own[3 * i + v] = o;
  }
}

// Fused forward + backward for one center at a time (moments stay on chip).
template <int L, int NS>
__global__ void __launch_bounds__(256) k_vjp(KParams K) {
  using SH = Shape<L, NS>;
  extern __shared__ __align__(16) float smem[];
  const GmpPass& P = K.pass;
  float* s_rad = smem;
  float* s_dens = s_rad + (size_t)P.n_el * rad_elem_stride(L, NS, P.kmax);
  float* s_warp = s_dens + (size_t)P.n_el * dens_elem_stride(P.kmax);
  load_tables<L>(P, NS, s_rad, s_dens);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  float* Rt = s_warp + (size_t)wib * SH::WARP_FLOATS;
  float* St = Rt + SH::TILE * SH::RSTR;
  float* Mu = Rt;
  float* Lam = St;
  int it_l[SH::Q], it_sb[SH::Q], it_ch[SH::Q];
  bool it_ok[SH::Q];
  setup_items<L, NS>(it_l, it_sb, it_ch, it_ok);
  for (int64_t i = next_center(K.counter); i < K.N; i = next_center(K.counter)) {
    const int64_t p0 = K.nbr_beg[i], p1 = K.nbr_end[i];
    if (p1 > K.pair_cap) continue;  // over capacity: flagged by the fill pass
    const int M = (int)(p1 - p0);
    const float rho = forward_sweep<L, NS>(P, s_rad, s_dens, K.pairs, p0, M, Rt, St, Mu, it_l, it_sb, it_ch, it_ok);
    const float* grow = K.grad_feat + i * P.F;
    if (K.features) write_features<L, NS>(K, i, Mu, rho);
    adjoints<L, NS>(P, Mu, grow, Lam);
    const float gd = P.want_density ? grow[P.dens_col] : 0.0f;
    backward_sweep<L, NS, false, true>(K, s_rad, s_dens, i, p0, M, Lam, gd);
    __syncwarp();
  }
}

template <int L, int NS, bool VIRIAL = false, bool MIXED = false>
__global__ void __launch_bounds__(384) k_backward(KParams K) {
  using SH = Shape<L, NS>;
  extern __shared__ __align__(16) float smem[];
  const GmpPass& P = K.pass;
  // table layout by register budget: each variant with the one it keeps
  // 168 registers without spilling
  constexpr bool PADG = VIRIAL;
  float* s_rad = smem;
  float* s_dens = s_rad + (size_t)P.n_el * rad_elem_stride(L, NS, P.kmax, PADG);
  float* s_warp = s_dens + (size_t)P.n_el * dens_elem_stride(P.kmax);
  load_tables<L, PADG>(P, NS, s_rad, s_dens);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  constexpr int EXTRA = VIRIAL ? virial_extra_floats<L, NS>() : 0;
  float* Mu = s_warp + (size_t)wib * (SH::WARP_FLOATS + EXTRA);
  float* Lam = Mu + SH::TILE * SH::RSTR;
  float* Wv = EXTRA ? Mu + SH::WARP_FLOATS : Mu;  // Mu is dead once Lam is formed
  for (int64_t i = next_center(K.counter); i < K.N; i = next_center(K.counter)) {
    const int64_t p0 = K.nbr_beg[i], p1 = K.nbr_end[i];
    if (p1 > K.pair_cap) continue;  // over capacity: flagged by the fill pass
    const int M = (int)(p1 - p0);
    const float* mrow = K.mu_out + i * (int64_t)P.nsig * SH::NIND;
    for (int t = lane; t < NS * SH::NIND; t += 32) Mu[t] = (t < P.nsig * SH::NIND) ? mrow[t] : 0.0f;
    __syncwarp();
    const float* grow = K.grad_feat + i * P.F;
    adjoints<L, NS>(P, Mu, grow, Lam);
    const float gd = P.want_density ? grow[P.dens_col] : 0.0f;
    backward_sweep<L, NS, VIRIAL, !VIRIAL && !MIXED, PADG, MIXED>(K, s_rad, s_dens, i, p0, M, Lam, gd, Wv);
    __syncwarp();
  }
}

// gmp_mcsh_shift_contract_order_<l> by a compile-time order.
template <int l>
__device__ __forceinline__ void shift_contract_order(const float* lam, const float* S1, float* V) {
  if constexpr (l == 0) gmp_mcsh_shift_contract_order_0(lam, S1, V);
  else if constexpr (l == 1) gmp_mcsh_shift_contract_order_1(lam, S1, V);
  else if constexpr (l == 2) gmp_mcsh_shift_contract_order_2(lam, S1, V);
  else if constexpr (l == 3) gmp_mcsh_shift_contract_order_3(lam, S1, V);
  else if constexpr (l == 4) gmp_mcsh_shift_contract_order_4(lam, S1, V);
  else if constexpr (l == 5) gmp_mcsh_shift_contract_order_5(lam, S1, V);
  else gmp_mcsh_shift_contract_order_6(lam, S1, V);
}

// ------------------------------------------------------------------------
// Jacobian: lanes = (pair group, sigma), NS lanes per group and 32 / NS
// groups per warp.  The center's rows (distinct neighbor atoms; the pairs
// of one atom, its images, are consecutive) are split evenly among the
// groups, and each group walks the pairs of its rows with one lane per
// sigma, looping over the orders with compile-time contractions.  Per pair
//   d f_{l,s} / d d = 2 d dR_{l,s} P + R_{l,s} grad P,   P = sum_k lam_k S_k,
//   r^2 grad P = (2l+1) d P - V,  V = sum_k lam_k S_{k+e}.
// The center's own row is minus the sum over the pairs of other atoms (its
// own images do not move relative to it).  The moments come from the
// forward kernel (K.mu_out, after the double-float refinement of the
// ill-conditioned ones); K.jac_row holds each pair's row within its center.
__device__ __forceinline__ int64_t first_pair_of_row(const int32_t* __restrict__ row_of, int64_t lo, int64_t hi,
                                                    int row) {
  while (lo < hi) {  // lower bound: row_of is non-decreasing over a center's pairs
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (row_of[mid] < row) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

template <int L, int NS>
__global__ void __maxnreg__(L >= 6 ? 168 : 128) k_jacobian(KParams K) {
  using SH = Shape<L, NS>;
  constexpr int G = 32 / NS;  // pair groups per warp
  constexpr int NO = L + 1;   // at most L + 1 orders >= 0 per pass
  extern __shared__ __align__(16) float smem[];
  const GmpPass& P = K.pass;
  // unpadded table: the padded group stride took the order-6 kernel from
  // 165 to 169 registers, two resident 4-warp CTAs per SM instead of three
  float* s_rad = smem;
  float* s_dens = s_rad + (size_t)P.n_el * rad_elem_stride(L, NS, P.kmax, false);
  float* s_warp = s_dens + (size_t)P.n_el * dens_elem_stride(P.kmax);
  load_tables<L, false>(P, NS, s_rad, s_dens);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int pg = lane / NS, s = lane % NS;
  const bool s_ok = s < P.nsig;
  const bool dens_lane = P.want_density && s == 0;
  const float nb = P.nbeta[s];
  float* Mu = s_warp + (size_t)wib * SH::WARP_FLOATS;
  float* Lam = Mu + SH::TILE * SH::RSTR;
  const float* lam_s = Lam + s * SH::NINDP;
  for (int64_t i = next_center(K.counter); i < K.N; i = next_center(K.counter)) {
    const int64_t p0 = K.nbr_beg[i], p1 = K.nbr_end[i];
    if (p1 > K.pair_cap) continue;  // over capacity: flagged by the fill pass
    const float* mrow = K.mu_out + i * (int64_t)P.nsig * SH::NIND;
    for (int t = lane; t < NS * SH::NIND; t += 32) Mu[t] = (t < P.nsig * SH::NIND) ? mrow[t] : 0.0f;
    __syncwarp();
    adjoints<L, NS>(P, Mu, nullptr, Lam);  // g = 1 per feature: lam = d f / d mu
    // Exponent offset of this lane's radial factors (its sigma, this
    // center): the largest S (at most 90, at least 32) that keeps the scaled
    // intermediates below 2^126.  They are bounded by 2^S max|lam_s|
    // 2^jac_exp[s] max(1, beta_s) 2^32 (jac_exp: the radial factors times
    // max(1, r)^(L+1); MCSH values up to 2^15 r^(L+1) at order 7, 2l+1 terms
    // and factors, 1/r^2 up to 2^8, the sums).  Large adjoints lift a far
    // pair's row above 2^-126 even when its exponentials lie below 2^-158
    // (the fixed offset of 32 alone).
    float lm = 0.0f;
    for (int t = 0; t < SH::NIND; ++t) lm = fmaxf(lm, fabsf(lam_s[t]));
    const int le = ((__float_as_int(lm) >> 23) & 255) - 126;                 // > log2(lm)
    const int lb = max(0, ((__float_as_int(-nb) >> 23) & 255) - 126);       // >= log2(beta)
    const int Si = max(32, min(90, 94 - le - lb - P.jac_exp[s]));
    const float shift = (float)Si;  // 2^-S is formed where a row is written
    auto unshift_of = [](float s) { return __int_as_float((127 - (int)s) << 23); };
    const int64_t r0 = K.jac_off[i - K.center0];
    const int R = (int)(K.jac_off[i - K.center0 + 1] - r0);
    // the center's own row: the rank of atom i among its neighbor atoms
    int64_t lo = p0, hi = p1;
    while (lo < hi) {
      const int64_t mid = lo + ((hi - lo) >> 1);
      if (K.pairs[mid].j < (int32_t)i) lo = mid + 1;
      else hi = mid;
    }
    // (the self pair, j = i with no shift, is always in the list)
    const int r_self = (lo < p1 && K.pairs[lo].j == (int32_t)i) ? K.jac_row[lo] : -1;
    // this group's rows [ra, rb) and their pairs [pa, pb)
    const int ra = (int)((int64_t)R * pg / G), rb = (int)((int64_t)R * (pg + 1) / G);
    const int64_t pa = first_pair_of_row(K.jac_row, p0, p1, ra);
    const int64_t pb = first_pair_of_row(K.jac_row, pa, p1, rb);
    float acc[NO][3], self[NO][3], dacc[3] = {0.0f, 0.0f, 0.0f}, dself[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int o = 0; o < NO; ++o)
#pragma unroll
      for (int v = 0; v < 3; ++v) { acc[o][v] = 0.0f; self[o][v] = 0.0f; }
    int cur = -1;  // row being accumulated
    auto flush = [&]() {
      if (cur < 0 || cur == r_self) return;  // the own row is written below
      const int64_t row = r0 + cur;
      if (s_ok) {
        static_for<NO>([&](auto oo) {
          constexpr int o = decltype(oo)::value;
          if (o < P.n_ord) {
            float* dst = K.jac + (row * P.F + P.ord_col[o] + s) * 3;
            const float unshift = unshift_of(shift);
            dst[0] = acc[o][0] * unshift;
            dst[1] = acc[o][1] * unshift;
            dst[2] = acc[o][2] * unshift;
          }
        });
      }
      if (dens_lane) {
        float* dst = K.jac + (row * P.F + P.dens_col) * 3;
        dst[0] = dacc[0] * GMP_EXP_UNSHIFT;
        dst[1] = dacc[1] * GMP_EXP_UNSHIFT;
        dst[2] = dacc[2] * GMP_EXP_UNSHIFT;
      }
    };
    for (int64_t p = pa; p < pb; ++p) {
      // the group walks its pairs one at a time: pull the record four ahead
      // (the next 128-byte line) and the row ranks 32 ahead into L1
      if (p + 4 < pb) prefetch_pair(K.pairs + p + 4);
      if (((p - pa) & 31) == 0 && p + 32 < pb) prefetch_l1(K.jac_row + p + 32);
      float dx, dy, dz, r2h, r2l;
      int e, j;
      load_pair(K.pairs, p, dx, dy, dz, r2h, r2l, e, j);
      const int row = K.jac_row[p];
      if (row != cur) {
        flush();
#pragma unroll
        for (int o = 0; o < NO; ++o) acc[o][0] = acc[o][1] = acc[o][2] = 0.0f;
        dacc[0] = dacc[1] = dacc[2] = 0.0f;
        if (s == 0) K.jac_j[r0 + row] = j;
        cur = row;
      }
      const bool other = j != (int32_t)i;
      if (s_ok) {
        float S1[SH::NIND1];
        const float r2c = mcsh_r2(dx, dy, dz);
        GmpMcsh<L + 1>::eval(dx, dy, dz, r2c, S1);
        // radial factors of this lane's sigma, orders 0..L+1, scaled by 2^S
        // (double-float exponent argument: a row of one neighbor averages no
        // other terms)
        float Rl[L + 2];
#pragma unroll
        for (int l = 0; l < L + 2; ++l) Rl[l] = 0.0f;
        const float* tab_e = s_rad + (size_t)e * rad_elem_stride(L, NS, P.kmax, false);
        for (int q = 0; q < P.kmax; ++q) {
          const float* ent = tab_e + ((s / 4) * P.kmax + q) * gmp_rad_block(L) * 4 + (s % 4);
          const float E = gmp_exp_neg_shifted_by(ent[0], ent[4], r2h, r2l, shift);
#pragma unroll
          for (int l = 0; l < L + 2; ++l) Rl[l] = __fmaf_rn(ent[4 * (2 + l)], E, Rl[l]);
        }
        const float inv = r2c > 0.0f ? 1.0f / r2c : 0.0f;
        // d f_{lc,s} / d d of this pair for a compile-time order lc
        auto order_term = [&](auto ll, float (&g)[3]) {
          constexpr int lc = decltype(ll)::value;
          float pv = 0.0f, V[3];
#pragma unroll
          for (int k = lc * lc; k < (lc + 1) * (lc + 1); ++k) pv = __fmaf_rn(lam_s[k], S1[k], pv);
          shift_contract_order<lc>(lam_s, S1, V);
          const float Rv = Rl[lc], Rd = nb * Rl[lc + 1];  // dR_l/dr^2 = -beta R_{l+1}
          if (r2c > 0.0f) {
            const float c = 2.0f * Rd * pv + Rv * (float)(2 * lc + 1) * pv * inv;
            g[0] = dx * c - Rv * V[0] * inv;
            g[1] = dy * c - Rv * V[1] * inv;
            g[2] = dz * c - Rv * V[2] * inv;
          } else if (lc == 1) {  // d = 0: only order 1 has a gradient
            g[0] = Rv * lam_s[3]; g[1] = Rv * lam_s[1]; g[2] = Rv * lam_s[2];
          }
        };
        auto accumulate = [&](int o, const float (&g)[3]) {
          acc[o][0] += g[0]; acc[o][1] += g[1]; acc[o][2] += g[2];
          if (other) { self[o][0] -= g[0]; self[o][1] -= g[1]; self[o][2] -= g[2]; }
        };
        if (P.ord_dense) {  // orders 0, 1, ... in order: one block per order
          static_for<NO>([&](auto oo) {
            constexpr int o = decltype(oo)::value;
            if (o < P.n_ord) {
              float g[3] = {0.0f, 0.0f, 0.0f};
              order_term(oo, g);
              accumulate(o, g);
            }
          });
        } else {
          static_for<NO>([&](auto oo) {
            constexpr int o = decltype(oo)::value;
            if (o < P.n_ord) {
              const int l = P.ord_l[o];
              float g[3] = {0.0f, 0.0f, 0.0f};
              static_for<L + 1>([&](auto ll) {
                if (l == decltype(ll)::value) order_term(ll, g);
              });
              accumulate(o, g);
            }
          });
        }
      }
      if (dens_lane) {
        float drho;
        density_term(s_dens + (size_t)e * dens_elem_stride(P.kmax), P.kmax, r2h, r2l, &drho);
        const float g[3] = {2.0f * drho * dx, 2.0f * drho * dy, 2.0f * drho * dz};
        dacc[0] += g[0]; dacc[1] += g[1]; dacc[2] += g[2];
        if (other) { dself[0] -= g[0]; dself[1] -= g[1]; dself[2] -= g[2]; }
      }
    }
    flush();
    // own row: the groups' sums of minus the other atoms' terms
#pragma unroll
    for (int o = 0; o < NO; ++o)
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int k = NS; k < 32; k <<= 1) self[o][v] += __shfl_xor_sync(0xffffffffu, self[o][v], k);
#pragma unroll
    for (int v = 0; v < 3; ++v)
#pragma unroll
      for (int k = NS; k < 32; k <<= 1) dself[v] += __shfl_xor_sync(0xffffffffu, dself[v], k);
    if (pg == 0 && r_self >= 0) {
      const int64_t row = r0 + r_self;
      if (s_ok) {
        static_for<NO>([&](auto oo) {
          constexpr int o = decltype(oo)::value;
          if (o < P.n_ord) {
            float* dst = K.jac + (row * P.F + P.ord_col[o] + s) * 3;
            const float unshift = unshift_of(shift);
            dst[0] = self[o][0] * unshift;
            dst[1] = self[o][1] * unshift;
            dst[2] = self[o][2] * unshift;
          }
        });
      }
      if (dens_lane) {
        float* dst = K.jac + (row * P.F + P.dens_col) * 3;
        dst[0] = dself[0] * GMP_EXP_UNSHIFT;
        dst[1] = dself[1] * GMP_EXP_UNSHIFT;
        dst[2] = dself[2] * GMP_EXP_UNSHIFT;
      }
    }
    __syncwarp();
  }
}

}  // namespace gmpk
