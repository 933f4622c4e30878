// Internal declarations shared by the libgmp translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define GMP_WARP 32
#define GMP_MAX_SIGMAS 16      // sigmas per kernel pass (host splits larger sets)
#define GMP_TILE 32            // neighbor pairs staged per warp tile

// Device error word bits (OR-ed by kernels, read by the host after a call).
#define GMP_DEV_BAD_SPECIES 1u
#define GMP_DEV_NONFINITE 2u
#define GMP_DEV_TOO_MANY_NEIGHBORS 4u
#define GMP_DEV_SHIFT_RANGE 8u
#define GMP_DEV_CAPACITY 16u

struct __align__(32) GmpD4 {
  double x, y, z, w;
};

// Per-structure geometry used by binning and neighbor search (host-built).
struct GmpStruct {
  double A[9];        // lattice vectors as rows (identity frame when no axis is periodic)
  double Ainv[9];     // inverse: frac = x . Ainv (u_k = sum_c x_c Ainv[c*3+k])
  float Ahi[9], Alo[9];  // double-float split of A
  double reach[3];    // cutoff * |b_k| in fractional units (b_k = column k of Ainv)
  int periodic[3];
  int64_t atom_base;  // first atom
  int32_t n_atoms;
  int32_t pad0;
  int64_t bin_base;   // first bin slot of this structure
  int32_t bin_cap;    // bin slots reserved
  int32_t pad1;
  float prescreen2;   // FP32 r^2 above this: certainly outside the cutoff (see neighbors.cu)
  float inside2;      // FP32 r^2 below this: certainly inside the cutoff
  float pad2[2];
};

// Per-structure bin grid (device-built from bounding boxes).
struct GmpGrid {
  double umin[3];     // fractional coordinate of bin 0 edge
  double binw[3];     // bin width (fractional)
  double inv_binw[3]; // 1 / binw
  int nb[3];          // bins per axis
  int pad;
};

// One neighbor image of a center, 32 bytes.
struct __align__(16) GmpPair {
  float dx, dy, dz, r2hi;   // displacement x_j + shift - x_i (FP32), r^2 high part
  float r2lo;               // r^2 = r2hi + r2lo (double-float)
  int32_t e;                // species of j
  int32_t j;                // neighbor atom (global index)
  int32_t shift;            // packed image n: (n1+512) | (n2+512)<<10 | (n3+512)<<20
};

__host__ __device__ inline int32_t gmp_pack_shift(int n1, int n2, int n3) {
  return (n1 + 512) | ((n2 + 512) << 10) | ((n3 + 512) << 20);
}
__host__ __device__ inline void gmp_unpack_shift(int32_t s, int* n) {
  n[0] = (s & 1023) - 512;
  n[1] = ((s >> 10) & 1023) - 512;
  n[2] = ((s >> 20) & 1023) - 512;
}

// Radial table block per (element, group of 4 sigmas, primitive): L + 4
// float4s, each holding one quantity for the 4 sigmas of the group, so one
// 16-byte shared-memory load serves four sigmas:
//   [0] Bhi, [1] Blo : B = alpha*beta/gamma * log2(e) as a double-float
//   [2 + l] A_l      : c * N_sigma * (pi/gamma)^(3/2) * (alpha/gamma)^l, l = 0..L+1
// Blocks are ordered [element][sigma group][primitive].  Order L+1 serves
// the derivative: since the exponent rate is alpha*beta/gamma = beta *
// (alpha/gamma), d R_l / d r^2 = -beta R_{l+1} exactly.
__host__ __device__ constexpr int gmp_rad_block(int L) { return L + 4; }
// Density table entry per (element, primitive): Bhi, Blo, b, c, b_lo, c_lo, 0, 0
// with B = alpha*log2(e) split into (hi, lo), b = alpha and c rounded to FP32
// and their rounding errors b_lo, c_lo (the double-float density of tables
// with coefficients of both signs).
#define GMP_DENS_STRIDE 8

// Shapes of one forward/backward pass.
struct GmpPass {
  int lmax;            // highest non-negative order computed
  int nsig;            // sigmas in this pass (<= 16)
  int nsig_pad;        // 4, 8 or 16
  int kmax;            // primitives per element (padded)
  int n_el;
  int want_density;    // order -1 requested
  int mixed_sign;      // some density coefficient is negative (radial factors may be < 0)
  int F;               // total feature columns
  int n_ord;           // number of orders >= 0 written by this pass
  int ord_l[8];        // orders written
  int ord_col[8];      // feature column of (order, sigma 0) for this pass
  int dens_col;        // column of order -1 or -1
  int ord_dense;       // 1 when ord_l[o] == o for every o (orders 0 .. n_ord-1 in order)
  const float* rad;    // [n_el][nsig_pad / 4][kmax][gmp_rad_block(lmax)] float4
  float nbeta[16];     // -beta = -1/(2 sigma^2) per sigma of the pass (0 for padding)
  const float* dens;   // [n_el][kmax][GMP_DENS_STRIDE]: alpha log2(e) (hi, lo),
                       // alpha, c, alpha's and c's low words, 0, 0
  const float2* exp_tab;  // [64] 2^(-j/64) as double-floats (gmp_df_exp_neg)
  // per sigma of the pass: ceil(log2) of the largest, over elements, of
  // sum_q max_{0 <= r <= cutoff} |A_{0,q,s}| exp(-B_{q,s} r^2) max(1, r)^(lmax+1)
  // (a bound on |R_{l,s}(r)| max(1, r)^(lmax+1), orders 0..lmax+1): with the
  // adjoints' size it bounds the Jacobian kernel's intermediates (its
  // exponent offset per center and sigma)
  int jac_exp[16];
};

// ---------------------------------------------------------------- double-float
struct gmp_f2 {
  float hi, lo;
};

__device__ __forceinline__ gmp_f2 gmp_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ gmp_f2 gmp_fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ gmp_f2 gmp_two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
// Accurate double-float addition (two TwoSums, two renormalisations).
__device__ __forceinline__ gmp_f2 gmp_df_add(gmp_f2 a, gmp_f2 b) {
  gmp_f2 s = gmp_two_sum(a.hi, b.hi);
  gmp_f2 t = gmp_two_sum(a.lo, b.lo);
  float e = __fadd_rn(s.lo, t.hi);
  gmp_f2 u = gmp_fast_two_sum(s.hi, e);
  e = __fadd_rn(t.lo, u.lo);
  return gmp_fast_two_sum(u.hi, e);
}
__device__ __forceinline__ gmp_f2 gmp_df_neg(gmp_f2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ gmp_f2 gmp_df_mul(gmp_f2 a, gmp_f2 b) {
  gmp_f2 p = gmp_two_prod(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return gmp_fast_two_sum(p.hi, e);
}
// Double-float times a float.
__device__ __forceinline__ gmp_f2 gmp_df_mul_f(gmp_f2 a, float b) {
  gmp_f2 p = gmp_two_prod(a.hi, b);
  float e = __fmaf_rn(a.lo, b, p.lo);
  return gmp_fast_two_sum(p.hi, e);
}
// Addition where |a| >= |b| is not required but the result's low word is
// the plain sum of the rounding errors (one renormalisation): enough for a
// Horner step whose terms decrease.
__device__ __forceinline__ gmp_f2 gmp_df_add_sloppy(gmp_f2 a, gmp_f2 b) {
  gmp_f2 s = gmp_two_sum(a.hi, b.hi);
  return gmp_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

// Integer (|n| < 2^24) times double-float, exact product of the high part.
__device__ __forceinline__ gmp_f2 gmp_df_mul_int(int n, gmp_f2 a) {
  float fn = (float)n;
  gmp_f2 p = gmp_two_prod(fn, a.hi);
  float e = __fmaf_rn(fn, a.lo, p.lo);
  return gmp_fast_two_sum(p.hi, e);
}

// 2^x on the SFU (PTX ex2.approx.ftz.f32): about 2 ulp, flushes tiny results to 0.
__device__ __forceinline__ float gmp_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Packed FP32 pairs: on the sm_100 family one instruction performs the
// operation for both lanes of a float2, rounded to nearest exactly like
// the scalar __fmaf_rn / __fadd_rn / __fmul_rn, while taking one issue slot.
__device__ __forceinline__ float2 gmp_fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 gmp_mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 gmp_add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// TwoSum on packed pairs: returns a + b rounded and adds its exact rounding
// error to lo (the operations of gmp_two_sum per lane; x - y as x + (-1) y,
// which rounds once like the subtraction).
__device__ __forceinline__ float2 gmp_two_sum2(float2 a, float2 b, float2& lo) {
  const float2 m1 = make_float2(-1.0f, -1.0f);
  const float2 s = gmp_add2(a, b);
  const float2 bb = gmp_fma2(a, m1, s);
  const float2 e = gmp_add2(gmp_fma2(gmp_fma2(bb, m1, s), m1, a), gmp_fma2(bb, m1, b));
  lo = gmp_add2(lo, e);
  return s;
}

// Two exponentials exp(-B r^2) (B of two sigmas, one pair's r^2), with the
// operations of gmp_exp_neg below in packed form: bit-identical results.
// nr2h = -r2hi in both lanes, r2h = r2hi, r2l = r2lo in both lanes.
__device__ __forceinline__ float2 gmp_exp_neg2(float2 Bhi, float2 Blo, float2 nr2h, float2 r2h, float2 r2l) {
  const float2 nxh = gmp_mul2(Bhi, nr2h);        // -(Bhi r2hi), rounded as the scalar product
  float2 xl = gmp_fma2(Bhi, r2h, nxh);
  xl = gmp_fma2(Bhi, r2l, xl);
  xl = gmp_fma2(Blo, r2h, xl);
  const float2 E = make_float2(gmp_ex2(nxh.x), gmp_ex2(nxh.y));
  return gmp_fma2(E, gmp_mul2(make_float2(-0.69314718055994531f, -0.69314718055994531f), xl), E);
}

// exp(-B r^2) with B and r^2 given as double-floats: the product is formed
// to about 2^-44 relative, the SFU takes its high part and the low part is
// applied to first order, exp2(-(h+l)) = exp2(-h) (1 - ln2 l).
__device__ __forceinline__ float gmp_exp_neg(float Bhi, float Blo, float r2hi, float r2lo) {
  float xh = __fmul_rn(Bhi, r2hi);
  float xl = __fmaf_rn(Bhi, r2hi, -xh);
  xl = __fmaf_rn(Bhi, r2lo, xl);
  xl = __fmaf_rn(Blo, r2hi, xl);
  float E = gmp_ex2(-xh);
  return __fmaf_rn(E, -0.69314718055994531f * xl, E);
}

// 2^32 exp(-B r^2), for the dense Jacobian rows.  A row there holds the
// terms of one neighbor atom alone, multiplied by adjoints that can be large,
// so a radial factor that is subnormal in FP32 (few significant bits) or
// flushed to zero by the SFU would show in the row.  Offsetting the exponent
// by 32 keeps the factor normal down to exp(-B r^2) = 2^-158; the kernel
// scales its sums back by 2^-32 when it writes them.  32 - xh is rounded
// only when xh < 16, and there Fast2Sum (|32| >= |xh|) recovers its rounding
// error exactly; for xh >= 16 the difference is exact and the recovered
// error is 0.  The error joins the low part of the argument.
#define GMP_EXP_SHIFT 32.0f
#define GMP_EXP_UNSHIFT 0x1p-32f
// 2^S exp(-B r^2) for an integer S in 0..126 (the same steps: S - xh is
// rounded only when xh < S, where Fast2Sum applies; beyond it the
// difference is exact).
__device__ __forceinline__ float gmp_exp_neg_shifted_by(float Bhi, float Blo, float r2hi, float r2lo, float S) {
  float xh = __fmul_rn(Bhi, r2hi);
  float xl = __fmaf_rn(Bhi, r2hi, -xh);
  xl = __fmaf_rn(Bhi, r2lo, xl);
  xl = __fmaf_rn(Blo, r2hi, xl);
  const float d = __fadd_rn(S, -xh);
  const float e = __fadd_rn(__fadd_rn(S, -d), -xh);  // (S - xh) - d, exactly
  const float E = gmp_ex2(d);
  return __fmaf_rn(E, -0.69314718055994531f * __fadd_rn(xl, -e), E);
}
__device__ __forceinline__ float gmp_exp_neg_shifted(float Bhi, float Blo, float r2hi, float r2lo) {
  return gmp_exp_neg_shifted_by(Bhi, Blo, r2hi, r2lo, GMP_EXP_SHIFT);
}

// exp(-x) for a double-float x to about 1e-13 relative, in FP32
// arithmetic, by table-driven reduction (Tang's method):
// x = k ln2/64 + r with |r| <= ln2/128 (ln2/64 as a double-float), so that
// exp(-x) = 2^-(k div 64) * 2^-((k mod 64)/64) * exp(-r); the middle factor
// is a double-float table entry (tab[j] = 2^(-j/64)) and
// exp(-r) = 1 - r + r^2 w, w = 1/2 + r t, t = -1/6 + r/24 - r^2/120, where
// |r t| < 1e-3 lets t be FP32 (the omitted r^6/720 term is below 3e-17).
// Results below the FP32 normal range (x > 87) are returned as 0.  A
// negative x (down to about -88) works the same way: k and its shift by 6
// are then negative, the table index k mod 64 stays in 0..63.
__device__ __forceinline__ gmp_f2 gmp_df_exp_neg(gmp_f2 x, const float2* __restrict__ tab) {
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

// Double-float displacement of j's image n from i, and its r^2.
__device__ __forceinline__ void gmp_df_disp(const float4& xhi, const float4& xli, const float4& xhj,
                                        const float4& xlj, const GmpStruct& st, const int* n,
                                        gmp_f2* d, gmp_f2& r2, float& mag) {
  const float xi_h[3] = {xhi.x, xhi.y, xhi.z}, xi_l[3] = {xli.x, xli.y, xli.z};
  const float xj_h[3] = {xhj.x, xhj.y, xhj.z}, xj_l[3] = {xlj.x, xlj.y, xlj.z};
  const bool shifted = (n[0] | n[1] | n[2]) != 0;
  mag = 0.0f;
  for (int c = 0; c < 3; ++c) {
    gmp_f2 dd = gmp_df_add(gmp_f2{xj_h[c], xj_l[c]}, gmp_f2{-xi_h[c], -xi_l[c]});
    float m = fabsf(xj_h[c]) + fabsf(xi_h[c]);
    if (shifted) {
      gmp_f2 s0 = gmp_df_mul_int(n[0], gmp_f2{st.Ahi[c], st.Alo[c]});
      gmp_f2 s1 = gmp_df_mul_int(n[1], gmp_f2{st.Ahi[3 + c], st.Alo[3 + c]});
      gmp_f2 s2 = gmp_df_mul_int(n[2], gmp_f2{st.Ahi[6 + c], st.Alo[6 + c]});
      gmp_f2 sh = gmp_df_add(gmp_df_add(s0, s1), s2);
      dd = gmp_df_add(dd, sh);
      m += fabsf(s0.hi) + fabsf(s1.hi) + fabsf(s2.hi);
    }
    d[c] = dd;
    mag = fmaxf(mag, m);
  }
  r2 = gmp_df_add(gmp_df_add(gmp_df_mul(d[0], d[0]), gmp_df_mul(d[1], d[1])), gmp_df_mul(d[2], d[2]));
}

// ---------------------------------------------------------------- host side
struct GmpWorkspace;

// Launchers implemented in the .cu files (all asynchronous on `stream`).
// Binning of a small batch (at most kSmallBinAtoms atoms, 256 structures)
// in one launch of one CTA: the outputs of gmp_launch_neighbors_prepare +
// gmp_launch_bins (atom_xh/xl/u/bin/rng/y, grid, pre-screen bounds,
// bin_start/bin_y/bin_je), bit for bit.  gmp_bin_small_fits says whether
// a batch qualifies (shared memory for its bins and slots).
// One SM runs the batch's FP64 set-up (GB300: 1/64 of the FP32 rate), so
// the single CTA wins only for small batches: on a GB300, 64 atoms took
// 0.054 ms against 0.088 for the multi-kernel path, 4096 atoms 0.34 against
// 0.17.
constexpr int64_t kSmallBinAtoms = 1024;
bool gmp_bin_small_fits(int64_t N, int64_t n_bins, int n_struct);
cudaError_t gmp_launch_bin_small(GmpStruct* d_structs, int n_struct, const int32_t* d_struct_of, int64_t N,
                                 double cutoff, const double* pos, const int32_t* species, int n_el,
                                 GmpGrid* d_grid, int64_t n_bins, float4* atom_xh, float4* atom_xl, GmpD4* atom_u,
                                 int32_t* atom_bin, int32_t* bin_start, float4* bin_y, int2* bin_je,
                                 int4* atom_rng, float4* atom_y, uint32_t* d_err, cudaStream_t stream,
                                 int64_t* launches);
cudaError_t gmp_launch_neighbors_prepare(const GmpStruct* d_structs, int n_struct,
                                         const int32_t* d_struct_of, int64_t N, double cutoff,
                                         const double* pos, const int32_t* species, int n_el,
                                         GmpGrid* d_grid, float4* atom_xh, float4* atom_xl,
                                         GmpD4* atom_u, int32_t* atom_bin,
                                         unsigned long long* d_bbox, uint32_t* d_err,
                                         cudaStream_t stream, int sm_count, int64_t* launches);
cudaError_t gmp_launch_bins(const GmpStruct* d_structs, const GmpGrid* d_grid,
                            const int32_t* d_struct_of, int64_t N, int64_t n_bins,
                            const int32_t* atom_bin, int32_t* bin_count, int32_t* bin_start,
                            int32_t* bin_cursor, int4* atom_rng, float4* atom_y, float4* bin_y, int2* bin_je,
                            const GmpD4* atom_u, const float4* atom_xh, const float4* atom_xl, void* scan_tmp,
                            size_t scan_tmp_bytes, cudaStream_t stream, int sm_count, int64_t* launches);
size_t gmp_scan_tmp_bytes(int64_t n);
cudaError_t gmp_exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* tmp,
                                   cudaStream_t stream, int64_t* launches);
// The points that neighbor lists are built around: the atoms themselves or
// reference points (gmp_featurize_points).  Per center: structure id, FP64
// position [3], double-float split (xl.w = packed wrap of the fractional
// coordinates), scanned bin range and wrapped FP32 position (k_ranges).
struct GmpCenters {
  const int32_t* sid;
  const double* pos;
  const float4* xh;
  const float4* xl;
  const int4* rng;
  const float4* y;
};
// Per reference point: the GmpCenters fields above from its FP64 position
// and structure (after the atom grid of each structure is built); atom_pos
// gives each structure's reference cell (that of its first atom).
cudaError_t gmp_launch_point_prepare(const GmpStruct* d_structs, const GmpGrid* d_grid,
                                     const int32_t* point_struct, int64_t n_points, const double* points,
                                     const double* atom_pos, float4* pt_xh, float4* pt_xl, int4* pt_rng,
                                     float4* pt_y, uint32_t* d_err, cudaStream_t stream, int sm_count,
                                     int64_t* launches);
// fill: 0 = count only, 1 = records grouped by species (deterministic),
// 2 = records sorted by (neighbor atom, image).  Centers C [N]; neighbors
// are the binned atoms (pos, atom_xh, atom_xl).  Records go to the CSR
// offsets (from a count pass), or, with cursor (fill 1 or 2), to blocks
// allocated from *cursor whose ranges are written to rng[i], rng[N + i].
// Over-capacity blocks set GMP_DEV_CAPACITY.
cudaError_t gmp_launch_neighbor_pass(int fill, const GmpStruct* d_structs, const GmpGrid* d_grid,
                                     const GmpCenters& C, int64_t N, double cutoff,
                                     const double* pos, const float4* atom_xh, const float4* atom_xl,
                                     const int32_t* bin_start, const float4* bin_y, const int2* bin_je, int n_el,
                                     int64_t* counts, const int64_t* offsets,
                                     GmpPair* pairs, int64_t pair_cap, int max_keys, int32_t* d_maxm,
                                     uint32_t* d_err, cudaStream_t stream, int sm_count, int64_t* launches,
                                     unsigned long long* cursor = nullptr, int64_t* rng = nullptr);
// Distinct neighbor atoms per center (counts [N]) and each pair's row
// among them (local_row [P]); center i's pairs are [nbr_beg[i], nbr_end[i]),
// sorted by atom.
cudaError_t gmp_launch_jacobian_count(int64_t N, const int64_t* nbr_beg, const int64_t* nbr_end, const GmpPair* pairs,
                                      int64_t* counts, int32_t* local_row, cudaStream_t stream, int sm_count,
                                      int64_t* launches);
cudaError_t gmp_launch_grad_finish(int64_t N, const double* grad_acc, float* grad_pos,
                                   cudaStream_t stream, int64_t* launches);
// grad_acc[j] += own[j] + the value of j's exact fixed-point bins (filled by
// the backward kernels without float atomics; 12 per atom and component).
cudaError_t gmp_launch_grad_bins_finish(int64_t N, const unsigned long long* bins, const double* own,
                                        double* grad_acc, cudaStream_t stream, int sm_count, int64_t* launches);
// virial[s] += sum of vir_c over the centers atom_off[s] .. atom_off[s+1]-1 (fixed order).
cudaError_t gmp_launch_virial_reduce(int n_struct, const int64_t* atom_off, const double* vir_c, double* virial,
                                     cudaStream_t stream, int sm_count, int64_t* launches);
// Double-float recomputation of the flagged features: one queue per
// order slot o (queue + o * cap, count[o] entries, at most cap; qidx[l] is
// the slot of order l, -1 when l is not requested), entries center << 32 |
// first column of the order << 16 | mask of its flagged sigmas;
// col_info[col] = (order << 16) | sigma.  With mu_out, the
// recomputed moments of sigmas mu_sig0 .. mu_sig0 + mu_nsig - 1 also
// overwrite mu_out[center][sigma - mu_sig0][l^2 .. l^2 + 2l] (row length
// mu_nind), the moments a derivative kernel reads next.
struct GmpRefine {
  const unsigned long long* queue;
  const unsigned long long* count;
  int64_t cap;
  int qidx[7];
  int64_t n_centers;
  const int32_t* col_info;
  float* features;
  int F;
  const float4* atom_xh;
  const float4* atom_xl;
  const float4* center_xh;
  const float4* center_xl;
  const int32_t* center_struct;
  const GmpStruct* structs;
  const int64_t* nbr_beg;
  const int64_t* nbr_end;
  const GmpPair* pairs;
  const float* ktab;
  const float2* exp_tab;  // [64] 2^(-j/64) as double-floats
  int nsig_total;
  int kmax;
  float* mu_out;
  int mu_sig0, mu_nsig, mu_nind;
};
// One launch per order set in order_mask (bit l: order l >= 0 requested).
cudaError_t gmp_launch_refine(const GmpRefine& args, unsigned order_mask, int sm_count, cudaStream_t stream,
                              int64_t* launches);
cudaError_t gmp_launch_unpack_neighbors(int64_t P, const GmpPair* pairs, int32_t* nbr_j,
                                        int32_t* nbr_shift, cudaStream_t stream,
                                        int64_t* launches);
