// Cell-list binning and exact neighbor images on the GPU.
//
// Neighbor set (GMP-Featurizer, Statement of Needs / Overview: molecules,
// clusters and periodic crystals given lattice vectors and positions): all
// (j, n in Z^3, n_k = 0 on non-periodic axes) with
//   d = (x_j - x_i) + ((n1 a1 + n2 a2) + n3 a3),   dx*dx + dy*dy + dz*dz < rc*rc
// where the expression is FP64, evaluated left to right without FMA.  The
// GPU reaches the same decision with far less FP64 work:
//   1. atoms are binned on a grid in (wrapped) fractional coordinates;
//   2. a center scans the bins that its cutoff sphere can touch (periodic
//      axes wrap, giving an image index m); each candidate is pre-screened
//      in FP32 against a rigorous bound on the FP32 error;
//   3. survivors get d and r^2 in double-float arithmetic (about 2^-44
//      relative), which decides every case except a shell of relative width
//      ~1e-9 around rc^2; inside that shell the FP64 expression above is
//      evaluated exactly as written, so the set equals the FP64 one;
//   4. each center's accepted (j, n) records are written in a fixed order,
//      which makes every later sum over a center's neighbors deterministic:
//      grouped by neighbor species, enumeration order within a species
//      (the feature kernels then read the same table rows across a tile),
//      or sorted by (j, n) for the Jacobian and the neighbor-list output.
#include "gmp_internal.cuh"

#include <math.h>

namespace {

__device__ __forceinline__ unsigned long long order_key(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_to_double(unsigned long long k) {
  unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)b);
}

__device__ __forceinline__ int floor_div(int a, int b) {  // b > 0
  int q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// floor(a / b) for |a| < 2^20 and 1 <= b < 2^24 (both exact in FP32)
// without an integer division: the approximate reciprocal (2 ulp) and the
// rounded product leave the single-precision quotient within a relative
// 2^-21 of a / b, i.e. off by less than |a| / b * 2^-21 < 0.5, so its floor
// is within one of the true one and the remainder test corrects it.
__device__ __forceinline__ int floor_div_small(int a, int b) {
  int q = __float2int_rd(__fmul_rn(__int2float_rn(a), __fdividef(1.0f, __int2float_rn(b))));
  const int r = a - q * b;
  if (r < 0) --q;
  else if (r >= b) ++q;
  return q;
}

__device__ __forceinline__ int32_t pack_wrap(int w0, int w1, int w2) {
  return gmp_pack_shift(w0, w1, w2);
}

// Sort key of a neighbor image: atom first, then n1, n2, n3 (each biased by 512).
__device__ __forceinline__ unsigned long long sort_key(int64_t j, const int* n) {
  return ((unsigned long long)j << 30) | ((unsigned long long)(n[0] + 512) << 20) |
         ((unsigned long long)(n[1] + 512) << 10) | (unsigned long long)(n[2] + 512);
}
__device__ __forceinline__ void sort_key_image(unsigned long long key, int* n) {
  n[0] = (int)((key >> 20) & 1023) - 512;
  n[1] = (int)((key >> 10) & 1023) - 512;
  n[2] = (int)(key & 1023) - 512;
}

// Reference cell of a structure: the cell index of its first atom along
// each periodic axis (0 when it has no atoms or that position is not
// finite).  Atoms and reference points store their cell index relative to
// it, so a structure placed any number of cells away from its cell keeps
// small stored indices; pair image indices, which are differences of the
// stored indices, do not change.
__device__ inline void struct_ref_cell(const GmpStruct& st, const double* __restrict__ atom_pos, double (&f0)[3]) {
  f0[0] = f0[1] = f0[2] = 0.0;
  if (st.n_atoms <= 0) return;
  const double* x = atom_pos + 3 * st.atom_base;
  const double x0 = x[0], x1 = x[1], x2 = x[2];
  if (!isfinite(x0) || !isfinite(x1) || !isfinite(x2)) return;
  for (int k = 0; k < 3; ++k) {
    if (!st.periodic[k]) continue;
    const double f = floor(x0 * st.Ainv[k] + x1 * st.Ainv[3 + k] + x2 * st.Ainv[6 + k]);
    if (fabs(f) < 1e9) f0[k] = f;
  }
}

// Wraps the fractional coordinate u of a periodic axis into [0, 1) and
// returns the cell index relative to the reference cell f0 (error flag and
// 0 when it does not fit the packed image index).
__device__ inline int wrap_axis(double& u, double f0, uint32_t* err) {
  const double fl = floor(u);
  const double f = fl - f0;
  int w = 0;
  if (fabs(f) > 500.0) {  // image index would not fit the packed shift
    atomicOr(err, GMP_DEV_SHIFT_RANGE);
  } else {
    w = (int)f;
  }
  u -= fl;
  if (u >= 1.0) { u -= 1.0; w += 1; }
  if (u < 0.0) u = 0.0;
  return w;
}

// Per atom: checks, fractional coordinates, wrap, double-float split, bbox.
// bbox (6 keys per structure: min and complemented max of each
// non-periodic fractional axis) may be global or shared memory.
__device__ __forceinline__ void prepare_atom(const GmpStruct* S, const int32_t* __restrict__ struct_of, int64_t a,
                                             const double* __restrict__ pos, const int32_t* __restrict__ species,
                                             int n_el, float4* __restrict__ atom_xh, float4* __restrict__ atom_xl,
                                             GmpD4* __restrict__ atom_u, unsigned long long* bbox,
                                             uint32_t* __restrict__ err) {
  const int s = struct_of[a];
  const GmpStruct& st = S[s];
  double x[3] = {pos[3 * a], pos[3 * a + 1], pos[3 * a + 2]};
  int e = species[a];
  if (e < 0 || e >= n_el) {
    atomicOr(err, GMP_DEV_BAD_SPECIES);
    e = 0;
  }
  if (!isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2])) {
    atomicOr(err, GMP_DEV_NONFINITE);
    x[0] = x[1] = x[2] = 0.0;
  }
  double u[3], f0[3];
  int w[3] = {0, 0, 0};
  struct_ref_cell(st, pos, f0);
  for (int k = 0; k < 3; ++k) {
    u[k] = x[0] * st.Ainv[k] + x[1] * st.Ainv[3 + k] + x[2] * st.Ainv[6 + k];
    if (st.periodic[k]) {
      w[k] = wrap_axis(u[k], f0[k], err);
    } else {
      // both slots start at all-ones; the max slot stores the complemented key
      atomicMin(&bbox[6 * s + 2 * k], order_key(u[k]));
      atomicMin(&bbox[6 * s + 2 * k + 1], ~order_key(u[k]));
    }
  }
  float h[3], l[3];
  for (int k = 0; k < 3; ++k) {
    h[k] = (float)x[k];
    l[k] = (float)(x[k] - (double)h[k]);
  }
  atom_xh[a] = make_float4(h[0], h[1], h[2], __int_as_float(e));
  atom_xl[a] = make_float4(l[0], l[1], l[2], __int_as_float(pack_wrap(w[0], w[1], w[2])));
  atom_u[a] = GmpD4{u[0], u[1], u[2], 0.0};
}

__global__ void k_prepare(const GmpStruct* __restrict__ S, const int32_t* __restrict__ struct_of,
                          int64_t N, const double* __restrict__ pos,
                          const int32_t* __restrict__ species, int n_el,
                          float4* __restrict__ atom_xh, float4* __restrict__ atom_xl,
                          GmpD4* __restrict__ atom_u, unsigned long long* __restrict__ bbox,
                          uint32_t* __restrict__ err) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < N;
       a += (int64_t)gridDim.x * blockDim.x)
    prepare_atom(S, struct_of, a, pos, species, n_el, atom_xh, atom_xl, atom_u, bbox, err);
}

// Per structure: bin grid and the FP32 pre-screen bound.  bbox may be
// global or shared memory.
__device__ inline void grid_struct(GmpStruct* S, int s, const unsigned long long* bbox, GmpGrid* G,
                                   double cutoff) {
  const GmpStruct& st = S[s];
  GmpGrid g;
  double umax[3], ext[3];
  for (int k = 0; k < 3; ++k) {
    if (st.periodic[k]) {
      g.umin[k] = 0.0;
      umax[k] = 1.0;
      ext[k] = 1.0;
      double target = 0.5 * st.reach[k];
      double nbf = target > 0.0 ? floor(1.0 / target) : 1.0;
      g.nb[k] = (int)fmin(fmax(nbf, 1.0), 1024.0);
      g.binw[k] = 1.0 / g.nb[k];
    } else {
      double lo = st.n_atoms ? key_to_double(bbox[6 * s + 2 * k]) : 0.0;
      double hi = st.n_atoms ? key_to_double(~bbox[6 * s + 2 * k + 1]) : 0.0;
      g.umin[k] = lo;
      umax[k] = hi;
      ext[k] = hi - lo;
      g.binw[k] = fmax(0.5 * st.reach[k], 1e-12);
      double nbf = floor(ext[k] / g.binw[k]) + 1.0;
      g.nb[k] = (int)fmin(fmax(nbf, 1.0), 1024.0);
      if (g.nb[k] == 1024) g.binw[k] = fmax(ext[k] / 1023.0, g.binw[k]);
    }
  }
  // keep the grid within the reserved bin slots
  while ((int64_t)g.nb[0] * g.nb[1] * g.nb[2] > st.bin_cap) {
    int k = 0;
    if (g.nb[1] > g.nb[k]) k = 1;
    if (g.nb[2] > g.nb[k]) k = 2;
    if (st.periodic[k]) {
      g.nb[k] = (g.nb[k] + 1) / 2;
      g.binw[k] = 1.0 / g.nb[k];
    } else {
      g.binw[k] *= 2.0;
      g.nb[k] = (int)fmin(floor(ext[k] / g.binw[k]) + 1.0, 1024.0);
    }
  }
  // Rigorous two-sided FP32 bounds.  Wrapped Cartesian coordinates are
  // |y_c| <= Y, image shifts |s_c| <= Sh; the FP32 displacement
  // (y_j - y_i) + s has per-component error below 2^-22 (4Y + 4Sh + rc)
  // <= delta = 2^-21 (Y + Sh + rc) (a few roundings of magnitude <= 2Y + Sh
  // each, plus the rounding of the cell to FP32), so | |d32| - |d| | <=
  // sqrt(3) delta, and the three-term FP32 r^2 is within 2^-21 relative of
  // |d32|^2.  Hence FP32 r^2 > (rc + 2 delta)^2 (1 + 2^-20) means |d| > rc
  // and FP32 r^2 < (rc - 2 delta)^2 (1 - 2^-20) means |d| < rc, both by a
  // margin far above the FP64 rounding of the defining expression; only the
  // shell in between needs the exact test.
  // Centers need not be atoms (reference points): along a non-periodic axis
  // a center scans some bin only if its coordinate lies within reach + one
  // bin width of the atoms' range, which the bound on |y| covers.
  double Y = 0.0, Sh = 0.0;
  for (int c = 0; c < 3; ++c) {
    double yc = 0.0, sc = 0.0;
    for (int k = 0; k < 3; ++k) {
      double a = fabs(st.A[3 * k + c]);
      double uk = fmax(fabs(g.umin[k]), fabs(umax[k])) + 1.0 +
                  (st.periodic[k] ? 0.0 : st.reach[k] + 2.0 * g.binw[k]);
      yc += uk * a;
      sc += (ceil(st.reach[k]) + 2.0) * a;
    }
    Y = fmax(Y, yc);
    Sh = fmax(Sh, sc);
  }
  double delta = ldexp(Y + Sh + cutoff, -21);
  double b = (cutoff + 2.0 * delta);
  g.pad = 0;
  for (int k = 0; k < 3; ++k) g.inv_binw[k] = 1.0 / g.binw[k];
  G[s] = g;
  float p2 = (float)(b * b * (1.0 + ldexp(1.0, -20)));
  S[s].prescreen2 = nextafterf(p2, INFINITY);
  const double bi = fmax(cutoff - 2.0 * delta, 0.0);
  float q2 = (float)(bi * bi * (1.0 - ldexp(1.0, -20)));
  S[s].inside2 = fmaxf(nextafterf(q2, 0.0f), 0.0f);
}

__global__ void k_grid(GmpStruct* __restrict__ S, int n_struct,
                       const unsigned long long* __restrict__ bbox, GmpGrid* __restrict__ G,
                       double cutoff) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n_struct) grid_struct(S, s, bbox, G, cutoff);
}

// Bin of an atom at wrapped fractional coordinates u4 in structure s.
__device__ __forceinline__ int32_t bin_of(const GmpStruct* S, const GmpGrid* G, int s, const GmpD4& u4) {
  const GmpGrid& g = G[s];
  const double u[3] = {u4.x, u4.y, u4.z};
  int b[3];
  for (int k = 0; k < 3; ++k) {
    double t = floor((u[k] - g.umin[k]) * g.inv_binw[k]);  // as center_range scales
    t = fmin(fmax(t, 0.0), (double)(g.nb[k] - 1));
    b[k] = (int)t;
  }
  return (int32_t)(S[s].bin_base + b[0] + (int64_t)g.nb[0] * (b[1] + (int64_t)g.nb[1] * b[2]));
}

// Bin slot of atom a: bin_y = (wrapped FP32 position, packed wrap of the
// atom), bin_je = (atom index, species).
// (wrap = atom_xl[a].w, spec = atom_xh[a].w: packed wrap and species bits)
__device__ __forceinline__ void write_slot(const GmpStruct& st, int64_t a, int32_t slot, const GmpD4& u4,
                                           float spec, float wrap, float4* __restrict__ bin_y,
                                           int2* __restrict__ bin_je) {
  float y[3];
  for (int c = 0; c < 3; ++c) y[c] = (float)(u4.x * st.A[c] + u4.y * st.A[3 + c] + u4.z * st.A[6 + c]);
  bin_y[slot] = make_float4(y[0], y[1], y[2], wrap);
  bin_je[slot] = make_int2((int32_t)a, __float_as_int(spec));
}

__global__ void k_bin_assign(const GmpStruct* __restrict__ S, const GmpGrid* __restrict__ G,
                             const int32_t* __restrict__ struct_of, int64_t N,
                             const GmpD4* __restrict__ atom_u, int32_t* __restrict__ atom_bin,
                             int32_t* __restrict__ bin_count) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < N;
       a += (int64_t)gridDim.x * blockDim.x) {
    const int32_t bin = bin_of(S, G, struct_of[a], atom_u[a]);
    atom_bin[a] = bin;
    atomicAdd(&bin_count[bin], 1);
  }
}

// Slot lists in arbitrary order: slot_atom[bin_start[b] + k] = the k-th
// atom to arrive in bin b.
__global__ void k_bin_scatter(int64_t N, const int32_t* __restrict__ atom_bin,
                              const int32_t* __restrict__ bin_start, int32_t* __restrict__ bin_cursor,
                              int32_t* __restrict__ slot_atom) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < N;
       a += (int64_t)gridDim.x * blockDim.x) {
    const int32_t bin = atom_bin[a];
    slot_atom[bin_start[bin] + atomicAdd(&bin_cursor[bin], 1)] = (int32_t)a;
  }
}

// Per slot: the atom's rank by index within its bin gives its final slot
// (bins in atom-index order, which makes neighbor enumeration
// deterministic); the bin's slot list is read in parallel, not sorted in
// place.
__global__ void k_bin_place(const GmpStruct* __restrict__ S, const int32_t* __restrict__ struct_of, int64_t N,
                            const int32_t* __restrict__ atom_bin, const int32_t* __restrict__ bin_start,
                            const int32_t* __restrict__ slot_atom, const GmpD4* __restrict__ atom_u,
                            const float4* __restrict__ atom_xh, const float4* __restrict__ atom_xl,
                            float4* __restrict__ bin_y, int2* __restrict__ bin_je) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < N;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = slot_atom[t];
    const int32_t bin = atom_bin[a];
    const int32_t b0 = bin_start[bin], b1 = bin_start[bin + 1];
    int32_t rank = 0;
    for (int32_t u = b0; u < b1; ++u) rank += slot_atom[u] < a ? 1 : 0;
    write_slot(S[struct_of[a]], a, b0 + rank, atom_u[a], atom_xh[a].w, atom_xl[a].w, bin_y, bin_je);
  }
}

// Bins a center at wrapped fractional coordinates u can reach, and its
// wrapped FP32 position.
__device__ __forceinline__ void center_range(const GmpStruct& st, const GmpGrid& g, const double* u,
                                             int4& rng_out, float4& y_out) {
  int lo[3], span[3];
  for (int k = 0; k < 3; ++k) {
    const double lo_f = (u[k] - st.reach[k] - g.umin[k]) * g.inv_binw[k];
    const double hi_f = (u[k] + st.reach[k] - g.umin[k]) * g.inv_binw[k];
    int l0, h0;
    if (st.periodic[k]) {
      l0 = (int)floor(lo_f - 1e-7);
      h0 = (int)floor(hi_f + 1e-7);
    } else {
      // a reference point may lie far outside the atoms' range: clamp in
      // FP64 before converting (an empty range comes out as h0 < l0)
      l0 = (int)fmin(fmax(floor(lo_f - 1e-7), 0.0), (double)g.nb[k]);
      h0 = (int)fmax(fmin(floor(hi_f + 1e-7), (double)(g.nb[k] - 1)), -1.0);
    }
    lo[k] = l0;
    span[k] = max(h0 - l0 + 1, 0);
  }
  float y[3];
  for (int c = 0; c < 3; ++c) y[c] = (float)(u[0] * st.A[c] + u[1] * st.A[3 + c] + u[2] * st.A[6 + c]);
  rng_out = make_int4(lo[0], lo[1], lo[2], span[0] | (span[1] << 10) | (span[2] << 20));
  y_out = make_float4(y[0], y[1], y[2], 0.0f);
}

// Per atom: the bins its cutoff sphere can touch, lo[k] .. lo[k]+span[k]-1
// (periodic axes unwrapped), and its wrapped FP32 position.  Once per atom,
// so the neighbor kernels need no FP64 set-up.  atom_u is overwritten with
// {yx, yy, yz, packed (lo, span)} in a second array.
__global__ void k_ranges(const GmpStruct* __restrict__ S, const GmpGrid* __restrict__ G,
                         const int32_t* __restrict__ struct_of, int64_t N, const GmpD4* __restrict__ atom_u,
                         int4* __restrict__ atom_rng, float4* __restrict__ atom_y) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < N;
       a += (int64_t)gridDim.x * blockDim.x) {
    const int s = struct_of[a];
    const GmpStruct& st = S[s];
    const GmpGrid& g = G[s];
    const GmpD4 u4 = atom_u[a];
    const double u[3] = {u4.x, u4.y, u4.z};
    center_range(st, g, u, atom_rng[a], atom_y[a]);
  }
}

// Per reference point: the checks, wrap and double-float split of
// k_prepare and the bin range of k_ranges, in the structure's atom grid.
__global__ void k_point_prepare(const GmpStruct* __restrict__ S, const GmpGrid* __restrict__ G,
                                const int32_t* __restrict__ point_struct, int64_t n, const double* __restrict__ pts,
                                const double* __restrict__ atom_pos, float4* __restrict__ pt_xh,
                                float4* __restrict__ pt_xl, int4* __restrict__ pt_rng, float4* __restrict__ pt_y,
                                uint32_t* __restrict__ err) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n;
       a += (int64_t)gridDim.x * blockDim.x) {
    const int s = point_struct[a];
    const GmpStruct& st = S[s];
    double x[3] = {pts[3 * a], pts[3 * a + 1], pts[3 * a + 2]};
    if (!isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2])) {
      atomicOr(err, GMP_DEV_NONFINITE);
      x[0] = x[1] = x[2] = 0.0;
    }
    double u[3], f0[3];
    int w[3] = {0, 0, 0};
    struct_ref_cell(st, atom_pos, f0);  // the reference cell of the structure's atoms
    for (int k = 0; k < 3; ++k) {
      u[k] = x[0] * st.Ainv[k] + x[1] * st.Ainv[3 + k] + x[2] * st.Ainv[6 + k];
      if (st.periodic[k]) w[k] = wrap_axis(u[k], f0[k], err);
    }
    float h[3], l[3];
    for (int k = 0; k < 3; ++k) {
      h[k] = (float)x[k];
      l[k] = (float)(x[k] - (double)h[k]);
    }
    pt_xh[a] = make_float4(h[0], h[1], h[2], 0.0f);
    pt_xl[a] = make_float4(l[0], l[1], l[2], __int_as_float(pack_wrap(w[0], w[1], w[2])));
    center_range(st, G[s], u, pt_rng[a], pt_y[a]);
  }
}

// Small batches: the whole binning (k_prepare, k_grid, k_bin_assign, the
// scan, k_bin_scatter, k_bin_place, k_ranges) in one CTA, the bin counts,
// offsets and slot lists in shared memory; same outputs as those kernels
// (bins hold their atoms in index order).  A batch of up to about a
// thousand atoms spends most of its multi-kernel binning time in launch and
// tail latency, not work; past that the one SM's FP64 set-up dominates.
// The pointers written here and read back by other threads are plain
// (no __restrict__), so those reads see the writes after __syncthreads().
__host__ __device__ inline size_t small_bin_smem(int64_t N, int64_t n_bins, int n_struct) {
  return sizeof(unsigned long long) * 6 * (size_t)n_struct + sizeof(int32_t) * (size_t)(2 * n_bins + 1 + N);
}

__global__ void __launch_bounds__(1024) k_bin_small(GmpStruct* S, int n_struct, const int32_t* __restrict__ struct_of,
                                                   int64_t N, double cutoff, const double* __restrict__ pos,
                                                   const int32_t* __restrict__ species, int n_el, GmpGrid* G,
                                                   int64_t n_bins, float4* atom_xh, float4* atom_xl, GmpD4* atom_u,
                                                   int32_t* atom_bin, int32_t* __restrict__ bin_start,
                                                   float4* __restrict__ bin_y, int2* __restrict__ bin_je,
                                                   int4* __restrict__ atom_rng, float4* __restrict__ atom_y,
                                                   uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char sm_small[];
  __shared__ int32_t warp_tot[32];
  unsigned long long* bbox = reinterpret_cast<unsigned long long*>(sm_small);
  int32_t* cnt = reinterpret_cast<int32_t*>(bbox + 6 * n_struct);  // [n_bins] counts, then cursors
  int32_t* start = cnt + n_bins;                                    // [n_bins + 1] exclusive offsets
  int32_t* slot_atom = start + n_bins + 1;                          // [N] atom of each slot
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  for (int t = tid; t < 6 * n_struct; t += nt) bbox[t] = ~0ull;
  for (int64_t b = tid; b < n_bins; b += nt) cnt[b] = 0;
  __syncthreads();
  for (int64_t a = tid; a < N; a += nt)
    prepare_atom(S, struct_of, a, pos, species, n_el, atom_xh, atom_xl, atom_u, bbox, err);
  __syncthreads();
  for (int s = tid; s < n_struct; s += nt) grid_struct(S, s, bbox, G, cutoff);
  __syncthreads();
  for (int64_t a = tid; a < N; a += nt) {
    const int32_t b = bin_of(S, G, struct_of[a], atom_u[a]);
    atom_bin[a] = b;
    atomicAdd(&cnt[b], 1);
  }
  __syncthreads();
  // exclusive scan of the counts: a contiguous chunk per thread, then the
  // chunk totals across the block
  const int64_t chunk = (n_bins + nt - 1) / nt;
  const int64_t c0 = min((int64_t)tid * chunk, n_bins), c1 = min(c0 + chunk, n_bins);
  int32_t run = 0;
  for (int64_t b = c0; b < c1; ++b) run += cnt[b];
  int32_t incl = run;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int32_t w = lane < (nt >> 5) ? warp_tot[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t v = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += v;
    }
    warp_tot[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  int32_t off = incl - run + (wid > 0 ? warp_tot[wid - 1] : 0);
  for (int64_t b = c0; b < c1; ++b) {
    const int32_t c = cnt[b];
    start[b] = off;
    cnt[b] = off;  // cursor
    off += c;
  }
  if (tid == 0) start[n_bins] = (int32_t)N;
  __syncthreads();
  for (int64_t a = tid; a < N; a += nt) slot_atom[atomicAdd(&cnt[atom_bin[a]], 1)] = (int32_t)a;
  __syncthreads();
  // each bin's atoms in index order (insertion sort; a bin holds few atoms)
  for (int64_t b = tid; b < n_bins; b += nt) {
    const int b0 = start[b], b1 = start[b + 1];
    for (int t = b0 + 1; t < b1; ++t) {
      const int32_t v = slot_atom[t];
      int u = t - 1;
      while (u >= b0 && slot_atom[u] > v) {
        slot_atom[u + 1] = slot_atom[u];
        --u;
      }
      slot_atom[u + 1] = v;
    }
  }
  __syncthreads();
  for (int64_t t = tid; t < N; t += nt) {
    const int64_t a = slot_atom[t];
    write_slot(S[struct_of[a]], a, (int32_t)t, atom_u[a], atom_xh[a].w, atom_xl[a].w, bin_y, bin_je);
  }
  for (int64_t b = tid; b <= n_bins; b += nt) bin_start[b] = start[b];
  for (int64_t a = tid; a < N; a += nt) {
    const int s = struct_of[a];
    const GmpD4 u4 = atom_u[a];
    const double u[3] = {u4.x, u4.y, u4.z};
    center_range(S[s], G[s], u, atom_rng[a], atom_y[a]);
  }
}

// ------------------------------------------------------------------ scan
template <typename T>
__global__ void k_scan_block(const T* __restrict__ in, T* __restrict__ out, T* __restrict__ sums,
                             int64_t n) {
  __shared__ T sh[1024];
  const int64_t base = (int64_t)blockIdx.x * 1024;
  const int t = threadIdx.x;
  T v = (base + t < n) ? in[base + t] : T(0);
  sh[t] = v;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    T add = (t >= off) ? sh[t - off] : T(0);
    __syncthreads();
    sh[t] += add;
    __syncthreads();
  }
  if (base + t < n) out[base + t] = sh[t] - v;  // exclusive
  if (t == 1023) sums[blockIdx.x] = sh[1023];
}

template <typename T>
__global__ void k_scan_add(T* __restrict__ out, const T* __restrict__ offs, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  if (i < n) out[i] += offs[blockIdx.x];
}

// out[0..n] exclusive scan of in[0..n-1]; out[n] = total.  tmp sized by
// gmp_scan_tmp_bytes(n).
template <typename T>
cudaError_t exclusive_scan(const T* in, T* out, int64_t n, void* tmp, cudaStream_t st,
                           int64_t* launches) {
  if (n <= 0) {
    return cudaMemsetAsync(out, 0, sizeof(T), st);
  }
  const int64_t nb = (n + 1023) / 1024;
  T* sums = (T*)tmp;
  T* sums_scan = sums + nb + 1;
  void* rest = (void*)(sums_scan + nb + 1);
  k_scan_block<T><<<(unsigned)nb, 1024, 0, st>>>(in, out, sums, n);
  ++*launches;
  if (nb == 1) {
    // total = sums[0]
    cudaError_t e = cudaMemcpyAsync(out + n, sums, sizeof(T), cudaMemcpyDeviceToDevice, st);
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  cudaError_t e = exclusive_scan<T>(sums, sums_scan, nb, rest, st, launches);
  if (e != cudaSuccess) return e;
  k_scan_add<T><<<(unsigned)nb, 1024, 0, st>>>(out, sums_scan, n);
  ++*launches;
  return cudaMemcpyAsync(out + n, sums_scan + nb, sizeof(T), cudaMemcpyDeviceToDevice, st);
}

// ----------------------------------------------------------- neighbor pass
struct Cand {
  bool ok;
  int n[3];
};

// The FP64 expression of the neighbor definition, evaluated exactly as written.
__device__ __noinline__ bool fp64_within(const double* __restrict__ pos, const double* __restrict__ xi,
                                         int64_t j, const GmpStruct& st, const int* n, double rc2) {
  double d[3];
  for (int c = 0; c < 3; ++c) {
    double sh = __dadd_rn(__dadd_rn(__dmul_rn((double)n[0], st.A[c]), __dmul_rn((double)n[1], st.A[3 + c])),
                          __dmul_rn((double)n[2], st.A[6 + c]));
    d[c] = __dadd_rn(__dsub_rn(pos[3 * j + c], xi[c]), sh);
  }
  double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
  return r2 < rc2;
}

__device__ __forceinline__ bool exact_accept(const double* __restrict__ pos, const double* __restrict__ xi, int64_t j,
                                             const float4& xhi, const float4& xli, const float4& xhj,
                                             const float4& xlj, const GmpStruct& st, const int* n,
                                             float rc2hi, float rc2lo, double rc2, float cutoff) {
  gmp_f2 d[3], r2;
  float mag;
  gmp_df_disp(xhi, xli, xhj, xlj, st, n, d, r2, mag);
  gmp_f2 diff = gmp_df_add(r2, gmp_f2{-rc2hi, -rc2lo});
  // double-float error bound (generous): 2^-36 (mag + rc + 1) (rc + 1) * 16
  const float tol = ldexpf((mag + cutoff + 1.0f) * (cutoff + 1.0f) * 16.0f, -36);
  if (diff.hi < -tol) return true;
  if (diff.hi > tol) return false;
  return fp64_within(pos, xi, j, st, n, rc2);
}

// Per-warp shared memory of the fill passes: keys [max_keys] u64, species
// of each key [max_keys] u16 (FILL 1), per-species counters [n_el] int.
__host__ __device__ inline size_t fill_warp_bytes(int max_keys, int n_el) {
  return ((size_t)max_keys * 10 + (size_t)n_el * 4 + 15) / 16 * 16;
}

// Warp per center, latency-bound (dependent bin loads): the launch bounds
// hold the kernel at 80 registers, 24 resident warps per SM instead of 20
// at the 96 it would take (slab single pass 1.88 -> 1.82 ms).
// FILL = 0: count exact neighbors; FILL = 1: write the
// pair records grouped by neighbor species, in enumeration order within a
// species (cells in a fixed order, atoms in index order within a cell:
// deterministic); FILL = 2: sorted by (neighbor atom, image).
template <int FILL>
__global__ void __launch_bounds__(128, 6) k_neighbors(const GmpStruct* __restrict__ S, const GmpGrid* __restrict__ G,
                            const GmpCenters C, int64_t N, float cutoff,
                            float rc2hi, float rc2lo, double rc2, const double* __restrict__ pos,
                            const float4* __restrict__ atom_xh, const float4* __restrict__ atom_xl,
                            const int32_t* __restrict__ bin_start, const float4* __restrict__ bin_y,
                            const int2* __restrict__ bin_je, int n_el,
                            int64_t* __restrict__ counts, const int64_t* __restrict__ offsets,
                            unsigned long long* __restrict__ cursor, int64_t* __restrict__ rng,
                            GmpPair* __restrict__ pairs, int64_t pair_cap, int max_keys,
                            int32_t* __restrict__ maxm, uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char sh_fill[];
  constexpr int fill = FILL;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  if (i >= N) return;
  unsigned char* wbase = sh_fill + (size_t)wib * fill_warp_bytes(max_keys, n_el);
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(wbase);
  uint16_t* kel = reinterpret_cast<uint16_t*>(wbase + (size_t)max_keys * 8);
  int* ecnt = reinterpret_cast<int*>(wbase + (size_t)max_keys * 10);  // max_keys: a power of 2 >= 32

  const int s = C.sid[i];
  const GmpStruct& st = S[s];
  const GmpGrid& g = G[s];
  int nb[3], per[3];
  float ahi[9];
#pragma unroll
  for (int k = 0; k < 3; ++k) { nb[k] = g.nb[k]; per[k] = st.periodic[k]; }
#pragma unroll
  for (int k = 0; k < 9; ++k) ahi[k] = st.Ahi[k];
  const int64_t bin_base = st.bin_base;
  const float p2 = st.prescreen2, q2 = st.inside2;
  const float4 xhi = C.xh[i], xli = C.xl[i];
  const double* xi = C.pos + 3 * i;
  int wi[3];
  gmp_unpack_shift(__float_as_int(xli.w), wi);
  const int4 rg = C.rng[i];
  const int lo[3] = {rg.x, rg.y, rg.z};
  const int span[3] = {rg.w & 1023, (rg.w >> 10) & 1023, (rg.w >> 20) & 1023};
  const float4 yi4 = C.y[i];
  const float yi[3] = {yi4.x, yi4.y, yi4.z};
  const int total = span[0] * span[1] * span[2];
  int count = 0;   // per lane (count pass) / per warp (fill passes)
  for (int r0 = 0; r0 < total; r0 += 32) {
    const int cidx = r0 + lane;
    int m[3] = {0, 0, 0};
    int b0 = 0, b1 = 0;
    float sh[3] = {0.0f, 0.0f, 0.0f};
    if (cidx < total) {
      // cell (c0, c1, c2) of the box and its bin; all operands are below
      // 2^20 in magnitude unless the box is huge (then integer division:
      // a cutoff of over 50 cell widths along periodic axes reaches it, and
      // its image count then exceeds the per-center limit)
      int c0, c1, c2;
      const bool small = total < (1 << 20);
      if (small) {
        const int t01 = floor_div_small(cidx, span[0]);
        c0 = cidx - t01 * span[0];
        c2 = floor_div_small(t01, span[1]);
        c1 = t01 - c2 * span[1];
      } else {
        c0 = cidx % span[0];
        c1 = (cidx / span[0]) % span[1];
        c2 = cidx / (span[0] * span[1]);
      }
      const int bb[3] = {lo[0] + c0, lo[1] + c1, lo[2] + c2};
      int bw[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (per[k]) {
          m[k] = small ? floor_div_small(bb[k], nb[k]) : floor_div(bb[k], nb[k]);
          bw[k] = bb[k] - m[k] * nb[k];
        } else {
          bw[k] = bb[k];
        }
      }
      const int64_t bin = bin_base + bw[0] + (int64_t)nb[0] * (bw[1] + (int64_t)nb[1] * bw[2]);
#pragma unroll
      for (int c = 0; c < 3; ++c)
        sh[c] = (float)m[0] * ahi[c] + (float)m[1] * ahi[3 + c] + (float)m[2] * ahi[6 + c];
      b0 = bin_start[bin];
      b1 = bin_start[bin + 1];
    }
    // lockstep over the slots of this round's cells
    const int len = __reduce_max_sync(0xffffffffu, b1 - b0);
    for (int t = 0; t < len; ++t) {
      const int slot = b0 + t;
      bool acc = false;
      unsigned long long key = 0;
      int ej = 0;
      if (slot < b1) {
        const float4 yj = bin_y[slot];
        const float dx = (yj.x - yi[0]) + sh[0];
        const float dy = (yj.y - yi[1]) + sh[1];
        const float dz = (yj.z - yi[2]) + sh[2];
        // three roundings of non-negative terms: within 3 x 2^-24 relative
        const float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
        if (r2 <= p2) {
          int wj[3];
          gmp_unpack_shift(__float_as_int(yj.w), wj);
          int n[3] = {m[0] + wi[0] - wj[0], m[1] + wi[1] - wj[1], m[2] + wi[2] - wj[2]};
          acc = true;
          int64_t j = -1;
          if (r2 >= q2) {  // boundary shell: exact decision
            const int2 je = bin_je[slot];
            j = je.x;
            ej = je.y;
            const float4 xhj = atom_xh[j], xlj = atom_xl[j];
            acc = exact_accept(pos, xi, j, xhi, xli, xhj, xlj, st, n, rc2hi, rc2lo, rc2, cutoff);
          }
          if (acc && (abs(n[0]) >= 512 || abs(n[1]) >= 512 || abs(n[2]) >= 512)) {
            atomicOr(err, GMP_DEV_SHIFT_RANGE);  // reported after the count pass
            acc = false;
          }
          if (fill && acc) {
            if (j < 0) {
              const int2 je = bin_je[slot];
              j = je.x;
              ej = je.y;
            }
            key = sort_key(j, n);
          }
        }
      }
      if (!fill) {
        count += acc ? 1 : 0;
      } else {
        const unsigned mask = __ballot_sync(0xffffffffu, acc);
        const int slot_k = count + __popc(mask & ((1u << lane) - 1u));
        if (acc && slot_k < max_keys) {
          keys[slot_k] = key;
          if (fill == 1) kel[slot_k] = (uint16_t)ej;
        }
        count += __popc(mask);
      }
    }
  }
  if (!fill) {
    for (int o = 16; o; o >>= 1) count += __shfl_xor_sync(0xffffffffu, count, o);
    if (lane == 0) {
      counts[i] = count;
      atomicMax(maxm, count);
    }
    return;
  }
  __syncwarp();
  const int M = count;
  int64_t base;
  if (cursor) {
    // single pass (no count pass before): this center's block is allocated
    // here; its range goes to rng[i], rng[N + i]; a block beyond the
    // capacity guessed from an earlier call is flagged and the caller
    // repeats the build with the two-pass scheme
    unsigned long long b = 0;
    if (lane == 0) {
      b = atomicAdd(cursor, (unsigned long long)M);
      atomicMax(maxm, M);
    }
    base = (int64_t)__shfl_sync(0xffffffffu, b, 0);
    const bool over = base + M > pair_cap || M > max_keys;
    if (lane == 0) {
      rng[i] = over ? 0 : base;
      rng[N + i] = over ? 0 : base + M;
      if (over) atomicOr(err, GMP_DEV_CAPACITY);
    }
    if (over) return;
  } else {
    base = offsets[i];
    if (offsets[i + 1] > pair_cap || M > max_keys) {  // capacities fixed in advance (graph replay)
      if (lane == 0) atomicOr(err, GMP_DEV_CAPACITY);
      return;
    }
    if (M != (int)(offsets[i + 1] - base)) {
      if (lane == 0) atomicOr(err, GMP_DEV_TOO_MANY_NEIGHBORS);
      return;
    }
  }
  if (fill == 2) {
    // bitonic sort of the M keys (padded to a power of two with ~0)
    int P2 = 1;
    while (P2 < M) P2 <<= 1;
    for (int t = M + lane; t < P2; t += 32) keys[t] = ~0ull;
    __syncwarp();
    for (int k = 2; k <= P2; k <<= 1) {
      for (int jj = k >> 1; jj > 0; jj >>= 1) {
        for (int t = lane; t < P2; t += 32) {
          int partner = t ^ jj;
          if (partner > t) {
            unsigned long long a = keys[t], b = keys[partner];
            bool up = (t & k) == 0;
            if ((a > b) == up) {
              keys[t] = b;
              keys[partner] = a;
            }
          }
        }
        __syncwarp();
      }
    }
  }
  if (fill == 1) {
    // destination of key t: species-major, enumeration order within a
    // species (counting sort; lanes of one match group have one species)
    for (int e = lane; e < n_el; e += 32) ecnt[e] = 0;
    __syncwarp();
    for (int t0 = 0; t0 < M; t0 += 32) {
      const int t = t0 + lane;
      const int e = t < M ? (int)kel[t] : -1;
      const unsigned grp = __match_any_sync(0xffffffffu, e);
      if (t < M && lane == __ffs(grp) - 1) ecnt[e] += __popc(grp);
      __syncwarp();
    }
    if (lane == 0) {
      int run = 0;
      for (int e = 0; e < n_el; ++e) {
        const int c = ecnt[e];
        ecnt[e] = run;
        run += c;
      }
    }
    __syncwarp();
  }
  // records: the double-float displacement, rounded to FP32
  for (int t0 = 0; t0 < M; t0 += 32) {
    const int t = t0 + lane;
    int dst = t;
    if (fill == 1) {
      const int e = t < M ? (int)kel[t] : -1;
      const unsigned grp = __match_any_sync(0xffffffffu, e);
      if (t < M) dst = ecnt[e] + __popc(grp & ((1u << lane) - 1u));
      __syncwarp();
      if (t < M && lane == __ffs(grp) - 1) ecnt[e] += __popc(grp);
      __syncwarp();
    }
    if (t >= M) continue;
    const unsigned long long key = keys[t];
    const int64_t j = (int64_t)(key >> 30);
    int n[3];
    sort_key_image(key, n);
    const int32_t packed = gmp_pack_shift(n[0], n[1], n[2]);
    const float4 xhj = atom_xh[j], xlj = atom_xl[j];
    gmp_f2 d[3], r2;
    float mag;
    gmp_df_disp(xhi, xli, xhj, xlj, st, n, d, r2, mag);
    GmpPair p;
    p.dx = d[0].hi + d[0].lo;
    p.dy = d[1].hi + d[1].lo;
    p.dz = d[2].hi + d[2].lo;
    p.r2hi = r2.hi;
    p.r2lo = r2.lo;
    p.e = __float_as_int(xhj.w);
    p.j = (int32_t)j;
    p.shift = packed;
    pairs[base + dst] = p;
  }
}

__global__ void k_unpack(int64_t P, const GmpPair* __restrict__ pairs, int32_t* __restrict__ nbr_j,
                         int32_t* __restrict__ nbr_shift) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < P;
       t += (int64_t)gridDim.x * blockDim.x) {
    GmpPair p = pairs[t];
    int n[3];
    gmp_unpack_shift(p.shift, n);
    nbr_j[t] = p.j;
    nbr_shift[3 * t] = n[0];
    nbr_shift[3 * t + 1] = n[1];
    nbr_shift[3 * t + 2] = n[2];
  }
}

inline unsigned grid_for(int64_t n, int threads, int sm_count) {
  int64_t b = (n + threads - 1) / threads;
  int64_t cap = (int64_t)sm_count * 32;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

size_t gmp_scan_tmp_bytes(int64_t n) {
  size_t total = 0;
  while (true) {
    int64_t nb = (n + 1023) / 1024;
    total += 2 * (size_t)(nb + 1) * sizeof(int64_t);
    if (nb <= 1) break;
    n = nb;
  }
  return total + 256;
}

cudaError_t gmp_exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* tmp,
                                   cudaStream_t stream, int64_t* launches) {
  return exclusive_scan<int64_t>(in, out, n, tmp, stream, launches);
}

cudaError_t gmp_launch_neighbors_prepare(const GmpStruct* d_structs, int n_struct,
                                         const int32_t* d_struct_of, int64_t N, double cutoff,
                                         const double* pos, const int32_t* species, int n_el,
                                         GmpGrid* d_grid, float4* atom_xh, float4* atom_xl,
                                         GmpD4* atom_u, int32_t* atom_bin,
                                         unsigned long long* d_bbox, uint32_t* d_err,
                                         cudaStream_t stream, int sm_count, int64_t* launches) {
  (void)atom_bin;
  cudaError_t e = cudaMemsetAsync(d_bbox, 0xFF, sizeof(unsigned long long) * 6 * n_struct, stream);
  if (e != cudaSuccess) return e;
  k_prepare<<<grid_for(N, 256, sm_count), 256, 0, stream>>>(d_structs, d_struct_of, N, pos, species,
                                                            n_el, atom_xh, atom_xl, atom_u, d_bbox,
                                                            d_err);
  ++*launches;
  k_grid<<<(n_struct + 127) / 128, 128, 0, stream>>>((GmpStruct*)d_structs, n_struct, d_bbox, d_grid,
                                                     cutoff);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t gmp_launch_bins(const GmpStruct* d_structs, const GmpGrid* d_grid,
                            const int32_t* d_struct_of, int64_t N, int64_t n_bins,
                            const int32_t* atom_bin, int32_t* bin_count, int32_t* bin_start,
                            int32_t* bin_cursor, int4* atom_rng, float4* atom_y, float4* bin_y, int2* bin_je,
                            const GmpD4* atom_u, const float4* atom_xh, const float4* atom_xl, void* scan_tmp,
                            size_t scan_tmp_bytes, cudaStream_t stream, int sm_count, int64_t* launches) {
  (void)scan_tmp_bytes;
  cudaError_t e = cudaMemsetAsync(bin_count, 0, sizeof(int32_t) * n_bins, stream);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(bin_cursor, 0, sizeof(int32_t) * n_bins, stream);
  if (e != cudaSuccess) return e;
  k_bin_assign<<<grid_for(N, 256, sm_count), 256, 0, stream>>>(d_structs, d_grid, d_struct_of, N,
                                                               atom_u, (int32_t*)atom_bin, bin_count);
  ++*launches;
  e = exclusive_scan<int32_t>(bin_count, bin_start, n_bins, scan_tmp, stream, launches);
  if (e != cudaSuccess) return e;
  // bin_count is free once scanned: it holds the slot lists (n_bins >= N)
  k_bin_scatter<<<grid_for(N, 256, sm_count), 256, 0, stream>>>(N, atom_bin, bin_start, bin_cursor, bin_count);
  ++*launches;
  k_bin_place<<<grid_for(N, 256, sm_count), 256, 0, stream>>>(d_structs, d_struct_of, N, atom_bin, bin_start,
                                                              bin_count, atom_u, atom_xh, atom_xl, bin_y, bin_je);
  ++*launches;
  k_ranges<<<grid_for(N, 256, sm_count), 256, 0, stream>>>(d_structs, d_grid, d_struct_of, N, atom_u, atom_rng,
                                                           atom_y);
  ++*launches;
  return cudaGetLastError();
}

bool gmp_bin_small_fits(int64_t N, int64_t n_bins, int n_struct) {
  return N > 0 && N <= kSmallBinAtoms && n_struct <= 256 && small_bin_smem(N, n_bins, n_struct) <= 200 * 1024;
}

cudaError_t gmp_launch_bin_small(GmpStruct* d_structs, int n_struct, const int32_t* d_struct_of, int64_t N,
                                 double cutoff, const double* pos, const int32_t* species, int n_el,
                                 GmpGrid* d_grid, int64_t n_bins, float4* atom_xh, float4* atom_xl, GmpD4* atom_u,
                                 int32_t* atom_bin, int32_t* bin_start, float4* bin_y, int2* bin_je,
                                 int4* atom_rng, float4* atom_y, uint32_t* d_err, cudaStream_t stream,
                                 int64_t* launches) {
  if (!gmp_bin_small_fits(N, n_bins, n_struct)) return cudaErrorInvalidValue;
  const size_t smem = small_bin_smem(N, n_bins, n_struct);
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_bin_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_bin_small<<<1, 1024, smem, stream>>>(d_structs, n_struct, d_struct_of, N, cutoff, pos, species, n_el, d_grid,
                                         n_bins, atom_xh, atom_xl, atom_u, atom_bin, bin_start, bin_y, bin_je,
                                         atom_rng, atom_y, d_err);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t gmp_launch_point_prepare(const GmpStruct* d_structs, const GmpGrid* d_grid,
                                     const int32_t* point_struct, int64_t n_points, const double* points,
                                     const double* atom_pos, float4* pt_xh, float4* pt_xl, int4* pt_rng,
                                     float4* pt_y, uint32_t* d_err, cudaStream_t stream, int sm_count,
                                     int64_t* launches) {
  if (n_points <= 0) return cudaSuccess;
  k_point_prepare<<<grid_for(n_points, 256, sm_count), 256, 0, stream>>>(
      d_structs, d_grid, point_struct, n_points, points, atom_pos, pt_xh, pt_xl, pt_rng, pt_y, d_err);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t gmp_launch_neighbor_pass(int fill, const GmpStruct* d_structs, const GmpGrid* d_grid,
                                     const GmpCenters& C, int64_t N, double cutoff,
                                     const double* pos, const float4* atom_xh, const float4* atom_xl,
                                     const int32_t* bin_start, const float4* bin_y, const int2* bin_je, int n_el,
                                     int64_t* counts, const int64_t* offsets,
                                     GmpPair* pairs, int64_t pair_cap, int max_keys, int32_t* d_maxm,
                                     uint32_t* d_err, cudaStream_t stream, int sm_count, int64_t* launches,
                                     unsigned long long* cursor, int64_t* rng) {
  (void)sm_count;
  if (fill < 0 || fill > 2 || (cursor && fill == 0)) return cudaErrorInvalidValue;
  const double rc2 = cutoff * cutoff;
  const float rc2hi = (float)rc2;
  const float rc2lo = (float)(rc2 - (double)rc2hi);
  auto fn = fill == 0 ? k_neighbors<0> : fill == 1 ? k_neighbors<1> : k_neighbors<2>;
  int warps = 4;
  size_t smem = 0;
  if (fill) {
    while (warps > 1 && (size_t)warps * fill_warp_bytes(max_keys, n_el) > 96 * 1024) warps >>= 1;
    smem = (size_t)warps * fill_warp_bytes(max_keys, n_el);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
  }
  const unsigned blocks = (unsigned)((N + warps - 1) / warps);
  fn<<<blocks, warps * 32, smem, stream>>>(d_structs, d_grid, C, N, (float)cutoff, rc2hi, rc2lo, rc2, pos,
                                           atom_xh, atom_xl, bin_start, bin_y, bin_je, n_el, counts, offsets,
                                           cursor, rng, pairs, pair_cap, max_keys, d_maxm, d_err);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t gmp_launch_unpack_neighbors(int64_t P, const GmpPair* pairs, int32_t* nbr_j,
                                        int32_t* nbr_shift, cudaStream_t stream,
                                        int64_t* launches) {
  if (P <= 0) return cudaSuccess;
  k_unpack<<<grid_for(P, 256, 152), 256, 0, stream>>>(P, pairs, nbr_j, nbr_shift);
  ++*launches;
  return cudaGetLastError();
}
