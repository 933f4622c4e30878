// C ABI of libgmp (declared in include/gmp.h): validation, device tables,
// workspace, and the launch sequences of the featurize calls.
#include "gmp.h"
#include "gmp_internal.cuh"
#include "gmp_kernels.cuh"
#include "gmp_launch.h"

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

cudaError_t gmp_launch_struct_of(const int64_t* d_atom_off, int n_struct, int32_t* struct_of,
                                 cudaStream_t stream, int64_t* launches);

namespace {

// Device buffer that grows on demand and frees itself (move-only).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      bytes = o.bytes;
      o.p = nullptr;
      o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  cudaError_t ensure(size_t need) {
    if (need <= bytes && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    size_t n = need < 256 ? 256 : need + need / 8;  // grow with slack
    cudaError_t e = cudaMalloc(&p, n);
    if (e == cudaSuccess) bytes = n;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T>
  T* as() const { return static_cast<T*>(p); }
};

struct PassData {
  GmpPass pass;
  int L;
  int NS;
  DevBuf rad;
  // launch shapes (defaults until gmp_tune / gmp_tuning_set)
  GmpShape fwd{16, 0};
  GmpShape bwd{16, 0};
  GmpShape fused{16, 0};
  GmpShape jac{16, 0};
  int vjp_fused = 0;  // 1: one fused forward+backward kernel instead of two
};

}  // namespace

struct gmp_ctx {
  int device = 0;
  int sm_count = 0;
  // parameters
  int n_el = 0;
  std::vector<int> n_gauss;
  std::vector<double> coef, alpha;
  std::vector<int> orders;
  std::vector<double> sigmas;
  double cutoff = 0.0;
  uint32_t flags = 0;
  int F = 0;
  int kmax = 0;
  std::vector<PassData> passes;
  DevBuf dens;
  // cached structure description
  std::vector<int64_t> last_off;
  std::vector<double> last_cell;
  std::vector<uint8_t> last_pbc;
  int64_t n_bins = 0;
  // workspace
  DevBuf structs, grid, atom_off, struct_of, bbox, atom_xh, atom_xl, atom_u, atom_bin, atom_rng, atom_y;
  DevBuf bin_count, bin_cursor, bin_start, bin_y, bin_je, counts, nbr_off, scan_tmp, pairs;
  DevBuf scalars;  // err word, maxm, counter
  DevBuf grad_acc, jac_counts, jac_rows;
  // VJP sums without float atomics: fixed-point bins per (atom,
  // component), per-center own terms and strain-derivative sums
  DevBuf gbins, own, vir_c;
  DevBuf mu;     // per-center moments between the forward and backward kernels
  DevBuf ktab;   // double-float radial constants [n_el][n_sigmas][kmax][16] for the refinement kernel
  DevBuf exptab; // [64] 2^(-j/64) as double-floats (the refinement's exponential)
  DevBuf flagq;     // queued ill-conditioned features, one entry per (center, order)
  DevBuf colinfo;   // per feature column: (order << 16) | sigma, -1 for the density
  int n_ord_pos = 1;  // orders >= 0: refine queue entries per center and pass
  DevBuf stage_pos, stage_species, stage_feat, stage_gradf, stage_gradp, stage_virial;
  DevBuf pt_off, pt_struct, pt_xh, pt_xl, pt_rng, pt_y, stage_pts;  // reference points
  int64_t P = 0;  // pairs of the last neighbor build
  int max_m = 0;
  // Pair layout of the last build: CSR by center (nbr_off) or, after a
  // single-pass build, one block per center with ranges in nbr_rng [2N].
  DevBuf nbr_rng;
  bool rng_mode = false;
  int64_t last_nc = -1;    // batch (centers, description) the P / max_m above belong to
  int64_t last_gen = -1;
  // pinned host scratch for small readbacks
  int64_t* h_small = nullptr;
  std::string err;
  int64_t launches = 0;
  cudaEvent_t ev = nullptr;
  // host-buffer calls: copies on a side stream overlap the kernels
  cudaStream_t side = nullptr;
  cudaEvent_t ev_in = nullptr, ev_feat = nullptr, ev_out = nullptr;
  // CUDA-graph replay of whole calls (gmp_set_graph)
  bool graph_on = false;
  bool graph_valid = false;
  bool capturing = false;
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<uintptr_t> graph_key;
  int64_t cap_pairs = 0;   // capacities baked into the captured graph
  int cap_keys = 0;
  int64_t struct_gen = 0;  // bumped whenever the batch description changes
  // stage timing
  bool profiling = false;
  static constexpr int kStages = 4;     // neighbors, features kernel, backward kernel, refine/finish
  std::vector<cudaEvent_t> prof_ev[kStages];  // start/stop pairs per stage
  size_t prof_used[kStages] = {0, 0, 0, 0};
};

namespace {

gmp_status fail(gmp_ctx* h, gmp_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

gmp_status cuda_fail(gmp_ctx* h, cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(h, GMP_ERR_OOM, std::string("device allocation failed in ") + where);
  }
  return fail(h, GMP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define GMP_CK(expr, where)                      \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

int pad_sigmas(int n) { return n <= 4 ? 4 : (n <= 8 ? 8 : 16); }

cudaError_t launch_compute(int L, int kind, int ns, const gmpk::KParams& K, GmpShape shape, cudaStream_t st,
                           int sm, int64_t* launches) {
  switch (L) {
    case 0: return gmp_launch_compute_L0(kind, ns, K, shape, st, sm, launches);
    case 1: return gmp_launch_compute_L1(kind, ns, K, shape, st, sm, launches);
    case 2: return gmp_launch_compute_L2(kind, ns, K, shape, st, sm, launches);
    case 3: return gmp_launch_compute_L3(kind, ns, K, shape, st, sm, launches);
    case 4: return gmp_launch_compute_L4(kind, ns, K, shape, st, sm, launches);
    case 5: return gmp_launch_compute_L5(kind, ns, K, shape, st, sm, launches);
    case 6: return gmp_launch_compute_L6(kind, ns, K, shape, st, sm, launches);
    default: return cudaErrorInvalidValue;
  }
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool inv3(const double* A, double* Ai) {
  double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
               A[2] * (A[3] * A[7] - A[4] * A[6]);
  double scale = 0.0;
  for (int k = 0; k < 9; ++k) scale = std::fmax(scale, std::fabs(A[k]));
  if (!(std::fabs(det) > 1e-12 * scale * scale * scale) || !std::isfinite(det)) return false;
  Ai[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  Ai[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  Ai[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  Ai[3] = (A[5] * A[6] - A[3] * A[8]) / det;
  Ai[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  Ai[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  Ai[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  Ai[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  Ai[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  return true;
}

// Validates the batch description and uploads per-structure data when it
// changed since the previous call.
// Largest r where term(r) > t, for term(r) = a r^l exp(-b r^2) (a, b > 0):
// increasing up to r* = sqrt(l / (2b)), decreasing beyond; bisection on
// the decreasing branch.
double term_radius(double a, int l, double b, double t) {
  auto term = [&](double r) { return a * std::pow(r, l) * std::exp(-b * r * r); };
  const double rstar = l > 0 ? std::sqrt(l / (2.0 * b)) : 0.0;
  if (term(rstar) <= t) return 0.0;
  double lo = rstar, hi = std::max(2.0 * rstar, 1.0);
  while (term(hi) > t) hi *= 2.0;
  for (int it = 0; it < 200 && hi - lo > 1e-12 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    (term(mid) > t ? lo : hi) = mid;
  }
  return hi;
}

// Cutoff from the overlap threshold t (largest radius of any single
// primitive's bound above t; see gmp_cutoff in gmp.h).
double derived_cutoff(const gmp_ctx& h, double t) {
  double rc = 0.0;
  int64_t off = 0;
  for (int e = 0; e < h.n_el; ++e) {
    for (int q = 0; q < h.n_gauss[e]; ++q) {
      const double a = h.alpha[off + q], c = std::fabs(h.coef[off + q]);
      for (int l : h.orders) {
        if (l < 0) {
          rc = std::max(rc, term_radius(c, 0, a, t));
          continue;
        }
        double lf = 1.0, df = 1.0;
        for (int k = 2; k <= l; ++k) lf *= k;
        for (int k = 2 * l - 1; k > 1; k -= 2) df *= k;
        for (double sig : h.sigmas) {
          const double beta = 1.0 / (2.0 * sig * sig), g = a + beta;
          const double amp = c * std::pow(2.0 * M_PI * sig * sig, -1.5) * std::pow(M_PI / g, 1.5) *
                             std::pow(a / g, l) * std::sqrt(lf * df);
          rc = std::max(rc, term_radius(amp, l, a * beta / g, t));
        }
      }
    }
    off += h.n_gauss[e];
  }
  return rc;
}

gmp_status upload_structures(gmp_ctx* h, int32_t S, const int64_t* atom_off, const double* cell,
                             const uint8_t* pbc, cudaStream_t st) {
  if (S < 1 || !atom_off) return fail(h, GMP_ERR_INVALID_ARG, "n_struct must be >= 1 with atom_off");
  if (atom_off[0] != 0) return fail(h, GMP_ERR_INVALID_ARG, "atom_off[0] must be 0");
  for (int s = 0; s < S; ++s)
    if (atom_off[s + 1] < atom_off[s]) return fail(h, GMP_ERR_INVALID_ARG, "atom_off must be non-decreasing");
  const int64_t N = atom_off[S];
  if (N > (int64_t)INT32_MAX / 2) return fail(h, GMP_ERR_INVALID_ARG, "too many atoms");
  if (!cell || !pbc) return fail(h, GMP_ERR_INVALID_ARG, "cell and pbc (host arrays) are required");
  const bool same = (int64_t)h->last_off.size() == S + 1 &&
                    std::memcmp(h->last_off.data(), atom_off, sizeof(int64_t) * (S + 1)) == 0 &&
                    std::memcmp(h->last_cell.data(), cell, sizeof(double) * 9 * S) == 0 &&
                    std::memcmp(h->last_pbc.data(), pbc, S * 3) == 0;
  if (same) return GMP_OK;
  std::vector<GmpStruct> info(S);
  int64_t bin_base = 0;
  for (int s = 0; s < S; ++s) {
    GmpStruct& g = info[s];
    std::memset(&g, 0, sizeof(g));
    const double* A = cell + 9 * s;
    bool any = false;
    for (int k = 0; k < 3; ++k) {
      g.periodic[k] = pbc[3 * s + k] ? 1 : 0;
      any = any || g.periodic[k];
    }
    if (any) {
      for (int k = 0; k < 9; ++k) {
        if (!std::isfinite(A[k])) return fail(h, GMP_ERR_INVALID_ARG, "non-finite cell");
        g.A[k] = A[k];
      }
      if (!inv3(g.A, g.Ainv))
        return fail(h, GMP_ERR_INVALID_ARG, "singular cell for a structure with a periodic axis (structure " +
                                                std::to_string(s) + ")");
    } else {
      for (int k = 0; k < 9; ++k) g.A[k] = g.Ainv[k] = (k % 4 == 0) ? 1.0 : 0.0;
    }
    for (int k = 0; k < 3; ++k) {
      double bk = std::sqrt(g.Ainv[k] * g.Ainv[k] + g.Ainv[3 + k] * g.Ainv[3 + k] + g.Ainv[6 + k] * g.Ainv[6 + k]);
      g.reach[k] = h->cutoff * bk;
      if (g.periodic[k] && g.reach[k] > 64.0)
        return fail(h, GMP_ERR_INVALID_ARG, "cutoff spans more than 64 cell widths along a periodic axis");
    }
    for (int k = 0; k < 9; ++k) {
      g.Ahi[k] = (float)g.A[k];
      g.Alo[k] = (float)(g.A[k] - (double)g.Ahi[k]);
    }
    g.atom_base = atom_off[s];
    g.n_atoms = (int32_t)(atom_off[s + 1] - atom_off[s]);
    g.bin_base = bin_base;
    g.bin_cap = 2 * g.n_atoms + 8;
    bin_base += g.bin_cap;
  }
  h->n_bins = bin_base;
  GMP_CK(h->structs.ensure(sizeof(GmpStruct) * S), "structs");
  GMP_CK(h->grid.ensure(sizeof(GmpGrid) * S), "grid");
  GMP_CK(h->atom_off.ensure(sizeof(int64_t) * (S + 1)), "atom_off");
  GMP_CK(h->bbox.ensure(sizeof(unsigned long long) * 6 * S), "bbox");
  GMP_CK(cudaMemcpyAsync(h->structs.p, info.data(), sizeof(GmpStruct) * S, cudaMemcpyHostToDevice, st), "upload structs");
  GMP_CK(cudaMemcpyAsync(h->atom_off.p, atom_off, sizeof(int64_t) * (S + 1), cudaMemcpyHostToDevice, st), "upload atom_off");
  GMP_CK(h->struct_of.ensure(sizeof(int32_t) * (N > 0 ? N : 1)), "struct_of");
  if (N > 0) GMP_CK(gmp_launch_struct_of(h->atom_off.as<int64_t>(), S, h->struct_of.as<int32_t>(), st, &h->launches), "struct_of");
  // the copies above read host memory asynchronously: wait before returning
  GMP_CK(cudaStreamSynchronize(st), "upload sync");
  ++h->struct_gen;
  h->last_off.assign(atom_off, atom_off + S + 1);
  h->last_cell.assign(cell, cell + 9 * S);
  h->last_pbc.assign(pbc, pbc + 3 * S);
  return GMP_OK;
}

gmp_status decode_device_error(gmp_ctx* h, uint32_t w) {
  if (!w) return GMP_OK;
  std::string m = "device reported:";
  if (w & GMP_DEV_BAD_SPECIES) m += " species id out of range;";
  if (w & GMP_DEV_NONFINITE) m += " non-finite position;";
  if (w & GMP_DEV_TOO_MANY_NEIGHBORS) m += " neighbor list inconsistent;";
  if (w & GMP_DEV_SHIFT_RANGE) m += " periodic image index beyond +-511 (position far outside its cell?);";
  if (w & GMP_DEV_CAPACITY) m += " capacity exceeded;";
  return fail(h, GMP_ERR_DEVICE, m);
}

// Records a start (begin = true) or stop event of `stage` on `st`.
cudaError_t prof_mark(gmp_ctx* h, int stage, bool begin, cudaStream_t st) {
  if (!h->profiling || h->capturing) return cudaSuccess;
  auto& v = h->prof_ev[stage];
  size_t& u = h->prof_used[stage];
  if (begin && u + 2 > v.size()) {
    for (int k = 0; k < 2; ++k) {
      cudaEvent_t e;
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      v.push_back(e);
    }
  }
  cudaError_t r = cudaEventRecord(v[begin ? u : u + 1], st);
  if (!begin) u += 2;
  return r;
}

// Checks, fractional coordinates and the cell-list bins of the N atoms.
gmp_status bin_atoms(gmp_ctx* h, int32_t S, const double* pos, const int32_t* species, int64_t N,
                     int64_t n_centers, cudaStream_t st) {
  int64_t* L = &h->launches;
  uint32_t* d_err = h->scalars.as<uint32_t>();
  GMP_CK(h->atom_xh.ensure(sizeof(float4) * N), "atom_xh");
  GMP_CK(h->atom_xl.ensure(sizeof(float4) * N), "atom_xl");
  GMP_CK(h->atom_u.ensure(sizeof(GmpD4) * N), "atom_u");
  GMP_CK(h->atom_bin.ensure(sizeof(int32_t) * N), "atom_bin");
  GMP_CK(h->atom_rng.ensure(sizeof(int4) * N), "atom_rng");
  GMP_CK(h->atom_y.ensure(sizeof(float4) * N), "atom_y");
  GMP_CK(h->bin_count.ensure(sizeof(int32_t) * h->n_bins), "bin_count");
  GMP_CK(h->bin_cursor.ensure(sizeof(int32_t) * h->n_bins), "bin_cursor");
  GMP_CK(h->bin_start.ensure(sizeof(int32_t) * (h->n_bins + 1)), "bin_start");
  GMP_CK(h->bin_y.ensure(sizeof(float4) * N), "bin_y");
  GMP_CK(h->bin_je.ensure(sizeof(int2) * N), "bin_je");
  GMP_CK(h->counts.ensure(sizeof(int64_t) * n_centers), "counts");
  GMP_CK(h->nbr_off.ensure(sizeof(int64_t) * (n_centers + 1)), "nbr_off");
  const int64_t scan_n = std::max<int64_t>(std::max<int64_t>(N, n_centers), h->n_bins);
  GMP_CK(h->scan_tmp.ensure(gmp_scan_tmp_bytes(scan_n)), "scan_tmp");

  if (gmp_bin_small_fits(N, h->n_bins, S)) {
    GMP_CK(gmp_launch_bin_small(h->structs.as<GmpStruct>(), S, h->struct_of.as<int32_t>(), N, h->cutoff, pos, species,
                                h->n_el, h->grid.as<GmpGrid>(), h->n_bins, h->atom_xh.as<float4>(),
                                h->atom_xl.as<float4>(), h->atom_u.as<GmpD4>(), h->atom_bin.as<int32_t>(),
                                h->bin_start.as<int32_t>(), h->bin_y.as<float4>(), h->bin_je.as<int2>(),
                                h->atom_rng.as<int4>(), h->atom_y.as<float4>(), d_err, st, L),
           "bins (one block)");
    return GMP_OK;
  }
  GMP_CK(gmp_launch_neighbors_prepare(h->structs.as<GmpStruct>(), S, h->struct_of.as<int32_t>(), N, h->cutoff,
                                      pos, species, h->n_el, h->grid.as<GmpGrid>(), h->atom_xh.as<float4>(),
                                      h->atom_xl.as<float4>(), h->atom_u.as<GmpD4>(), h->atom_bin.as<int32_t>(),
                                      h->bbox.as<unsigned long long>(), d_err, st, h->sm_count, L),
         "prepare");
  GMP_CK(gmp_launch_bins(h->structs.as<GmpStruct>(), h->grid.as<GmpGrid>(), h->struct_of.as<int32_t>(), N,
                         h->n_bins, h->atom_bin.as<int32_t>(), h->bin_count.as<int32_t>(),
                         h->bin_start.as<int32_t>(), h->bin_cursor.as<int32_t>(), h->atom_rng.as<int4>(),
                         h->atom_y.as<float4>(), h->bin_y.as<float4>(), h->bin_je.as<int2>(), h->atom_u.as<GmpD4>(),
                         h->atom_xh.as<float4>(), h->atom_xl.as<float4>(), h->scan_tmp.p, h->scan_tmp.bytes, st,
                         h->sm_count, L),
         "bins");
  return GMP_OK;
}

// Exact neighbor lists of the NC centers C over the binned atoms into
// h->pairs / h->nbr_off.  Synchronises `st` once (to size the pair buffer)
// unless capturing.
gmp_status neighbor_lists(gmp_ctx* h, const GmpCenters& C, int64_t NC, const double* pos, cudaStream_t st,
                          bool sorted, bool capture, bool single_ok = false) {
  int64_t* L = &h->launches;
  uint32_t* d_err = h->scalars.as<uint32_t>();
  int32_t* d_maxm = reinterpret_cast<int32_t*>(d_err + 1);
  unsigned long long* d_cursor = reinterpret_cast<unsigned long long*>(h->scalars.as<char>() + 16);
  h->rng_mode = false;
  // the error word is cleared after it is read (below), so a condition
  // raised after the read of the previous call is reported here
  GMP_CK(cudaMemsetAsync(d_maxm, 0, 4, st), "memset maxm");
  if (single_ok && !capture && h->last_nc == NC && h->last_gen == h->struct_gen && h->P > 0) {
    // Repeated batch: one enumeration pass, each center allocating its
    // block of records, with capacities from the last build + 12.5%
    // (blocks in allocation order: no CSR offsets, ranges in nbr_rng).
    const int64_t cap = h->P + h->P / 8 + 4096;
    int keys = 32;
    while (keys < h->max_m + h->max_m / 8 + 8) keys <<= 1;
    if ((size_t)keys * 8 <= 200 * 1024) {
      GMP_CK(h->pairs.ensure(sizeof(GmpPair) * cap), "pairs");
      GMP_CK(h->nbr_rng.ensure(sizeof(int64_t) * 2 * NC), "nbr_rng");
      GMP_CK(cudaMemsetAsync(d_cursor, 0, 8, st), "memset cursor");
      GMP_CK(gmp_launch_neighbor_pass(sorted ? 2 : 1, h->structs.as<GmpStruct>(), h->grid.as<GmpGrid>(), C, NC, h->cutoff, pos,
                                      h->atom_xh.as<float4>(), h->atom_xl.as<float4>(), h->bin_start.as<int32_t>(),
                                      h->bin_y.as<float4>(), h->bin_je.as<int2>(), h->n_el, nullptr, nullptr,
                                      h->pairs.as<GmpPair>(), cap, keys, d_maxm, d_err, st, h->sm_count, L, d_cursor,
                                      h->nbr_rng.as<int64_t>()),
             "neighbor single pass");
      GMP_CK(cudaMemcpyAsync(h->h_small, d_cursor, 8, cudaMemcpyDeviceToHost, st), "read P");
      GMP_CK(cudaMemcpyAsync(h->h_small + 1, d_err, 8, cudaMemcpyDeviceToHost, st), "read err");
      GMP_CK(cudaStreamSynchronize(st), "neighbor sync");
      const uint32_t w = (uint32_t)(h->h_small[1] & 0xffffffffu);
      if (!w) {
        h->P = h->h_small[0];
        h->max_m = (int)(h->h_small[1] >> 32);
        h->rng_mode = true;
        return GMP_OK;
      }
      GMP_CK(cudaMemsetAsync(d_err, 0, 8, st), "clear err");  // error word and maxm
      if (w != GMP_DEV_CAPACITY) return decode_device_error(h, w);
      // outgrew the guessed capacity: count exactly below
    }
  }
  if (capture && !sorted) {
    // graph replay: the single pass with the capacities fixed at capture
    // time; a block beyond them is flagged on the device and the call then
    // runs eagerly (and recaptures)
    GMP_CK(h->nbr_rng.ensure(sizeof(int64_t) * 2 * NC), "nbr_rng");
    GMP_CK(cudaMemsetAsync(d_cursor, 0, 8, st), "memset cursor");
    GMP_CK(gmp_launch_neighbor_pass(1, h->structs.as<GmpStruct>(), h->grid.as<GmpGrid>(), C, NC, h->cutoff, pos,
                                    h->atom_xh.as<float4>(), h->atom_xl.as<float4>(), h->bin_start.as<int32_t>(),
                                    h->bin_y.as<float4>(), h->bin_je.as<int2>(), h->n_el, nullptr, nullptr,
                                    h->pairs.as<GmpPair>(), h->cap_pairs, h->cap_keys, d_maxm, d_err, st, h->sm_count,
                                    L, d_cursor, h->nbr_rng.as<int64_t>()),
           "neighbor single pass");
    h->rng_mode = true;
    return GMP_OK;
  }
  GMP_CK(gmp_launch_neighbor_pass(0, h->structs.as<GmpStruct>(), h->grid.as<GmpGrid>(), C, NC, h->cutoff, pos,
                                  h->atom_xh.as<float4>(), h->atom_xl.as<float4>(), h->bin_start.as<int32_t>(),
                                  h->bin_y.as<float4>(), h->bin_je.as<int2>(), h->n_el, h->counts.as<int64_t>(),
                                  nullptr, nullptr, 0, 0, d_maxm,
                                  d_err, st, h->sm_count, L),
         "neighbor count");
  GMP_CK(gmp_exclusive_scan_i64(h->counts.as<int64_t>(), h->nbr_off.as<int64_t>(), NC, h->scan_tmp.p, st, L), "scan");
  if (capture) {
    // capacities fixed at capture time; the fill and compute kernels skip
    // (and flag) centers beyond them
    GMP_CK(gmp_launch_neighbor_pass(2, h->structs.as<GmpStruct>(), h->grid.as<GmpGrid>(), C, NC,
                                    h->cutoff, pos, h->atom_xh.as<float4>(), h->atom_xl.as<float4>(),
                                    h->bin_start.as<int32_t>(), h->bin_y.as<float4>(), h->bin_je.as<int2>(), h->n_el, nullptr,
                                    h->nbr_off.as<int64_t>(), h->pairs.as<GmpPair>(), h->cap_pairs, h->cap_keys,
                                    d_maxm, d_err, st, h->sm_count, L),
           "neighbor fill");
    return GMP_OK;
  }
  GMP_CK(cudaMemcpyAsync(h->h_small, h->nbr_off.as<int64_t>() + NC, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "read P");
  GMP_CK(cudaMemcpyAsync(h->h_small + 1, d_err, 8, cudaMemcpyDeviceToHost, st), "read err");
  GMP_CK(cudaStreamSynchronize(st), "neighbor sync");
  const uint32_t w = (uint32_t)(h->h_small[1] & 0xffffffffu);
  const int maxm = (int)(h->h_small[1] >> 32);
  if (w) {
    GMP_CK(cudaMemsetAsync(d_err, 0, 4, st), "clear err");
    return decode_device_error(h, w);
  }
  h->P = h->h_small[0];
  h->max_m = maxm;
  h->last_nc = NC;
  h->last_gen = h->struct_gen;
  int keys = 32;
  while (keys < maxm) keys <<= 1;
  if ((size_t)keys * 8 > 200 * 1024)
    return fail(h, GMP_ERR_CAPACITY, "a center has " + std::to_string(maxm) + " neighbor images (limit 25600)");
  GMP_CK(h->pairs.ensure(sizeof(GmpPair) * (h->P > 0 ? h->P : 1)), "pairs");
  GMP_CK(gmp_launch_neighbor_pass(sorted ? 2 : 1, h->structs.as<GmpStruct>(), h->grid.as<GmpGrid>(), C, NC,
                                  h->cutoff, pos, h->atom_xh.as<float4>(), h->atom_xl.as<float4>(),
                                  h->bin_start.as<int32_t>(), h->bin_y.as<float4>(), h->bin_je.as<int2>(), h->n_el,
                                  nullptr, h->nbr_off.as<int64_t>(), h->pairs.as<GmpPair>(), h->P, keys, d_maxm,
                                  d_err, st, h->sm_count, L),
         "neighbor fill");
  return GMP_OK;
}

// Binning + exact neighbor lists of every atom into h->pairs / h->nbr_off.
// Synchronises `st` once (to size the pair buffer) unless capturing.
gmp_status build_neighbors(gmp_ctx* h, int32_t S, const double* pos, const int32_t* species,
                           int64_t N, cudaStream_t st, bool sorted, bool capture = false, bool need_csr = false) {
  if (!capture) h->graph_valid = false;  // buffers may move: a captured graph is stale
  GMP_CK(prof_mark(h, 0, true, st), "profile");
  gmp_status r = bin_atoms(h, S, pos, species, N, N, st);
  if (r != GMP_OK) return r;
  const GmpCenters C{h->struct_of.as<int32_t>(), pos, h->atom_xh.as<float4>(), h->atom_xl.as<float4>(),
                     h->atom_rng.as<int4>(), h->atom_y.as<float4>()};
  if ((r = neighbor_lists(h, C, N, pos, st, sorted, capture, !need_csr)) != GMP_OK) return r;
  GMP_CK(prof_mark(h, 0, false, st), "profile");
  return GMP_OK;
}

// Features below this fraction of their FP32 resolution bound are recomputed
// in double-float arithmetic (see gmp_refine.cu and the flag test in
// write_features).
constexpr float kFlagTau = 3e-4f;
// ... and above this fraction of the lower bound l! (2l-1)!! B^2 / 3^l of
// the feature's cancellation-free scale (below it the FP32 value already
// meets the absolute floor; see write_features).
constexpr float kFlagLow = 1e-10f;

// Refinement queues, one per requested order: a pass queues at most one
// entry per (center, order), and a call refines after each pass (derivative
// calls) or once after all of them (features), so a queue holds one entry
// per center and pass.  The flag buffer holds 8 counts, then the queues.
int64_t flag_capacity(const gmp_ctx* h, int64_t N) {
  return (int64_t)std::max<size_t>(h->passes.size(), 1) * N + 1024;
}
unsigned long long* flag_counter(gmp_ctx* h) { return h->flagq.as<unsigned long long>(); }
unsigned long long* flag_queues(gmp_ctx* h) { return h->flagq.as<unsigned long long>() + 8; }

gmpk::KParams base_params(gmp_ctx* h, const PassData& pd, int pass_index, int64_t N) {
  gmpk::KParams K;
  std::memset(&K, 0, sizeof(K));
  K.pass = pd.pass;
  K.N = N;
  K.nbr_beg = h->rng_mode ? h->nbr_rng.as<int64_t>() : h->nbr_off.as<int64_t>();
  K.nbr_end = h->rng_mode ? h->nbr_rng.as<int64_t>() + N : h->nbr_off.as<int64_t>() + 1;
  K.pairs = h->pairs.as<GmpPair>();
  K.counter = reinterpret_cast<int32_t*>(h->scalars.as<uint32_t>() + 2);
  K.flags = flag_queues(h);
  K.flag_count = flag_counter(h);
  K.flag_cap = flag_capacity(h, N);
  K.pair_cap = h->capturing ? h->cap_pairs : h->P;
  K.sig0 = 16 * pass_index;
  K.flag_tau = kFlagTau;
  K.flag_low = kFlagLow;
  return K;
}

// Clears the flag queue (before a call's compute kernels, and after each
// refinement so that the next pass queues only its own flags).
gmp_status reset_flags(gmp_ctx* h, int64_t N, cudaStream_t st) {
  (void)N;
  GMP_CK(cudaMemsetAsync(flag_counter(h), 0, 8 * sizeof(unsigned long long), st), "flag reset");
  return GMP_OK;
}

gmp_status begin_compute(gmp_ctx* h, int64_t N, cudaStream_t st) {
  GMP_CK(h->flagq.ensure(sizeof(unsigned long long) * (8 + (size_t)std::max(h->n_ord_pos, 1) * flag_capacity(h, N))),
         "flags");
  return reset_flags(h, N, st);
}

// The moments of one pass that a derivative kernel reads after the
// refinement (h->mu, [N][pass sigmas][(L+1)^2]).
struct MuTarget {
  float* mu = nullptr;
  int sig0 = 0, nsig = 0, nind = 0;
};
MuTarget pass_moments(gmp_ctx* h, const PassData& pd, int pass_index) {
  MuTarget t;
  t.mu = h->mu.as<float>();
  t.sig0 = 16 * pass_index;
  t.nsig = pd.pass.nsig;
  t.nind = (pd.L + 1) * (pd.L + 1);
  return t;
}

// Double-float recomputation of the flagged features (and, with mt.mu, of
// their moments in the pass's moment buffer).  Centers are the atoms unless
// center_xh / center_xl / center_struct give reference points.
gmp_status refine(gmp_ctx* h, int64_t N, float* features, cudaStream_t st, const float4* center_xh = nullptr,
                  const float4* center_xl = nullptr, const int32_t* center_struct = nullptr,
                  MuTarget mt = MuTarget()) {
  GmpRefine A;
  std::memset(&A, 0, sizeof(A));
  A.queue = flag_queues(h);
  A.count = flag_counter(h);
  A.cap = flag_capacity(h, N);
  for (int l = 0; l < 7; ++l) A.qidx[l] = -1;
  {
    int o = 0;
    for (int l : h->orders)
      if (l >= 0) A.qidx[l] = o++;
  }
  A.n_centers = N;
  A.col_info = h->colinfo.as<int32_t>();
  A.features = features;
  A.F = h->F;
  A.atom_xh = h->atom_xh.as<float4>();
  A.atom_xl = h->atom_xl.as<float4>();
  A.center_xh = center_xh ? center_xh : h->atom_xh.as<float4>();
  A.center_xl = center_xl ? center_xl : h->atom_xl.as<float4>();
  A.center_struct = center_struct ? center_struct : h->struct_of.as<int32_t>();
  A.structs = h->structs.as<GmpStruct>();
  A.nbr_beg = h->rng_mode ? h->nbr_rng.as<int64_t>() : h->nbr_off.as<int64_t>();
  A.nbr_end = h->rng_mode ? h->nbr_rng.as<int64_t>() + N : h->nbr_off.as<int64_t>() + 1;
  A.pairs = h->pairs.as<GmpPair>();
  A.ktab = h->ktab.as<float>();
  A.exp_tab = h->exptab.as<float2>();
  A.nsig_total = (int)std::max<size_t>(h->sigmas.size(), 1);
  A.kmax = h->kmax;
  A.mu_out = mt.mu;
  A.mu_sig0 = mt.sig0;
  A.mu_nsig = mt.nsig;
  A.mu_nind = mt.nind;
  unsigned order_mask = 0;
  for (int l : h->orders)
    if (l >= 0) order_mask |= 1u << l;
  GMP_CK(gmp_launch_refine(A, order_mask, h->sm_count, st, &h->launches), "refine");
  return GMP_OK;
}

// Inputs/outputs either all on the device or all in host memory.
struct Io {
  bool host = false;
  const double* pos = nullptr;
  const int32_t* species = nullptr;
};

gmp_status stage_inputs(gmp_ctx* h, int64_t N, const double* pos, const int32_t* species, Io& io,
                        cudaStream_t st) {
  io.host = !is_device_ptr(pos);
  if (io.host != !is_device_ptr(species))
    return fail(h, GMP_ERR_INVALID_ARG, "pos and species must both be device or both be host pointers");
  if (!io.host) {
    io.pos = pos;
    io.species = species;
    return GMP_OK;
  }
  GMP_CK(h->stage_pos.ensure(sizeof(double) * 3 * N), "stage pos");
  GMP_CK(h->stage_species.ensure(sizeof(int32_t) * N), "stage species");
  GMP_CK(cudaMemcpyAsync(h->stage_pos.p, pos, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, st), "h2d pos");
  GMP_CK(cudaMemcpyAsync(h->stage_species.p, species, sizeof(int32_t) * N, cudaMemcpyHostToDevice, st), "h2d species");
  io.pos = h->stage_pos.as<double>();
  io.species = h->stage_species.as<int32_t>();
  return GMP_OK;
}

gmp_status common_checks(gmp_ctx* h, int32_t S, const int64_t* atom_off, const double* pos,
                         const double* cell, const uint8_t* pbc, const int32_t* species,
                         cudaStream_t st, int64_t& N) {
  if (!h) return GMP_ERR_INVALID_ARG;
  GMP_CK(cudaSetDevice(h->device), "cudaSetDevice");
  gmp_status r = upload_structures(h, S, atom_off, cell, pbc, st);
  if (r != GMP_OK) return r;
  N = atom_off[S];
  if (N > 0 && (!pos || !species)) return fail(h, GMP_ERR_INVALID_ARG, "pos and species are required");
  return GMP_OK;
}

// Replays the captured graph of a call with this key.  Returns
// GMP_ERR_CAPACITY (with the graph dropped) when there is no matching graph
// or the batch outgrew the captured capacities: the caller then runs the
// call eagerly, which re-measures and recaptures.
gmp_status replay_graph(gmp_ctx* h, const std::vector<uintptr_t>& key, cudaStream_t st) {
  if (!h->graph_valid || key != h->graph_key) return GMP_ERR_CAPACITY;
  uint32_t* d_err = h->scalars.as<uint32_t>();
  GMP_CK(cudaGraphLaunch(h->graph_exec, st), "graph launch");
  GMP_CK(cudaMemcpyAsync(h->h_small + 1, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st), "read err");
  GMP_CK(cudaStreamSynchronize(st), "graph sync");
  const uint32_t w = (uint32_t)(h->h_small[1] & 0xffffffffu);
  if (!w) return GMP_OK;
  GMP_CK(cudaMemsetAsync(d_err, 0, 4, st), "clear err");
  if (w & GMP_DEV_CAPACITY) {
    h->graph_valid = false;
    return GMP_ERR_CAPACITY;
  }
  return decode_device_error(h, w);
}

// Captures `seq(true)` (the call's device work without host synchronisation)
// into a CUDA graph for later replays; capacities get 12.5% headroom over
// the eager run that just finished.
template <typename Seq>
gmp_status capture_graph(gmp_ctx* h, const std::vector<uintptr_t>& key, cudaStream_t st, Seq& seq, int64_t N) {
  if (!st) return GMP_OK;  // the legacy default stream cannot be captured
  h->cap_pairs = h->P + h->P / 8 + 4096;
  int keys = 32;
  while (keys < h->max_m + h->max_m / 8 + 8) keys <<= 1;
  if ((size_t)keys * 8 > 200 * 1024) return GMP_OK;  // too large for a fixed capacity: stay eager
  h->cap_keys = keys;
  // every buffer the captured sequence uses exists before the capture
  GMP_CK(h->pairs.ensure(sizeof(GmpPair) * h->cap_pairs), "pairs");
  GMP_CK(h->nbr_rng.ensure(sizeof(int64_t) * 2 * N), "nbr_rng");
  if (h->graph_exec) {
    cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
  }
  GMP_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed), "begin capture");
  h->capturing = true;
  gmp_status r = seq(true);
  h->capturing = false;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (r != GMP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return r;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
  const cudaError_t e2 = cudaGraphInstantiate(&h->graph_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) {
    h->graph_exec = nullptr;
    return cuda_fail(h, e2, "graph instantiate");
  }
  h->graph_key = key;
  h->graph_valid = true;
  return GMP_OK;
}

// Features and Jacobian rows of centers c0 .. c1-1 (all of them for
// gmp_featurize_grad).  The neighbor lists and the work buffers cover the
// whole batch; the compute kernels run over the range only.
gmp_status grad_impl(gmp_ctx* h, int32_t n_struct, const int64_t* atom_off, const double* pos, const double* cell,
                     const uint8_t* pbc, const int32_t* species, int64_t c0, int64_t c1, bool ranged,
                     float* features, int64_t* jac_off, int32_t* jac_j, float* jac, int64_t cap, int64_t* nnz_out,
                     cudaStream_t st) {
  int64_t N = 0;
  gmp_status r = common_checks(h, n_struct, atom_off, pos, cell, pbc, species, st, N);
  if (r != GMP_OK) return r;
  if (!nnz_out) return fail(h, GMP_ERR_INVALID_ARG, "nnz_out is required");
  *nnz_out = 0;
  if (!ranged) c1 = N;
  if (c0 < 0 || c1 < c0 || c1 > N) return fail(h, GMP_ERR_INVALID_ARG, "center range must satisfy 0 <= begin <= end <= N");
  if (N == 0) return GMP_OK;
  if (!jac_off) return fail(h, GMP_ERR_INVALID_ARG, "jac_off is required");
  const int64_t n = c1 - c0;
  const bool whole = c0 == 0 && c1 == N;
  Io io;
  if ((r = stage_inputs(h, N, pos, species, io, st)) != GMP_OK) return r;
  if ((r = build_neighbors(h, n_struct, io.pos, io.species, N, st, true)) != GMP_OK) return r;
  GMP_CK(h->jac_counts.ensure(sizeof(int64_t) * (2 * n + 1)), "jac counts");
  int64_t* cnt = h->jac_counts.as<int64_t>();
  int64_t* joff = cnt + n;
  GMP_CK(h->jac_rows.ensure(sizeof(int32_t) * std::max<int64_t>(h->P, 1)), "jac rows");
  const int64_t* nbeg = h->rng_mode ? h->nbr_rng.as<int64_t>() : h->nbr_off.as<int64_t>();
  const int64_t* nend = h->rng_mode ? h->nbr_rng.as<int64_t>() + N : h->nbr_off.as<int64_t>() + 1;
  GMP_CK(gmp_launch_jacobian_count(n, nbeg + c0, nend + c0, h->pairs.as<GmpPair>(), cnt,
                                   h->jac_rows.as<int32_t>(), st, h->sm_count, &h->launches), "jac count");
  GMP_CK(gmp_exclusive_scan_i64(cnt, joff, n, h->scan_tmp.p, st, &h->launches), "jac scan");
  GMP_CK(cudaMemcpyAsync(h->h_small, joff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "read nnz");
  GMP_CK(cudaStreamSynchronize(st), "jac sync");
  const int64_t nnz = h->h_small[0];
  *nnz_out = nnz;
  if (nnz > cap) return fail(h, GMP_ERR_CAPACITY, "jacobian needs " + std::to_string(nnz) + " rows, cap is " + std::to_string(cap));
  if (nnz > 0 && (!jac_j || !jac)) return fail(h, GMP_ERR_INVALID_ARG, "jac_j and jac are required");
  // features: straight into a device output of the whole batch, else into
  // the [N, F] scratch and the range's rows copied out at the end
  float* jd = jac;
  int32_t* jj = jac_j;
  DevBuf tmp_jac, tmp_jj;
  if (io.host && nnz > 0) {
    GMP_CK(tmp_jac.ensure(sizeof(float) * nnz * h->F * 3), "stage jac");
    GMP_CK(tmp_jj.ensure(sizeof(int32_t) * nnz), "stage jac_j");
    jd = tmp_jac.as<float>();
    jj = tmp_jj.as<int32_t>();
  }
  for (const PassData& pd : h->passes)
    GMP_CK(h->mu.ensure(sizeof(float) * (size_t)N * std::max(pd.pass.nsig, 1) * (pd.L + 1) * (pd.L + 1)), "moments");
  float* fout = (whole && features && !io.host) ? features : nullptr;
  if (!fout) {
    GMP_CK(h->stage_feat.ensure(sizeof(float) * N * h->F), "feature scratch");
    fout = h->stage_feat.as<float>();
  }
  if ((r = begin_compute(h, N, st)) != GMP_OK) return r;
  for (size_t g = 0; g < h->passes.size(); ++g) {
    // forward kernel (features, moments), refinement of the flagged
    // features and their moments, then the Jacobian rows from the moments
    const PassData& pd = h->passes[g];
    gmpk::KParams K = base_params(h, pd, (int)g, N);
    K.N = c1;
    K.center0 = c0;
    K.features = fout;
    K.mu_out = h->mu.as<float>();
    GMP_CK(prof_mark(h, 1, true, st), "profile");
    GMP_CK(launch_compute(pd.L, GMP_KIND_FORWARD, pd.NS, K, pd.fwd, st, h->sm_count, &h->launches), "forward");
    GMP_CK(prof_mark(h, 1, false, st), "profile");
    GMP_CK(prof_mark(h, 3, true, st), "profile");
    if ((r = refine(h, N, fout, st, nullptr, nullptr, nullptr, pass_moments(h, pd, (int)g))) != GMP_OK) return r;
    if ((r = reset_flags(h, N, st)) != GMP_OK) return r;
    GMP_CK(prof_mark(h, 3, false, st), "profile");
    K.features = nullptr;
    K.flags = nullptr;
    K.jac_off = joff;
    K.jac_row = h->jac_rows.as<int32_t>();
    K.jac_j = jj;
    K.jac = jd;
    GMP_CK(prof_mark(h, 2, true, st), "profile");
    GMP_CK(launch_compute(pd.L, GMP_KIND_JACOBIAN, pd.NS, K, pd.jac, st, h->sm_count, &h->launches), "jacobian");
    GMP_CK(prof_mark(h, 2, false, st), "profile");
  }
  const cudaMemcpyKind k_out = io.host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  GMP_CK(cudaMemcpyAsync(jac_off, joff, sizeof(int64_t) * (n + 1), k_out, st), "copy jac_off");
  if (features && fout != features)
    GMP_CK(cudaMemcpyAsync(features, fout + c0 * h->F, sizeof(float) * n * h->F, k_out, st), "copy features");
  if (io.host) {
    if (nnz > 0) {
      GMP_CK(cudaMemcpyAsync(jac, jd, sizeof(float) * nnz * h->F * 3, cudaMemcpyDeviceToHost, st), "d2h jac");
      GMP_CK(cudaMemcpyAsync(jac_j, jj, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, st), "d2h jac_j");
    }
    GMP_CK(cudaStreamSynchronize(st), "sync");
  }
  return GMP_OK;
}

}  // namespace

extern "C" {

gmp_status gmp_create(const gmp_params* p, int device, gmp_handle* out) {
  if (!out) return GMP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!p) return GMP_ERR_INVALID_ARG;
  gmp_ctx* h = new gmp_ctx();
  auto bad = [&](const std::string& m) {
    std::fprintf(stderr, "gmp_create: %s\n", m.c_str());
    gmp_destroy(h);
    return GMP_ERR_INVALID_ARG;
  };
  if (p->n_elements < 1 || !p->n_gauss || !p->gauss_coef || !p->gauss_exp) return bad("density tables missing");
  if (p->n_orders < 1 || p->n_orders > 8 || !p->orders) return bad("orders: 1..8 entries required");
  if (!std::isfinite(p->cutoff)) return bad("cutoff must be finite");
  if (p->flags != GMP_FLAG_NONE) return bad("unknown flags (only GMP_FLAG_NONE is defined)");
  if (!(p->cutoff > 0.0) && !(p->overlap_threshold > 0.0 && std::isfinite(p->overlap_threshold)))
    return bad("cutoff <= 0 needs overlap_threshold > 0");
  h->n_el = p->n_elements;
  int64_t tot = 0;
  for (int e = 0; e < p->n_elements; ++e) {
    if (p->n_gauss[e] < 1 || p->n_gauss[e] > 64) return bad("n_gauss must be in 1..64");
    h->n_gauss.push_back(p->n_gauss[e]);
    h->kmax = std::max(h->kmax, p->n_gauss[e]);
    tot += p->n_gauss[e];
  }
  for (int64_t k = 0; k < tot; ++k) {
    if (!(p->gauss_exp[k] > 0.0) || !std::isfinite(p->gauss_exp[k]) || !std::isfinite(p->gauss_coef[k]))
      return bad("Gaussian exponents must be finite and > 0, coefficients finite");
    h->coef.push_back(p->gauss_coef[k]);
    h->alpha.push_back(p->gauss_exp[k]);
  }
  int lmax = -1;
  bool dens = false;
  for (int o = 0; o < p->n_orders; ++o) {
    int l = p->orders[o];
    if (l < -1 || l > 6) return bad("orders must be in -1..6");
    for (int q = 0; q < o; ++q)
      if (p->orders[q] == l) return bad("repeated order");
    if (l == -1) dens = true;
    else lmax = std::max(lmax, l);
    h->orders.push_back(l);
  }
  if (lmax >= 0) {
    if (p->n_sigmas < 1 || !p->sigmas) return bad("sigmas required");
    for (int s = 0; s < p->n_sigmas; ++s) {
      if (!(p->sigmas[s] > 0.0) || !std::isfinite(p->sigmas[s])) return bad("sigmas must be > 0");
      h->sigmas.push_back(p->sigmas[s]);
    }
  }
  if (h->sigmas.size() > 1024) return bad("at most 1024 sigmas");
  h->cutoff = p->cutoff > 0.0 ? p->cutoff : derived_cutoff(*h, p->overlap_threshold);
  if (!(h->cutoff > 0.0)) return bad("overlap_threshold leaves no neighbor within reach (cutoff 0)");
  h->flags = p->flags;
  const int nsig = (int)h->sigmas.size();
  h->F = (dens ? 1 : 0);
  for (int l : h->orders)
    if (l >= 0) h->F += nsig;
  // feature column of (order slot o, sigma 0); order -1 takes one column
  std::vector<int> col(h->orders.size());
  {
    int c = 0;
    for (size_t o = 0; o < h->orders.size(); ++o) {
      col[o] = c;
      c += h->orders[o] < 0 ? 1 : nsig;
    }
  }
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return bad("cudaSetDevice failed"); }
  h->device = device;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { cudaGetLastError(); return bad("no CUDA device"); }
  h->sm_count = prop.multiProcessorCount;
  const int L = lmax < 0 ? 0 : lmax;
  const int nsplit = lmax < 0 ? 1 : (nsig + 15) / 16;
  const double LOG2E = 1.4426950408889634;
  for (int g = 0; g < nsplit; ++g) {
    PassData pd;
    std::memset(&pd.pass, 0, sizeof(pd.pass));
    const int s0 = g * 16;
    const int ns = lmax < 0 ? 0 : std::min(16, nsig - s0);
    pd.L = L;
    pd.NS = pad_sigmas(std::max(ns, 1));
    GmpPass& P = pd.pass;
    P.lmax = L;
    P.nsig = ns;
    P.nsig_pad = pd.NS;
    P.kmax = h->kmax;
    P.n_el = h->n_el;
    P.want_density = (g == 0 && dens) ? 1 : 0;
    for (int s = 0; s < 16; ++s)
      P.nbeta[s] = s < ns ? (float)(-1.0 / (2.0 * h->sigmas[s0 + s] * h->sigmas[s0 + s])) : 0.0f;
    P.mixed_sign = 0;
    for (double c : h->coef) P.mixed_sign |= (c < 0.0) ? 1 : 0;
    P.F = h->F;
    P.dens_col = -1;
    P.n_ord = 0;
    for (size_t o = 0; o < h->orders.size(); ++o) {
      if (h->orders[o] < 0) {
        P.dens_col = col[o];
        continue;
      }
      if (ns == 0) continue;
      P.ord_l[P.n_ord] = h->orders[o];
      P.ord_col[P.n_ord] = col[o] + s0;
      ++P.n_ord;
    }
    P.ord_dense = 1;
    for (int o = 0; o < P.n_ord; ++o) P.ord_dense &= P.ord_l[o] == o ? 1 : 0;
    const int RB = gmp_rad_block(L), NSB = pd.NS / 4;
    std::vector<float> tab((size_t)h->n_el * NSB * h->kmax * RB * 4, 0.0f);
    int64_t off = 0;
    double rbound[16] = {0};  // per sigma: see GmpPass::jac_exp
    const double rc = h->cutoff;
    for (int e = 0; e < h->n_el; ++e) {
      for (int s = 0; s < ns; ++s) {
        const double sig = h->sigmas[s0 + s];
        const double beta = 1.0 / (2.0 * sig * sig);
        const double Ns = std::pow(2.0 * M_PI * sig * sig, -1.5);
        // each primitive's |A_0| exp(-b r^2) max(1, r)^(L+1) at its largest on
        // [0, rc] (r^2 = (L+1)/(2b) clamped to [1, rc^2]); |A_l| <= |A_0|
        double bsum = 0.0;
        for (int q = 0; q < h->n_gauss[e]; ++q) {
          const double a = h->alpha[off + q], c = h->coef[off + q];
          const double gam = a + beta, b = a * beta / gam;
          const double K0 = std::fabs(c * Ns * std::pow(M_PI / gam, 1.5));
          const double r2 = std::min(std::max((L + 1) / (2.0 * b), 1.0), std::max(rc * rc, 1.0));
          bsum += std::max(K0, K0 * std::exp(-b * r2) * std::pow(r2, 0.5 * (L + 1)));
        }
        rbound[s] = std::max(rbound[s], bsum);
        for (int q = 0; q < h->n_gauss[e]; ++q) {
          const double a = h->alpha[off + q], c = h->coef[off + q];
          const double gam = a + beta;
          const double B = a * beta / gam * LOG2E;
          float* blk = &tab[(((size_t)e * NSB + s / 4) * h->kmax + q) * RB * 4];
          const int u = s % 4;
          blk[u] = (float)B;
          blk[4 + u] = (float)(B - (double)blk[u]);
          const double K0 = c * Ns * std::pow(M_PI / gam, 1.5);
          for (int l = 0; l <= L + 1; ++l) blk[4 * (2 + l) + u] = (float)(K0 * std::pow(a / gam, l));
        }
      }
      off += h->n_gauss[e];
    }
    if (pd.rad.ensure(tab.size() * sizeof(float)) != cudaSuccess ||
        cudaMemcpy(pd.rad.p, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      pd.rad.release();
      return bad("device allocation for tables failed");
    }
    P.rad = pd.rad.as<float>();
    for (int s = 0; s < 16; ++s)
      P.jac_exp[s] = rbound[s] > 0.0 ? (int)std::ceil(std::log2(rbound[s])) : 0;
    h->passes.push_back(std::move(pd));
  }
  {
    std::vector<float> dt((size_t)h->n_el * h->kmax * GMP_DENS_STRIDE, 0.0f);
    int64_t off = 0;
    for (int e = 0; e < h->n_el; ++e) {
      for (int q = 0; q < h->n_gauss[e]; ++q) {
        const double a = h->alpha[off + q];
        const double B = a * LOG2E;
        float* ent = &dt[((size_t)e * h->kmax + q) * GMP_DENS_STRIDE];
        ent[0] = (float)B;
        ent[1] = (float)(B - (double)ent[0]);
        ent[2] = (float)a;
        ent[3] = (float)h->coef[off + q];
        ent[4] = (float)(a - (double)ent[2]);
        ent[5] = (float)(h->coef[off + q] - (double)ent[3]);
      }
      off += h->n_gauss[e];
    }
    if (h->dens.ensure(dt.size() * sizeof(float)) != cudaSuccess ||
        cudaMemcpy(h->dens.p, dt.data(), dt.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      return bad("device allocation for tables failed");
    }
    for (auto& pd : h->passes) pd.pass.dens = h->dens.as<float>();
  }
  {
    // Double-float constants for the refinement kernel: per (element, sigma,
    // primitive) the exponent rate b = alpha beta/g and A_l = c N_s (pi/g)^(3/2)
    // (alpha/g)^l, l = 0..6, each computed in FP64 and split into (hi, lo)
    const int ns = std::max<int>((int)h->sigmas.size(), 1);
    std::vector<float> kt((size_t)h->n_el * ns * h->kmax * 16, 0.0f);
    auto split = [](double v, float* out) {
      out[0] = (float)v;
      out[1] = (float)(v - (double)out[0]);
    };
    int64_t off = 0;
    for (int e = 0; e < h->n_el; ++e) {
      for (int s = 0; s < (int)h->sigmas.size(); ++s) {
        const double sig = h->sigmas[s];
        const double beta = 1.0 / (2.0 * sig * sig);
        const double Ns = std::pow(2.0 * M_PI * sig * sig, -1.5);
        for (int q = 0; q < h->n_gauss[e]; ++q) {
          const double a = h->alpha[off + q], c = h->coef[off + q];
          const double gam = a + beta;
          float* ent = &kt[(((size_t)e * ns + s) * h->kmax + q) * 16];
          split(a * beta / gam, ent);
          const double K0 = c * Ns * std::pow(M_PI / gam, 1.5);
          for (int l = 0; l <= 6; ++l) split(K0 * std::pow(a / gam, l), ent + 2 + 2 * l);
        }
      }
      off += h->n_gauss[e];
    }
    // feature column -> (order << 16) | sigma for the refinement kernel
    std::vector<int32_t> ci((size_t)std::max(h->F, 1), -1);
    for (size_t o = 0; o < h->orders.size(); ++o)
      if (h->orders[o] >= 0)
        for (int s = 0; s < (int)h->sigmas.size(); ++s) ci[col[o] + s] = (h->orders[o] << 16) | s;
    h->n_ord_pos = 0;
    for (int l : h->orders) h->n_ord_pos += l >= 0 ? 1 : 0;
    float et[128];
    for (int j = 0; j < 64; ++j) split(std::exp2(-j / 64.0), et + 2 * j);
    if (h->exptab.ensure(sizeof(et)) != cudaSuccess ||
        cudaMemcpy(h->exptab.p, et, sizeof(et), cudaMemcpyHostToDevice) != cudaSuccess ||
        h->ktab.ensure(kt.size() * sizeof(float)) != cudaSuccess ||
        cudaMemcpy(h->ktab.p, kt.data(), kt.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        h->colinfo.ensure(ci.size() * sizeof(int32_t)) != cudaSuccess ||
        cudaMemcpy(h->colinfo.p, ci.data(), ci.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        h->scalars.ensure(64) != cudaSuccess || cudaMemset(h->scalars.p, 0, 64) != cudaSuccess) {
      cudaGetLastError();
      return bad("device allocation for tables failed");
    }
    for (auto& pd : h->passes) pd.pass.exp_tab = h->exptab.as<float2>();
  }
  if (cudaMallocHost((void**)&h->h_small, 64) != cudaSuccess) { cudaGetLastError(); return bad("pinned alloc failed"); }
  if (cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming) != cudaSuccess) { cudaGetLastError(); return bad("event"); }
  if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_feat, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return bad("stream/event creation failed");
  }
  *out = h;
  return GMP_OK;
}

gmp_status gmp_cutoff(gmp_handle h, double* cutoff) {
  if (!h || !cutoff) return GMP_ERR_INVALID_ARG;
  *cutoff = h->cutoff;
  return GMP_OK;
}

gmp_status gmp_num_features(gmp_handle h, int32_t* F) {
  if (!h || !F) return GMP_ERR_INVALID_ARG;
  *F = h->F;
  return GMP_OK;
}

gmp_status gmp_featurize(gmp_handle h, int32_t n_struct, const int64_t* atom_off, const double* pos,
                         const double* cell, const uint8_t* pbc, const int32_t* species, float* features,
                         void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int64_t N = 0;
  gmp_status r = common_checks(h, n_struct, atom_off, pos, cell, pbc, species, st, N);
  if (r != GMP_OK) return r;
  if (N == 0) return GMP_OK;
  if (!features) return fail(h, GMP_ERR_INVALID_ARG, "features is required");
  Io io;
  if ((r = stage_inputs(h, N, pos, species, io, st)) != GMP_OK) return r;
  float* feat = features;
  if (io.host) {
    GMP_CK(h->stage_feat.ensure(sizeof(float) * N * h->F), "stage features");
    feat = h->stage_feat.as<float>();
  } else if (!is_device_ptr(features)) {
    return fail(h, GMP_ERR_INVALID_ARG, "features must be a device pointer when inputs are");
  }
  const bool use_graph = h->graph_on && !io.host;
  const std::vector<uintptr_t> key = {0, (uintptr_t)io.pos, (uintptr_t)io.species, (uintptr_t)feat, (uintptr_t)st,
                                      (uintptr_t)N, (uintptr_t)n_struct, (uintptr_t)h->struct_gen};
  if (use_graph && (r = replay_graph(h, key, st)) != GMP_ERR_CAPACITY) return r;
  auto seq = [&](bool capture) -> gmp_status {
    gmp_status q = build_neighbors(h, n_struct, io.pos, io.species, N, st, false, capture);
    if (q != GMP_OK) return q;
    if ((q = begin_compute(h, N, st)) != GMP_OK) return q;
    GMP_CK(prof_mark(h, 1, true, st), "profile");
    for (size_t g = 0; g < h->passes.size(); ++g) {
      gmpk::KParams K = base_params(h, h->passes[g], (int)g, N);
      K.features = feat;
      GMP_CK(launch_compute(h->passes[g].L, GMP_KIND_FORWARD, h->passes[g].NS, K, h->passes[g].fwd, st,
                            h->sm_count, &h->launches),
             "forward");
    }
    GMP_CK(prof_mark(h, 1, false, st), "profile");
    GMP_CK(prof_mark(h, 3, true, st), "profile");
    if ((q = refine(h, N, feat, st)) != GMP_OK) return q;
    GMP_CK(prof_mark(h, 3, false, st), "profile");
    return GMP_OK;
  };
  if ((r = seq(false)) != GMP_OK) return r;
  if (use_graph && (r = capture_graph(h, key, st, seq, N)) != GMP_OK) return r;
  if (io.host) {
    GMP_CK(cudaMemcpyAsync(features, feat, sizeof(float) * N * h->F, cudaMemcpyDeviceToHost, st), "d2h features");
    GMP_CK(cudaStreamSynchronize(st), "sync");
  }
  return GMP_OK;
}

static gmp_status vjp_impl(gmp_handle h, int32_t n_struct, const int64_t* atom_off, const double* pos,
                           const double* cell, const uint8_t* pbc, const int32_t* species,
                           const float* grad_feat, float* features, float* grad_pos, double* virial,
                           void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int64_t N = 0;
  gmp_status r = common_checks(h, n_struct, atom_off, pos, cell, pbc, species, st, N);
  if (r != GMP_OK) return r;
  if (N == 0) {
    if (virial) {
      if (is_device_ptr(virial)) {
        GMP_CK(cudaMemsetAsync(virial, 0, sizeof(double) * 9 * n_struct, st), "zero virial");
      } else {
        std::memset(virial, 0, sizeof(double) * 9 * n_struct);
      }
    }
    return GMP_OK;
  }
  if (!grad_feat || !grad_pos) return fail(h, GMP_ERR_INVALID_ARG, "grad_feat and grad_pos are required");
  Io io;
  if ((r = stage_inputs(h, N, pos, species, io, st)) != GMP_OK) return r;
  const float* gf = grad_feat;
  float* feat = features;
  float* gp = grad_pos;
  double* vir = virial;
  if (virial && io.host) {
    GMP_CK(h->stage_virial.ensure(sizeof(double) * 9 * n_struct), "stage virial");
    vir = h->stage_virial.as<double>();
  } else if (virial && !is_device_ptr(virial)) {
    return fail(h, GMP_ERR_INVALID_ARG, "virial must be a device pointer when inputs are");
  }
  if (io.host) {
    // the upstream gradient goes up on the side stream while the neighbor
    // lists and the forward kernel run; the backward kernel waits for it
    GMP_CK(h->stage_gradf.ensure(sizeof(float) * N * h->F), "stage grad_feat");
    GMP_CK(cudaEventRecord(h->ev_in, st), "event");
    GMP_CK(cudaStreamWaitEvent(h->side, h->ev_in, 0), "side wait");
    GMP_CK(cudaMemcpyAsync(h->stage_gradf.p, grad_feat, sizeof(float) * N * h->F, cudaMemcpyHostToDevice, h->side),
           "h2d grad_feat");
    GMP_CK(cudaEventRecord(h->ev_in, h->side), "event");
    gf = h->stage_gradf.as<float>();
    if (features) {
      GMP_CK(h->stage_feat.ensure(sizeof(float) * N * h->F), "stage features");
      feat = h->stage_feat.as<float>();
    }
    GMP_CK(h->stage_gradp.ensure(sizeof(float) * N * 3), "stage grad_pos");
    gp = h->stage_gradp.as<float>();
  }
  const bool use_graph = h->graph_on && !io.host;
  const std::vector<uintptr_t> key = {1, (uintptr_t)io.pos, (uintptr_t)io.species, (uintptr_t)gf, (uintptr_t)feat,
                                      (uintptr_t)gp, (uintptr_t)vir, (uintptr_t)st, (uintptr_t)N,
                                      (uintptr_t)n_struct, (uintptr_t)h->struct_gen};
  if (use_graph && (r = replay_graph(h, key, st)) != GMP_ERR_CAPACITY) return r;
  // buffers first (no allocation may happen while a graph is captured)
  GMP_CK(h->grad_acc.ensure(sizeof(double) * 3 * N), "grad_acc");
  GMP_CK(h->gbins.ensure(sizeof(unsigned long long) * 3 * gmpk::kGradBins * N), "gradient bins");
  GMP_CK(h->own.ensure(sizeof(double) * 3 * N), "own");
  if (vir) GMP_CK(h->vir_c.ensure(sizeof(double) * 9 * N), "vir_c");
  for (const PassData& pd : h->passes)
    GMP_CK(h->mu.ensure(sizeof(float) * (size_t)N * std::max(pd.pass.nsig, 1) * (pd.L + 1) * (pd.L + 1)), "moments");
  if (!feat) GMP_CK(h->stage_feat.ensure(sizeof(float) * N * h->F), "feature scratch");
  // No float atomics in the VJP: the backward kernel adds each pair's
  // gradient, exactly, into integer fixed-point bins of its neighbor atom
  // and writes each center's own term; a finishing kernel combines them in
  // a fixed order.  Results are bit-reproducible.
  auto vjp_begin = [&](gmpk::KParams& K) -> gmp_status {
    K.gbins = h->gbins.as<unsigned long long>();
    K.own = h->own.as<double>();
    K.vir_c = vir ? h->vir_c.as<double>() : nullptr;
    GMP_CK(cudaMemsetAsync(K.gbins, 0, sizeof(unsigned long long) * 3 * gmpk::kGradBins * N, st), "memset bins");
    GMP_CK(cudaMemsetAsync(K.own, 0, sizeof(double) * 3 * N, st), "memset own");
    if (vir) GMP_CK(cudaMemsetAsync(K.vir_c, 0, sizeof(double) * 9 * N, st), "memset vir_c");
    return GMP_OK;
  };
  auto vjp_end = [&](const gmpk::KParams& K) -> gmp_status {
    GMP_CK(gmp_launch_grad_bins_finish(N, K.gbins, K.own, h->grad_acc.as<double>(), st, h->sm_count, &h->launches),
           "gradient sums");
    if (vir)
      GMP_CK(gmp_launch_virial_reduce(n_struct, h->atom_off.as<int64_t>(), K.vir_c, vir, st, h->sm_count,
                                      &h->launches),
             "virial sums");
    return GMP_OK;
  };
  auto seq = [&](bool capture) -> gmp_status {
  gmp_status q = build_neighbors(h, n_struct, io.pos, io.species, N, st, false, capture);
  if (q != GMP_OK) return q;
  GMP_CK(cudaMemsetAsync(h->grad_acc.p, 0, sizeof(double) * 3 * N, st), "memset grad");
  if (vir) GMP_CK(cudaMemsetAsync(vir, 0, sizeof(double) * 9 * n_struct, st), "memset virial");
  if ((q = begin_compute(h, N, st)) != GMP_OK) return q;
  bool refined = false, waited = false, pending = false;
  const bool overlap = io.host && !capture;
  for (size_t g = 0; g < h->passes.size(); ++g) {
    const PassData& pd = h->passes[g];
    // forward kernel (features + moments), then the backward kernel reading
    // the moments (or one fused kernel, if the autotuner chose it)
    float* fout = feat ? feat : h->stage_feat.as<float>();
    gmpk::KParams K = base_params(h, pd, (int)g, N);
    K.features = fout;
    // (tables with coefficients of both signs take the split kernels: their
    // backward kernel computes the exponentials exactly, see radial4x)
    const bool fused = pd.vjp_fused && !vir && !pd.pass.mixed_sign;
    if (overlap && !waited && fused) {
      GMP_CK(cudaStreamWaitEvent(st, h->ev_in, 0), "wait grad_feat");
      waited = true;
    }
    if (fused) {
      K.grad_feat = gf;
      K.grad_acc = h->grad_acc.as<double>();
      GMP_CK(prof_mark(h, 2, true, st), "profile");
      if ((q = vjp_begin(K)) != GMP_OK) return q;
      GMP_CK(launch_compute(pd.L, GMP_KIND_VJP, pd.NS, K, pd.fused, st, h->sm_count, &h->launches), "vjp");
      if ((q = vjp_end(K)) != GMP_OK) return q;
      GMP_CK(prof_mark(h, 2, false, st), "profile");
      pending = true;
      continue;
    }
    K.mu_out = h->mu.as<float>();
    GMP_CK(prof_mark(h, 1, true, st), "profile");
    GMP_CK(launch_compute(pd.L, GMP_KIND_FORWARD, pd.NS, K, pd.fwd, st, h->sm_count, &h->launches), "forward");
    GMP_CK(prof_mark(h, 1, false, st), "profile");
    // refinement of the flagged features (this pass's, and any a fused pass
    // left); the backward kernel then reads the refined moments
    GMP_CK(prof_mark(h, 3, true, st), "profile");
    if ((q = refine(h, N, fout, st, nullptr, nullptr, nullptr, pass_moments(h, pd, (int)g))) != GMP_OK) return q;
    if ((q = reset_flags(h, N, st)) != GMP_OK) return q;
    GMP_CK(prof_mark(h, 3, false, st), "profile");
    pending = false;
    if (g + 1 == h->passes.size()) {
      // every feature is final once the last forward kernel and its
      // refinement ran: the download overlaps the backward kernel
      refined = true;
      if (overlap && features) {
        GMP_CK(cudaEventRecord(h->ev_feat, st), "event");
        GMP_CK(cudaStreamWaitEvent(h->side, h->ev_feat, 0), "side wait");
        GMP_CK(cudaMemcpyAsync(features, feat, sizeof(float) * N * h->F, cudaMemcpyDeviceToHost, h->side),
               "d2h features");
      }
    }
    if (overlap && !waited) {
      GMP_CK(cudaStreamWaitEvent(st, h->ev_in, 0), "wait grad_feat");
      waited = true;
    }
    K.features = nullptr;
    K.flags = nullptr;
    K.grad_feat = gf;
    K.grad_acc = h->grad_acc.as<double>();
    K.virial = vir;
    K.center_struct = h->struct_of.as<int32_t>();
    GMP_CK(prof_mark(h, 2, true, st), "profile");
    if ((q = vjp_begin(K)) != GMP_OK) return q;
    GMP_CK(launch_compute(pd.L, vir ? GMP_KIND_BACKWARD_VIRIAL : GMP_KIND_BACKWARD, pd.NS, K, pd.bwd, st,
                          h->sm_count, &h->launches),
           "backward");
    if ((q = vjp_end(K)) != GMP_OK) return q;
    GMP_CK(prof_mark(h, 2, false, st), "profile");
  }
  if (feat && pending) {
    GMP_CK(prof_mark(h, 3, true, st), "profile");
    if ((q = refine(h, N, feat, st)) != GMP_OK) return q;
    GMP_CK(prof_mark(h, 3, false, st), "profile");
  }
  GMP_CK(gmp_launch_grad_finish(N, h->grad_acc.as<double>(), gp, st, &h->launches), "grad finish");
  if (overlap && features && !refined) {  // fused path: features final only now
    GMP_CK(cudaEventRecord(h->ev_feat, st), "event");
    GMP_CK(cudaStreamWaitEvent(h->side, h->ev_feat, 0), "side wait");
    GMP_CK(cudaMemcpyAsync(features, feat, sizeof(float) * N * h->F, cudaMemcpyDeviceToHost, h->side),
           "d2h features");
  }
  return GMP_OK;
  };
  if ((r = seq(false)) != GMP_OK) {
    if (io.host) cudaStreamSynchronize(h->side);  // no copy may outlive the call
    return r;
  }
  if (use_graph && (r = capture_graph(h, key, st, seq, N)) != GMP_OK) return r;
  if (io.host) {
    GMP_CK(cudaMemcpyAsync(grad_pos, gp, sizeof(float) * N * 3, cudaMemcpyDeviceToHost, st), "d2h grad");
    if (virial)
      GMP_CK(cudaMemcpyAsync(virial, vir, sizeof(double) * 9 * n_struct, cudaMemcpyDeviceToHost, st), "d2h virial");
    GMP_CK(cudaEventRecord(h->ev_out, h->side), "event");
    GMP_CK(cudaStreamWaitEvent(st, h->ev_out, 0), "wait d2h features");
    GMP_CK(cudaStreamSynchronize(st), "sync");
  }
  return GMP_OK;
}

gmp_status gmp_featurize_vjp(gmp_handle h, int32_t n_struct, const int64_t* atom_off, const double* pos,
                             const double* cell, const uint8_t* pbc, const int32_t* species,
                             const float* grad_feat, float* features, float* grad_pos, void* stream) {
  return vjp_impl(h, n_struct, atom_off, pos, cell, pbc, species, grad_feat, features, grad_pos, nullptr, stream);
}

gmp_status gmp_featurize_vjp_virial(gmp_handle h, int32_t n_struct, const int64_t* atom_off, const double* pos,
                                    const double* cell, const uint8_t* pbc, const int32_t* species,
                                    const float* grad_feat, float* features, float* grad_pos, double* virial,
                                    void* stream) {
  if (!virial) return fail(h, GMP_ERR_INVALID_ARG, "virial is required");
  return vjp_impl(h, n_struct, atom_off, pos, cell, pbc, species, grad_feat, features, grad_pos, virial, stream);
}

gmp_status gmp_featurize_grad(gmp_handle h, int32_t n_struct, const int64_t* atom_off, const double* pos,
                                  const double* cell, const uint8_t* pbc, const int32_t* species, float* features,
                                  int64_t* jac_off, int32_t* jac_j, float* jac, int64_t cap, int64_t* nnz_out,
                                  void* stream) {
  return grad_impl(h, n_struct, atom_off, pos, cell, pbc, species, 0, 0, false, features, jac_off, jac_j, jac, cap,
                   nnz_out, (cudaStream_t)stream);
}

gmp_status gmp_featurize_grad_centers(gmp_handle h, int32_t n_struct, const int64_t* atom_off, const double* pos,
                                      const double* cell, const uint8_t* pbc, const int32_t* species,
                                      int64_t center_begin, int64_t center_end, float* features, int64_t* jac_off,
                                      int32_t* jac_j, float* jac, int64_t cap, int64_t* nnz_out, void* stream) {
  return grad_impl(h, n_struct, atom_off, pos, cell, pbc, species, center_begin, center_end, true, features, jac_off,
                   jac_j, jac, cap, nnz_out, (cudaStream_t)stream);
}

gmp_status gmp_featurize_points(gmp_handle h, int32_t n_struct, const int64_t* atom_off, const double* pos,
                                const double* cell, const uint8_t* pbc, const int32_t* species,
                                const int64_t* point_off, const double* points, float* features, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int64_t N = 0;
  gmp_status r = common_checks(h, n_struct, atom_off, pos, cell, pbc, species, st, N);
  if (r != GMP_OK) return r;
  if (!point_off || point_off[0] != 0) return fail(h, GMP_ERR_INVALID_ARG, "point_off with point_off[0] = 0 is required");
  for (int s = 0; s < n_struct; ++s)
    if (point_off[s + 1] < point_off[s]) return fail(h, GMP_ERR_INVALID_ARG, "point_off must be non-decreasing");
  const int64_t NP = point_off[n_struct];
  if (NP > (int64_t)INT32_MAX / 2) return fail(h, GMP_ERR_INVALID_ARG, "too many points");
  if (NP == 0) return GMP_OK;
  if (!points || !features) return fail(h, GMP_ERR_INVALID_ARG, "points and features are required");
  const bool host = !is_device_ptr(points);
  if (host != !is_device_ptr(features)) return fail(h, GMP_ERR_INVALID_ARG, "points and features must both be device or both host pointers");
  if (N > 0 && host != !is_device_ptr(pos)) return fail(h, GMP_ERR_INVALID_ARG, "points and pos must both be device or both host pointers");
  h->graph_valid = false;  // shares the neighbor buffers with the graph-captured calls
  Io io;
  if (N > 0 && (r = stage_inputs(h, N, pos, species, io, st)) != GMP_OK) return r;
  const double* pts = points;
  float* feat = features;
  if (host) {
    GMP_CK(h->stage_pts.ensure(sizeof(double) * 3 * NP), "stage points");
    GMP_CK(cudaMemcpyAsync(h->stage_pts.p, points, sizeof(double) * 3 * NP, cudaMemcpyHostToDevice, st), "h2d points");
    pts = h->stage_pts.as<double>();
    GMP_CK(h->stage_feat.ensure(sizeof(float) * NP * h->F), "stage features");
    feat = h->stage_feat.as<float>();
  }
  if (N == 0) {
    GMP_CK(cudaMemsetAsync(feat, 0, sizeof(float) * NP * h->F, st), "zero features");
  } else {
    GMP_CK(h->pt_off.ensure(sizeof(int64_t) * (n_struct + 1)), "point_off");
    GMP_CK(h->pt_struct.ensure(sizeof(int32_t) * NP), "point struct");
    GMP_CK(h->pt_xh.ensure(sizeof(float4) * NP), "point xh");
    GMP_CK(h->pt_xl.ensure(sizeof(float4) * NP), "point xl");
    GMP_CK(h->pt_rng.ensure(sizeof(int4) * NP), "point ranges");
    GMP_CK(h->pt_y.ensure(sizeof(float4) * NP), "point y");
    GMP_CK(cudaMemcpyAsync(h->pt_off.p, point_off, sizeof(int64_t) * (n_struct + 1), cudaMemcpyHostToDevice, st),
           "upload point_off");
    GMP_CK(gmp_launch_struct_of(h->pt_off.as<int64_t>(), n_struct, h->pt_struct.as<int32_t>(), st, &h->launches),
           "point struct");
    GMP_CK(prof_mark(h, 0, true, st), "profile");
    if ((r = bin_atoms(h, n_struct, io.pos, io.species, N, NP, st)) != GMP_OK) return r;
    GMP_CK(gmp_launch_point_prepare(h->structs.as<GmpStruct>(), h->grid.as<GmpGrid>(), h->pt_struct.as<int32_t>(), NP,
                                    pts, io.pos, h->pt_xh.as<float4>(), h->pt_xl.as<float4>(), h->pt_rng.as<int4>(),
                                    h->pt_y.as<float4>(), h->scalars.as<uint32_t>(), st, h->sm_count, &h->launches),
           "point prepare");
    const GmpCenters C{h->pt_struct.as<int32_t>(), pts, h->pt_xh.as<float4>(), h->pt_xl.as<float4>(),
                       h->pt_rng.as<int4>(), h->pt_y.as<float4>()};
    h->last_nc = -1;  // the capacities below describe the points, not the atoms
    if ((r = neighbor_lists(h, C, NP, io.pos, st, false, false)) != GMP_OK) return r;
    h->last_nc = -1;
    GMP_CK(prof_mark(h, 0, false, st), "profile");
    if ((r = begin_compute(h, NP, st)) != GMP_OK) return r;
    GMP_CK(prof_mark(h, 1, true, st), "profile");
    for (size_t g = 0; g < h->passes.size(); ++g) {
      gmpk::KParams K = base_params(h, h->passes[g], (int)g, NP);
      K.features = feat;
      GMP_CK(launch_compute(h->passes[g].L, GMP_KIND_FORWARD, h->passes[g].NS, K, h->passes[g].fwd, st,
                            h->sm_count, &h->launches),
             "forward");
    }
    GMP_CK(prof_mark(h, 1, false, st), "profile");
    GMP_CK(prof_mark(h, 3, true, st), "profile");
    if ((r = refine(h, NP, feat, st, h->pt_xh.as<float4>(), h->pt_xl.as<float4>(), h->pt_struct.as<int32_t>())) != GMP_OK) return r;
    GMP_CK(prof_mark(h, 3, false, st), "profile");
  }
  if (host) {
    GMP_CK(cudaMemcpyAsync(features, feat, sizeof(float) * NP * h->F, cudaMemcpyDeviceToHost, st), "d2h features");
    GMP_CK(cudaStreamSynchronize(st), "sync");
  }
  return GMP_OK;
}

gmp_status gmp_neighbors(gmp_handle h, int32_t n_struct, const int64_t* atom_off, const double* pos,
                         const double* cell, const uint8_t* pbc, const int32_t* species, int64_t* nbr_off,
                         int32_t* nbr_j, int32_t* nbr_shift, int64_t cap, int64_t* nnz_out, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int64_t N = 0;
  gmp_status r = common_checks(h, n_struct, atom_off, pos, cell, pbc, species, st, N);
  if (r != GMP_OK) return r;
  if (!nnz_out) return fail(h, GMP_ERR_INVALID_ARG, "nnz_out is required");
  *nnz_out = 0;
  if (N == 0) return GMP_OK;
  if (!nbr_off) return fail(h, GMP_ERR_INVALID_ARG, "nbr_off is required");
  Io io;
  if ((r = stage_inputs(h, N, pos, species, io, st)) != GMP_OK) return r;
  if ((r = build_neighbors(h, n_struct, io.pos, io.species, N, st, true, false, true)) != GMP_OK) return r;
  *nnz_out = h->P;
  if (h->P > cap) return fail(h, GMP_ERR_CAPACITY, "neighbor list needs " + std::to_string(h->P) + " entries");
  if (h->P > 0 && (!nbr_j || !nbr_shift)) return fail(h, GMP_ERR_INVALID_ARG, "nbr_j and nbr_shift are required");
  DevBuf tj, ts;
  int32_t* dj = nbr_j;
  int32_t* ds = nbr_shift;
  if (io.host) {
    GMP_CK(tj.ensure(sizeof(int32_t) * (h->P + 1)), "stage nbr_j");
    GMP_CK(ts.ensure(sizeof(int32_t) * 3 * (h->P + 1)), "stage nbr_shift");
    dj = tj.as<int32_t>();
    ds = ts.as<int32_t>();
  }
  GMP_CK(gmp_launch_unpack_neighbors(h->P, h->pairs.as<GmpPair>(), dj, ds, st, &h->launches), "unpack");
  const cudaMemcpyKind k = io.host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  GMP_CK(cudaMemcpyAsync(nbr_off, h->nbr_off.p, sizeof(int64_t) * (N + 1), k, st), "copy nbr_off");
  if (io.host) {
    GMP_CK(cudaMemcpyAsync(nbr_j, dj, sizeof(int32_t) * h->P, cudaMemcpyDeviceToHost, st), "d2h nbr_j");
    GMP_CK(cudaMemcpyAsync(nbr_shift, ds, sizeof(int32_t) * 3 * h->P, cudaMemcpyDeviceToHost, st), "d2h shift");
    GMP_CK(cudaStreamSynchronize(st), "sync");
    tj.release();
    ts.release();
  }
  return GMP_OK;
}

gmp_status gmp_tune(gmp_handle h, int32_t n_struct, const int64_t* atom_off, const double* pos,
                    const double* cell, const uint8_t* pbc, const int32_t* species, int32_t reps,
                    int64_t* pairs_out, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int64_t N = 0;
  gmp_status r = common_checks(h, n_struct, atom_off, pos, cell, pbc, species, st, N);
  if (r != GMP_OK) return r;
  if (pairs_out) *pairs_out = 0;
  if (N == 0) return GMP_OK;
  if (reps < 1) reps = 1;
  Io io;
  if ((r = stage_inputs(h, N, pos, species, io, st)) != GMP_OK) return r;
  if ((r = build_neighbors(h, n_struct, io.pos, io.species, N, st, false)) != GMP_OK) return r;
  if (pairs_out) *pairs_out = h->P;
  GMP_CK(h->stage_feat.ensure(sizeof(float) * N * h->F), "tune features");
  GMP_CK(h->stage_gradf.ensure(sizeof(float) * N * h->F), "tune grad");
  GMP_CK(cudaMemsetAsync(h->stage_gradf.p, 0, sizeof(float) * N * h->F, st), "tune grad zero");
  GMP_CK(h->grad_acc.ensure(sizeof(double) * 3 * N), "grad_acc");
  cudaEvent_t e0, e1;
  GMP_CK(cudaEventCreate(&e0), "event");
  GMP_CK(cudaEventCreate(&e1), "event");
  auto timed = [&](int kind, const PassData& pd, const gmpk::KParams& K, GmpShape shape, float* ms) -> cudaError_t {
    cudaError_t e = launch_compute(pd.L, kind, pd.NS, K, shape, st, h->sm_count, &h->launches);  // warm-up
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(e0, st)) != cudaSuccess) return e;
    for (int k = 0; k < reps; ++k)
      if ((e = launch_compute(pd.L, kind, pd.NS, K, shape, st, h->sm_count, &h->launches)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(e1, st)) != cudaSuccess) return e;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
    if ((e = cudaEventElapsedTime(ms, e0, e1)) != cudaSuccess) return e;
    *ms /= reps;
    return cudaSuccess;
  };
  gmp_status out = GMP_OK;
  for (size_t g = 0; g < h->passes.size() && out == GMP_OK; ++g) {
    PassData& pd = h->passes[g];
    const size_t mu_floats = (size_t)N * std::max(pd.pass.nsig, 1) * (pd.L + 1) * (pd.L + 1);
    if (h->mu.ensure(sizeof(float) * mu_floats) != cudaSuccess ||
        (out = begin_compute(h, N, st)) != GMP_OK) {
      if (out == GMP_OK) out = fail(h, GMP_ERR_OOM, "tune buffers");
      break;
    }
    gmpk::KParams K = base_params(h, pd, (int)g, N);
    K.flags = nullptr;
    K.features = h->stage_feat.as<float>();
    K.mu_out = h->mu.as<float>();
    float best_f = 1e30f, t = 0.0f;
    GmpShape fwd_best = pd.fwd;
    for (int tile : {16, 32})
      for (int warps : {4, 8, 16}) {
        cudaError_t e = timed(GMP_KIND_FORWARD, pd, K, GmpShape{tile, warps}, &t);
        if (e != cudaSuccess) { out = cuda_fail(h, e, "tune forward"); break; }
        if (t < best_f) { best_f = t; fwd_best = GmpShape{tile, warps}; }
      }
    if (out != GMP_OK) break;
    // moments for the backward candidates
    if (cudaError_t e = launch_compute(pd.L, GMP_KIND_FORWARD, pd.NS, K, fwd_best, st, h->sm_count, &h->launches)) {
      out = cuda_fail(h, e, "tune forward");
      break;
    }
    gmpk::KParams Kb = K;
    Kb.features = nullptr;
    Kb.grad_feat = h->stage_gradf.as<float>();
    Kb.grad_acc = h->grad_acc.as<double>();
    float best_b = 1e30f;
    GmpShape bwd_best = pd.bwd;
    for (int warps : {4, 6, 12}) {
      cudaError_t e = timed(GMP_KIND_BACKWARD, pd, Kb, GmpShape{16, warps}, &t);
      if (e != cudaSuccess) { out = cuda_fail(h, e, "tune backward"); break; }
      if (t < best_b) { best_b = t; bwd_best = GmpShape{16, warps}; }
    }
    if (out != GMP_OK) break;
    gmpk::KParams Kv = Kb;
    Kv.features = h->stage_feat.as<float>();
    Kv.mu_out = nullptr;
    float best_v = 1e30f;
    GmpShape fused_best = pd.fused;
    for (int warps : {4, 8}) {
      cudaError_t e = timed(GMP_KIND_VJP, pd, Kv, GmpShape{16, warps}, &t);
      if (e != cudaSuccess) { out = cuda_fail(h, e, "tune fused"); break; }
      if (t < best_v) { best_v = t; fused_best = GmpShape{16, warps}; }
    }
    if (out != GMP_OK) break;
    pd.fwd = fwd_best;
    pd.bwd = bwd_best;
    pd.fused = fused_best;
    pd.vjp_fused = (best_v < best_f + best_b && !pd.pass.mixed_sign) ? 1 : 0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return out;
}

gmp_status gmp_set_graph(gmp_handle h, int enable) {
  if (!h) return GMP_ERR_INVALID_ARG;
  h->graph_on = enable != 0;
  h->graph_valid = false;
  return GMP_OK;
}

gmp_status gmp_tuning_get(gmp_handle h, int32_t* values, int32_t n) {
  if (!h || !values) return GMP_ERR_INVALID_ARG;
  const int need = 6 * (int)h->passes.size();
  if (n < need) return fail(h, GMP_ERR_CAPACITY, "tuning record needs " + std::to_string(need) + " values");
  for (size_t g = 0; g < h->passes.size(); ++g) {
    const PassData& pd = h->passes[g];
    int32_t* v = values + 6 * g;
    v[0] = pd.fwd.tile; v[1] = pd.fwd.warps; v[2] = pd.bwd.warps;
    v[3] = pd.vjp_fused; v[4] = pd.fused.warps; v[5] = pd.jac.warps;
  }
  return GMP_OK;
}

gmp_status gmp_tuning_set(gmp_handle h, const int32_t* values, int32_t n) {
  if (!h || !values) return GMP_ERR_INVALID_ARG;
  if (n != 6 * (int)h->passes.size()) return fail(h, GMP_ERR_INVALID_ARG, "tuning record has the wrong length");
  for (size_t g = 0; g < h->passes.size(); ++g) {
    const int32_t* v = values + 6 * g;
    if ((v[0] != 16 && v[0] != 32) || v[1] < 0 || v[1] > 16 || v[2] < 0 || v[2] > 16 || (v[3] != 0 && v[3] != 1) ||
        v[4] < 0 || v[4] > 16 || v[5] < 0 || v[5] > 16)
      return fail(h, GMP_ERR_INVALID_ARG, "tuning record out of range");
  }
  for (size_t g = 0; g < h->passes.size(); ++g) {
    PassData& pd = h->passes[g];
    const int32_t* v = values + 6 * g;
    pd.fwd = GmpShape{v[0], v[1]};
    pd.bwd = GmpShape{16, v[2]};
    pd.vjp_fused = v[3];
    pd.fused = GmpShape{16, v[4]};
    pd.jac = GmpShape{16, v[5]};
  }
  return GMP_OK;
}

gmp_status gmp_sync(gmp_handle h, void* stream, double timeout_s) {
  if (!h) return GMP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  GMP_CK(cudaEventRecord(h->ev, st), "event record");
  auto t0 = std::chrono::steady_clock::now();
  while (true) {
    cudaError_t e = cudaEventQuery(h->ev);
    if (e == cudaSuccess) {
      uint32_t w = 0;
      GMP_CK(cudaMemcpy(&w, h->scalars.p, sizeof(w), cudaMemcpyDeviceToHost), "read err");
      if (w) {
        GMP_CK(cudaMemset(h->scalars.p, 0, sizeof(w)), "clear err");
        return decode_device_error(h, w);
      }
      return GMP_OK;
    }
    if (e != cudaErrorNotReady) return cuda_fail(h, e, "event query");
    if (timeout_s > 0) {
      double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > timeout_s) return fail(h, GMP_ERR_TIMEOUT, "gmp_sync timed out");
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

const char* gmp_last_error(gmp_handle h) {
  if (!h) return "null handle";
  return h->err.c_str();
}

int64_t gmp_kernel_launches(gmp_handle h) { return h ? h->launches : 0; }

gmp_status gmp_profile(gmp_handle h, int enable) {
  if (!h) return GMP_ERR_INVALID_ARG;
  h->profiling = enable != 0;
  for (int s = 0; s < gmp_ctx::kStages; ++s) h->prof_used[s] = 0;
  return GMP_OK;
}

gmp_status gmp_profile_read(gmp_handle h, double* ms, int64_t* count, int n_stages) {
  if (!h || !ms || !count || n_stages < 1 || n_stages > gmp_ctx::kStages) return GMP_ERR_INVALID_ARG;
  for (int s = 0; s < n_stages; ++s) {
    double tot = 0.0;
    for (size_t u = 0; u + 1 < h->prof_used[s] + 1 && u < h->prof_used[s]; u += 2) {
      GMP_CK(cudaEventSynchronize(h->prof_ev[s][u + 1]), "profile sync");
      float t = 0.0f;
      GMP_CK(cudaEventElapsedTime(&t, h->prof_ev[s][u], h->prof_ev[s][u + 1]), "profile elapsed");
      tot += t;
    }
    ms[s] = tot;
    count[s] = (int64_t)(h->prof_used[s] / 2);
    h->prof_used[s] = 0;
  }
  return GMP_OK;
}

void gmp_destroy(gmp_handle h) {
  if (!h) return;
  cudaSetDevice(h->device);
  for (auto& pd : h->passes) pd.rad.release();
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->h_small) cudaFreeHost(h->h_small);
  for (auto& v : h->prof_ev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
  if (h->ev) cudaEventDestroy(h->ev);
  for (cudaEvent_t e : {h->ev_in, h->ev_feat, h->ev_out})
    if (e) cudaEventDestroy(e);
  if (h->side) cudaStreamDestroy(h->side);
  delete h;  // the device buffers free themselves, with this device current
}

}  // extern "C"
