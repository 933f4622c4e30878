// Allocation-free neighbor counting for one structure.
//
// gmp_neighbor_counts_noalloc runs the same binning and exact neighbor-count
// kernels as gmp_neighbors (always the multi-kernel binning, whose bins equal
// those of the single-CTA binning gmp_neighbors uses for small batches), but
// every scratch buffer they need (per-atom
// fractional coordinates, the bin grid, bin counts and offsets, the scan
// workspace, the error word) lives in one file-scope device array of fixed
// size instead of memory obtained from cudaMalloc.  It exists for callers
// that cannot allocate device memory: code running inside another library's
// allocator or memory-pool callbacks, loops that cannot afford cudaMalloc's
// implicit device-wide synchronisation, and processes that reserve all
// device memory up front.  The array is sized for kNoAllocMaxAtoms atoms and
// every GPU that loads this library holds it until the process exits.
#include "gmp.h"
#include "gmp_internal.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

namespace {

constexpr int64_t kNoAllocMaxAtoms = 32768;
constexpr int64_t kMaxBins = 2 * kNoAllocMaxAtoms + 8;

constexpr size_t align256(size_t n) { return (n + 255) / 256 * 256; }

// Byte offsets of the sub-buffers inside the static scratch array.
struct Layout {
  static constexpr size_t st = 0;
  static constexpr size_t grid = st + align256(sizeof(GmpStruct));
  static constexpr size_t bbox = grid + align256(sizeof(GmpGrid));
  static constexpr size_t scal = bbox + align256(6 * sizeof(unsigned long long));
  static constexpr size_t struct_of = scal + 256;
  static constexpr size_t species = struct_of + align256(4 * kNoAllocMaxAtoms);
  static constexpr size_t xh = species + align256(4 * kNoAllocMaxAtoms);
  static constexpr size_t xl = xh + align256(16 * kNoAllocMaxAtoms);
  static constexpr size_t u = xl + align256(16 * kNoAllocMaxAtoms);
  static constexpr size_t bin = u + align256(32 * kNoAllocMaxAtoms);
  static constexpr size_t bcount = bin + align256(4 * kNoAllocMaxAtoms);
  static constexpr size_t bcursor = bcount + align256(4 * kMaxBins);
  static constexpr size_t bstart = bcursor + align256(4 * kMaxBins);
  static constexpr size_t by = bstart + align256(4 * (kMaxBins + 1));
  static constexpr size_t bje = by + align256(16 * kNoAllocMaxAtoms);
  static constexpr size_t rng = bje + align256(8 * kNoAllocMaxAtoms);
  static constexpr size_t ay = rng + align256(16 * kNoAllocMaxAtoms);
  static constexpr size_t scan = ay + align256(16 * kNoAllocMaxAtoms);
  static constexpr size_t scan_bytes = 16 * 1024;
  static constexpr size_t total = scan + scan_bytes;
};

// The scratch itself (about 5 MB).  Host code must not use this name as an
// address: it is only a host-side stand-in; the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[Layout::total];

std::mutex g_mutex;
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};

gmp_status report(gmp_status st, const char* msg) {
  std::fprintf(stderr, "gmp_neighbor_counts_noalloc: %s\n", msg);
  return st;
}

bool inv3(const double* A, double* Ai) {
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
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

}  // namespace

extern "C" gmp_status gmp_neighbor_counts_noalloc(int32_t n_atoms, const double* pos, const double* cell,
                                                  const uint8_t* pbc, double cutoff, int64_t* counts,
                                                  void* stream) {
  if (n_atoms < 0 || n_atoms > kNoAllocMaxAtoms) {
    char m[160];
    std::snprintf(m, sizeof(m), "n_atoms = %d is outside 0..%lld, the size of the static scratch array",
                  (int)n_atoms, (long long)kNoAllocMaxAtoms);
    return report(GMP_ERR_CAPACITY, m);
  }
  if (!(cutoff > 0.0) || !std::isfinite(cutoff)) return report(GMP_ERR_INVALID_ARG, "cutoff must be > 0");
  if (n_atoms == 0) return GMP_OK;
  if (!pos || !counts || !cell || !pbc) return report(GMP_ERR_INVALID_ARG, "pos, cell, pbc and counts are required");
  cudaStream_t st = (cudaStream_t)stream;

  // per-device set-up, done by the first call on each device (which should
  // come before any stream capture): the device address of the scratch array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return report(GMP_ERR_CUDA, "no current CUDA device");
  }
  int sm_count = 0;
  if (cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sm_count < 1) {
    cudaGetLastError();
    sm_count = 1;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return report(GMP_ERR_CUDA, cudaGetErrorString(e));
      }
      g_scratch_addr[dev] = ptr;
    }
    base = static_cast<unsigned char*>(g_scratch_addr[dev]);
  }

  // host-side structure description (same fields as the batched path)
  GmpStruct g;
  std::memset(&g, 0, sizeof(g));
  bool any = false;
  for (int k = 0; k < 3; ++k) {
    g.periodic[k] = pbc[k] ? 1 : 0;
    any = any || g.periodic[k];
  }
  if (any) {
    for (int k = 0; k < 9; ++k) g.A[k] = cell[k];
    if (!inv3(g.A, g.Ainv)) return report(GMP_ERR_INVALID_ARG, "singular cell with a periodic axis");
  } else {
    for (int k = 0; k < 9; ++k) g.A[k] = g.Ainv[k] = (k % 4 == 0) ? 1.0 : 0.0;
  }
  for (int k = 0; k < 3; ++k) {
    const double bk = std::sqrt(g.Ainv[k] * g.Ainv[k] + g.Ainv[3 + k] * g.Ainv[3 + k] + g.Ainv[6 + k] * g.Ainv[6 + k]);
    g.reach[k] = cutoff * bk;
    if (g.periodic[k] && g.reach[k] > 64.0) return report(GMP_ERR_INVALID_ARG, "cutoff spans more than 64 cell widths");
  }
  for (int k = 0; k < 9; ++k) {
    g.Ahi[k] = (float)g.A[k];
    g.Alo[k] = (float)(g.A[k] - (double)g.Ahi[k]);
  }
  g.n_atoms = n_atoms;
  g.bin_cap = 2 * n_atoms + 8;
  const int64_t n_bins = g.bin_cap;

  GmpStruct* d_st = reinterpret_cast<GmpStruct*>(base + Layout::st);
  GmpGrid* d_grid = reinterpret_cast<GmpGrid*>(base + Layout::grid);
  unsigned long long* d_bbox = reinterpret_cast<unsigned long long*>(base + Layout::bbox);
  uint32_t* d_err = reinterpret_cast<uint32_t*>(base + Layout::scal);
  int32_t* d_maxm = reinterpret_cast<int32_t*>(d_err + 1);
  int32_t* d_struct_of = reinterpret_cast<int32_t*>(base + Layout::struct_of);
  int32_t* d_species = reinterpret_cast<int32_t*>(base + Layout::species);
  float4* d_xh = reinterpret_cast<float4*>(base + Layout::xh);
  float4* d_xl = reinterpret_cast<float4*>(base + Layout::xl);
  GmpD4* d_u = reinterpret_cast<GmpD4*>(base + Layout::u);
  int32_t* d_bin = reinterpret_cast<int32_t*>(base + Layout::bin);
  int32_t* d_bcount = reinterpret_cast<int32_t*>(base + Layout::bcount);
  int32_t* d_bcursor = reinterpret_cast<int32_t*>(base + Layout::bcursor);
  int32_t* d_bstart = reinterpret_cast<int32_t*>(base + Layout::bstart);
  float4* d_by = reinterpret_cast<float4*>(base + Layout::by);
  int2* d_bje = reinterpret_cast<int2*>(base + Layout::bje);
  int4* d_rng = reinterpret_cast<int4*>(base + Layout::rng);
  float4* d_ay = reinterpret_cast<float4*>(base + Layout::ay);
  void* d_scan = base + Layout::scan;
  if (gmp_scan_tmp_bytes(n_bins) > Layout::scan_bytes) return report(GMP_ERR_CAPACITY, "scan workspace too small");

  // the array keeps the previous call's contents: reset what starts at zero
  int64_t launches = 0;
  cudaError_t e = cudaMemcpyAsync(d_st, &g, sizeof(g), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_struct_of, 0, sizeof(int32_t) * n_atoms, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_species, 0, sizeof(int32_t) * n_atoms, st);
  if (e == cudaSuccess)
    e = gmp_launch_neighbors_prepare(d_st, 1, d_struct_of, n_atoms, cutoff, pos, d_species, 1, d_grid, d_xh, d_xl,
                                     d_u, d_bin, d_bbox, d_err, st, sm_count, &launches);
  if (e == cudaSuccess)
    e = gmp_launch_bins(d_st, d_grid, d_struct_of, n_atoms, n_bins, d_bin, d_bcount, d_bstart, d_bcursor, d_rng,
                        d_ay, d_by, d_bje, d_u, d_xh, d_xl, d_scan, Layout::scan_bytes, st, sm_count, &launches);
  const GmpCenters centers{d_struct_of, pos, d_xh, d_xl, d_rng, d_ay};
  if (e == cudaSuccess)
    e = gmp_launch_neighbor_pass(0, d_st, d_grid, centers, n_atoms, cutoff, pos, d_xh, d_xl, d_bstart, d_by,
                                 d_bje, 1, counts, nullptr, nullptr, 0, 0, d_maxm, d_err, st, sm_count, &launches);
  uint32_t w = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&w, d_err, sizeof(w), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return report(GMP_ERR_CUDA, cudaGetErrorString(e));
  }
  if (w & GMP_DEV_NONFINITE) return report(GMP_ERR_DEVICE, "non-finite position");
  if (w) return report(GMP_ERR_DEVICE, "periodic image index out of range");
  return GMP_OK;
}
