// Small helper kernels: structure ids, Jacobian row counts, the
// order-independent gradient sums, strain-derivative sums, gradient output.
#include "gmp_internal.cuh"

namespace {

__global__ void k_struct_of(const int64_t* __restrict__ atom_off, int n_struct,
                            int32_t* __restrict__ struct_of) {
  for (int s = blockIdx.x; s < n_struct; s += gridDim.x) {
    const int64_t a0 = atom_off[s], a1 = atom_off[s + 1];
    for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) struct_of[a] = s;
  }
}

// Distinct neighbor atoms per center (lists are sorted by atom), and for
// every pair the rank of its atom among them (the pair's Jacobian row
// within the center's rows).
__global__ void k_jac_count(int64_t N, const int64_t* __restrict__ nbr_beg, const int64_t* __restrict__ nbr_end,
                            const GmpPair* __restrict__ pairs, int64_t* __restrict__ counts,
                            int32_t* __restrict__ local_row) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= N) return;
  const int64_t p0 = nbr_beg[i], p1 = nbr_end[i];
  int c = 0;  // rows so far (warp-uniform)
  for (int64_t base = p0; base < p1; base += 32) {
    const int64_t p = base + lane;
    const bool in = p < p1;
    const bool first = in && (p == p0 || pairs[p - 1].j != pairs[p].j);
    const unsigned m = __ballot_sync(0xffffffffu, first);
    if (in) local_row[p] = c + __popc(m & ((2u << lane) - 1u)) - 1;
    c += __popc(m);
  }
  if (lane == 0) counts[i] = c;
}

// grad_acc[j] += own[j] + the value of j's fixed-point bins (bin b counts in
// units of 2^(24 b - 149); added in a fixed order, so the result does not
// depend on the order in which the bins were filled).  Bin 11 holds flags
// of non-finite contributions: NaN if any was NaN or infinities of both
// signs came in, else that infinity.  One thread per (atom, component).
__global__ void k_grad_bins_finish(int64_t n, const unsigned long long* __restrict__ bins,
                                   const double* __restrict__ own, double* __restrict__ grad_acc) {
  constexpr int kBins = 12;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long* bt = bins + t * kBins;
    const unsigned long long fl = bt[11];
    double v;
    if (fl) {
      v = ((fl & 1ull) || ((fl & 6ull) == 6ull)) ? (double)NAN : ((fl & 2ull) ? (double)INFINITY : -(double)INFINITY);
    } else {
      v = 0.0;
#pragma unroll
      for (int b = 0; b < 11; ++b) v += ldexp((double)(long long)bt[b], 24 * b - 149);
    }
    grad_acc[t] = grad_acc[t] + (own[t] + v);
  }
}

// virial[s] += sum over the centers of structure s of vir_c[center] (nine
// values), one warp per structure, lanes over centers in a fixed order.
__global__ void k_virial_reduce(int n_struct, const int64_t* __restrict__ atom_off, const double* __restrict__ vir_c,
                                double* __restrict__ virial) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = w0; s < n_struct; s += nw) {
    const int64_t a0 = atom_off[s], a1 = atom_off[s + 1];
    double acc[9];
#pragma unroll
    for (int v = 0; v < 9; ++v) acc[v] = 0.0;
    for (int64_t a = a0 + lane; a < a1; a += 32)
#pragma unroll
      for (int v = 0; v < 9; ++v) acc[v] += vir_c[9 * a + v];
#pragma unroll
    for (int v = 0; v < 9; ++v) {
      double x = acc[v];
#pragma unroll
      for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) virial[9 * s + v] += x;
    }
  }
}

__global__ void k_grad_finish(int64_t n, const double* __restrict__ acc, float* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (float)acc[t];
}

}  // namespace

cudaError_t gmp_launch_struct_of(const int64_t* d_atom_off, int n_struct, int32_t* struct_of,
                                 cudaStream_t stream, int64_t* launches) {
  const int blocks = n_struct < 65535 ? n_struct : 65535;
  k_struct_of<<<blocks > 0 ? blocks : 1, 256, 0, stream>>>(d_atom_off, n_struct, struct_of);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t gmp_launch_jacobian_count(int64_t N, const int64_t* nbr_beg, const int64_t* nbr_end, const GmpPair* pairs,
                                      int64_t* counts, int32_t* local_row, cudaStream_t stream, int sm_count,
                                      int64_t* launches) {
  (void)sm_count;
  if (N <= 0) return cudaSuccess;
  const int64_t threads = N * 32;
  k_jac_count<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(N, nbr_beg, nbr_end, pairs, counts, local_row);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t gmp_launch_grad_finish(int64_t N, const double* grad_acc, float* grad_pos,
                                   cudaStream_t stream, int64_t* launches) {
  if (N <= 0) return cudaSuccess;
  const int64_t n = 3 * N;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_grad_finish<<<(unsigned)blocks, 256, 0, stream>>>(n, grad_acc, grad_pos);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t gmp_launch_grad_bins_finish(int64_t N, const unsigned long long* bins, const double* own,
                                        double* grad_acc, cudaStream_t stream, int sm_count, int64_t* launches) {
  if (N <= 0) return cudaSuccess;
  const int64_t n = 3 * N;
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = (int64_t)sm_count * 8;
  if (blocks > cap) blocks = cap;
  k_grad_bins_finish<<<(unsigned)blocks, 256, 0, stream>>>(n, bins, own, grad_acc);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t gmp_launch_virial_reduce(int n_struct, const int64_t* atom_off, const double* vir_c, double* virial,
                                     cudaStream_t stream, int sm_count, int64_t* launches) {
  if (n_struct <= 0) return cudaSuccess;
  int64_t blocks = ((int64_t)n_struct * 32 + 255) / 256;
  const int64_t cap = (int64_t)sm_count * 8;
  if (blocks > cap) blocks = cap;
  k_virial_reduce<<<(unsigned)blocks, 256, 0, stream>>>(n_struct, atom_off, vir_c, virial);
  ++*launches;
  return cudaGetLastError();
}
