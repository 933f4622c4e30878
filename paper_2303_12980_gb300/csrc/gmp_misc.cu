// Small helper kernels: structure ids, Jacobian row counts, gradient output.
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
