/*
 * gmp.h -- C ABI of libgmp: Gaussian Multipole (GMP) features of atomic
 * structures and their position derivatives on one NVIDIA GB300 (sm_103a).
 *
 * Method (GMP-Featurizer, arXiv 2303.12980):
 *   Each atom's electron density is a sum of Gaussians c_k exp(-alpha_k r^2)
 *   taken from per-element tables (Overview: pseudopotential files specify
 *   the Gaussians; Examples: psp_path).  For every center atom i, the
 *   density of all atoms within the cutoff -- periodic images included --
 *   is projected on probes = MCSH angular function of order l times a
 *   Gaussian radial function of width sigma (Examples: "orders", "sigmas");
 *   the projections of one (l, sigma) group are reduced to one rotation
 *   invariant number, the weighted sum of squares over the group's
 *   components.  The feature set is the Cartesian product orders x sigmas,
 *   order-major; order -1 is the local density at the center, one feature
 *   (Examples, feature-set listing).  Derivatives of the features with
 *   respect to atom positions are available (Examples: calc_derivatives,
 *   feature_primes).
 *
 * Conventions for every call below:
 *   - Units: Angstrom and Angstrom^-2.
 *   - N = total atoms over a batch of S structures; structure s owns atoms
 *     atom_off[s] .. atom_off[s+1]-1 (host array, int64, atom_off[0] = 0).
 *   - pos [N,3] float64 raw Cartesian positions (no wrapping is applied to
 *     the displacement: d = (x_j - x_i) + n1 a1 + n2 a2 + n3 a3).
 *   - cell [S,3,3] float64 HOST array, rows are lattice vectors a1, a2, a3;
 *     pbc [S,3] uint8 HOST array.  A structure with any periodic axis needs
 *     a non-singular cell; a structure with none ignores its cell (zeros ok).
 *   - species [N] int32 in 0 .. n_elements-1.
 *   - pos, species and all outputs may be DEVICE pointers (the call is then
 *     asynchronous on `stream`) or HOST pointers (pageable or pinned; the
 *     call then stages copies through device memory and returns after the
 *     results are in host memory).  Inputs and outputs of one call must be
 *     all device or all host.
 *   - The caller owns every buffer it passes; the handle owns its tables and
 *     a growable device workspace (so concurrent calls on one handle must be
 *     serialised by the caller).
 *   - Errors are returned as gmp_status; gmp_last_error() gives a message.
 *     Conditions detected on the device (bad species id, non-finite
 *     position, too many neighbors of one center) are reported through a
 *     device error word checked at the end of the call (device-pointer
 *     calls synchronise `stream` once per call to read it).
 */
#ifndef GMP_H_
#define GMP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gmp_ctx *gmp_handle;

typedef enum {
  GMP_OK = 0,
  GMP_ERR_INVALID_ARG = 1, /* bad sizes, pointers, orders, singular cell ... */
  GMP_ERR_CUDA = 2,        /* a CUDA runtime call failed                      */
  GMP_ERR_OOM = 3,         /* device allocation failed                        */
  GMP_ERR_CAPACITY = 4,    /* caller buffer too small (see nnz_out)            */
  GMP_ERR_TIMEOUT = 5,     /* gmp_sync timed out                               */
  GMP_ERR_DEVICE = 6       /* a condition flagged by a kernel (see message)    */
} gmp_status;

/* Flags for gmp_params.flags (reserved: gmp_create rejects any other value
 * with GMP_ERR_INVALID_ARG). */
#define GMP_FLAG_NONE 0u

/* Probe set and density tables (Examples: the GMPs dictionary). */
typedef struct {
  int32_t n_elements;         /* species ids are 0 .. n_elements-1             */
  const int32_t *n_gauss;     /* [n_elements] Gaussians per element (>= 1)     */
  const double *gauss_coef;   /* [sum n_gauss] c_k (any sign)                   */
  const double *gauss_exp;    /* [sum n_gauss] alpha_k > 0, Angstrom^-2         */
  int32_t n_orders;           /* >= 1                                           */
  const int32_t *orders;      /* each in {-1, 0, 1, ..., 6}, no repeats         */
  int32_t n_sigmas;           /* >= 1 when any order >= 0                       */
  const double *sigmas;       /* each > 0, Angstrom                             */
  double cutoff;              /* Angstrom; hard cutoff |d| < cutoff.  <= 0:
                                 derived from overlap_threshold (below)        */
  uint32_t flags;             /* GMP_FLAG_*                                     */
  double overlap_threshold;   /* used when cutoff <= 0 (the paper's Examples
                                 section sets the accuracy of the features by
                                 this threshold): the cutoff is the smallest
                                 radius beyond which every single-primitive
                                 contribution to any moment is below this value
                                 (see gmp_cutoff)                              */
} gmp_params;

/* Create a handle on CUDA device `device`: validates `params`, copies the
 * tables (host memory, read during the call only) and builds the per
 * (element, sigma, primitive) radial prefactors on the device.
 * Returns GMP_ERR_INVALID_ARG for any invalid field. */
gmp_status gmp_create(const gmp_params *params, int device, gmp_handle *out);

/* Number of features per atom F = (#orders >= 0) * n_sigmas + (#order -1). */
gmp_status gmp_num_features(gmp_handle h, int32_t *F);

/* The cutoff in use (Angstrom).  When it was derived from overlap_threshold
 * t (the paper's Examples section: with no cutoff given, the threshold on
 * overlaps decides it), it is the largest r at which some single-primitive
 * bound still exceeds t:
 *   order l >= 0, sigma s, primitive (c, alpha), g = alpha + 1/(2 s^2):
 *     |c| N_s (pi/g)^(3/2) (alpha/g)^l sqrt(l! (2l-1)!!) r^l exp(-(alpha/(2 s^2 g)) r^2)
 *     (the largest overlap of that primitive with any MCSH component of the
 *     probe, since |S_c(d)| <= sqrt(l!(2l-1)!!) |d|^l);
 *   order -1: |c| exp(-alpha r^2). */
gmp_status gmp_cutoff(gmp_handle h, double *cutoff);

/* Features of every atom (Examples: entry["features"]).
 * features [N, F] float32, order-major: column (o, s) = o * n_sigmas + s for
 * orders >= 0 in the order given, order -1 (if requested) at its own
 * position in the order list with a single column. */
gmp_status gmp_featurize(gmp_handle h, int32_t n_struct, const int64_t *atom_off,
                         const double *pos, const double *cell, const uint8_t *pbc,
                         const int32_t *species, float *features, void *stream);

/* Features and the vector-Jacobian product with an upstream gradient:
 * grad_pos[j] = sum_i sum_f grad_feat[i, f] * d features[i, f] / d pos[j].
 * grad_feat [N, F] float32 in; features [N, F] (may be NULL) and
 * grad_pos [N, 3] float32 out.  This is the force path (autograd backward). */
gmp_status gmp_featurize_vjp(gmp_handle h, int32_t n_struct, const int64_t *atom_off,
                             const double *pos, const double *cell, const uint8_t *pbc,
                             const int32_t *species, const float *grad_feat,
                             float *features, float *grad_pos, void *stream);

/* gmp_featurize_vjp plus the strain derivative of each structure (the
 * virial, for stresses; an extension beyond the paper's outputs): with
 * L = sum_i sum_f grad_feat[i, f] * features[i, f] and a homogeneous strain
 * eps applied to positions and lattice vectors alike (x -> (I + eps) x, so
 * every neighbor displacement d -> (I + eps) d),
 *   virial[s, a, b] = dL / d eps_ab = sum over the neighbor images of the
 *   centers of structure s of (dL/dd)_a * d_b.
 * virial [S, 3, 3] float64 out, device or host like the other outputs.
 * The stress of an energy E(features) is virial / cell volume with
 * grad_feat = dE/dfeatures.  Symmetric up to rounding (rotation invariance). */
gmp_status gmp_featurize_vjp_virial(gmp_handle h, int32_t n_struct, const int64_t *atom_off,
                                    const double *pos, const double *cell, const uint8_t *pbc,
                                    const int32_t *species, const float *grad_feat,
                                    float *features, float *grad_pos, double *virial,
                                    void *stream);

/* Features and the dense per-(center, neighbor atom) Jacobian
 * (Examples: entry["feature_primes"]).  Row i lists the distinct atoms j
 * whose position moves feature row i (the center itself included), images
 * of one atom summed:
 *   jac_off [N+1] int64, jac_j [cap] int32 (ascending within a row),
 *   jac [cap, F, 3] float32 = d features[i, :] / d pos[j, :].
 * If the total nnz exceeds `cap`, nothing but *nnz_out is written and
 * GMP_ERR_CAPACITY is returned; call again with cap >= *nnz_out.
 * nnz_out is a host pointer; this call synchronises `stream`. */
gmp_status gmp_featurize_grad(gmp_handle h, int32_t n_struct, const int64_t *atom_off,
                                  const double *pos, const double *cell, const uint8_t *pbc,
                                  const int32_t *species, float *features, int64_t *jac_off,
                                  int32_t *jac_j, float *jac, int64_t cap, int64_t *nnz_out,
                                  void *stream);

/* The same for the centers center_begin .. center_end-1 of the batch only
 * (0 <= begin <= end <= N, else GMP_ERR_INVALID_ARG): a Jacobian too large
 * for memory at once (262,144 slab atoms: ~37 M rows, ~50 GB) is taken in
 * center chunks, each with its own capacity.  Rows and values equal those
 * of gmp_featurize_grad for these centers; outputs are relative to the
 * range:
 *   features [end-begin, F] (optional, may be null), jac_off [end-begin+1]
 *   (jac_off[0] = 0), jac_j [cap], jac [cap, F, 3].
 * The neighbor lists are built for the whole batch on every call. */
gmp_status gmp_featurize_grad_centers(gmp_handle h, int32_t n_struct, const int64_t *atom_off,
                                      const double *pos, const double *cell, const uint8_t *pbc,
                                      const int32_t *species, int64_t center_begin, int64_t center_end,
                                      float *features, int64_t *jac_off, int32_t *jac_j, float *jac,
                                      int64_t cap, int64_t *nnz_out, void *stream);

/* Features at reference points (the paper's Overview section: features are
 * defined around arbitrary points of a structure, not only around its
 * atoms).  The probes are centred on each point; the neighbor set is every
 * atom image of the point's structure with |(x_j - p) + n1 a1 + n2 a2 + n3 a3|
 * < cutoff, decided in FP64 exactly as gmp_neighbors does for atoms (a point
 * that coincides with an atom gets that atom's features).
 *   point_off [S+1] int64 HOST array: structure s owns points
 *     point_off[s] .. point_off[s+1]-1 (point_off[0] = 0);
 *   points [n_points, 3] float64 raw Cartesian (any position, inside the
 *     cell or not; periodic axes wrap as for atoms);
 *   features [n_points, F] float32 out, columns as in gmp_featurize.
 * points and features follow pos (device or host; with no atoms at all the
 * features are zero).  A structure may own points and no atoms, or atoms and
 * no points.  Synchronises `stream` once (to size the neighbor buffer). */
gmp_status gmp_featurize_points(gmp_handle h, int32_t n_struct, const int64_t *atom_off,
                                const double *pos, const double *cell, const uint8_t *pbc,
                                const int32_t *species, const int64_t *point_off,
                                const double *points, float *features, void *stream);

/* Exact neighbor images (for checking; the featurize calls build their own).
 * Pairs (i, j, n) with |(x_j - x_i) + n1 a1 + n2 a2 + n3 a3| < cutoff, the
 * self pair included, decided in FP64 exactly as that expression reads
 * (left to right, no FMA).  nbr_off [N+1] int64; nbr_j [cap] int32;
 * nbr_shift [cap, 3] int32 (n1, n2, n3); each row ordered by (j, n1, n2, n3).
 * Capacity semantics as in gmp_featurize_grad. */
gmp_status gmp_neighbors(gmp_handle h, int32_t n_struct, const int64_t *atom_off,
                         const double *pos, const double *cell, const uint8_t *pbc,
                         const int32_t *species, int64_t *nbr_off, int32_t *nbr_j,
                         int32_t *nbr_shift, int64_t cap, int64_t *nnz_out, void *stream);

/* Neighbor-image counts of one structure without allocating device memory.
 * The paper has no counterpart: this entry point is for callers that cannot
 * call cudaMalloc -- code running inside another library's allocator or
 * memory-pool callbacks, loops that cannot afford cudaMalloc's implicit
 * device-wide synchronisation, processes that reserve all device memory up
 * front.  It runs the same binning (the multi-kernel path) and exact count
 * kernels as gmp_neighbors and needs no handle: all scratch lives in a
 * fixed static device array
 * (about 5 MB, held by every GPU that loads the library until the process
 * exits), sized for at most 32768 atoms; larger n_atoms returns
 * GMP_ERR_CAPACITY with a message on stderr before any GPU work.
 *   pos [n_atoms, 3] float64 DEVICE pointer (raw Cartesian, Angstrom);
 *   cell [3,3] float64 and pbc [3] uint8 HOST arrays (as in gmp_featurize);
 *   counts [n_atoms] int64 DEVICE output: neighbor images of each atom
 *   within `cutoff`, self included (equal to nbr_off[i+1] - nbr_off[i] of
 *   gmp_neighbors with the same cutoff).
 * The call runs on `stream` and synchronises it before returning (to read
 * the device error word).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current
 * and keeps it for the life of the process; make that first call on a
 * device before any stream capture.  A device reset
 * (cudaDeviceReset) after that first call would leave the kept address
 * stale: it is not supported.  All calls share the one
 * array and each call resets what must start at zero, so calls that overlap
 * on the GPU (other streams, other host threads) race: serialise them. */
gmp_status gmp_neighbor_counts_noalloc(int32_t n_atoms, const double *pos, const double *cell,
                                       const uint8_t *pbc, double cutoff, int64_t *counts,
                                       void *stream);

/* CUDA-graph mode (default off).  When on, a gmp_featurize /
 * gmp_featurize_vjp call with device buffers on a non-default stream first
 * runs eagerly, then captures its whole device sequence (binning, neighbor
 * passes, compute kernels, refinement) into a CUDA graph whose neighbor
 * capacities carry 12.5% headroom over the eager run; the next calls with
 * the same buffers, stream and batch description replay the graph and
 * synchronise the stream once.  A batch that outgrows the captured
 * capacities is detected on the device; that call then re-runs eagerly and
 * recaptures, so results are always complete.  Any other call on the handle
 * invalidates the graph. */
gmp_status gmp_set_graph(gmp_handle h, int enable);

/* Autotuner (not part of the method): builds the neighbor lists of the given
 * batch, then times on it (CUDA events, `reps` launches after a warm-up)
 * the candidate launch shapes of each compute kernel -- forward tile of 16
 * or 32 pairs x 4/8/16 warps per CTA, backward 4/6/12 warps, the fused
 * forward+backward VJP kernel 4/8 warps versus the forward + backward pair
 * -- and keeps the fastest in the handle for later calls.  Synchronises
 * `stream`; writes the number of neighbor pairs to *pairs_out (host, may be
 * NULL).  Inputs as in gmp_featurize. */
gmp_status gmp_tune(gmp_handle h, int32_t n_struct, const int64_t *atom_off, const double *pos,
                    const double *cell, const uint8_t *pbc, const int32_t *species, int32_t reps,
                    int64_t *pairs_out, void *stream);

/* The handle's launch shapes as 6 int32 per sigma pass (forward tile,
 * forward warps, backward warps, fused-VJP flag, fused warps, Jacobian
 * warps; 0 warps = largest that fits), for persisting tuning results.
 * gmp_tuning_get needs n >= 6 * passes (GMP_ERR_CAPACITY otherwise);
 * gmp_tuning_set needs exactly that many values in range. */
gmp_status gmp_tuning_get(gmp_handle h, int32_t *values, int32_t n);
gmp_status gmp_tuning_set(gmp_handle h, const int32_t *values, int32_t n);

/* Wait for `stream` with a timeout (seconds, <= 0: wait forever) by polling
 * an event; returns GMP_ERR_TIMEOUT if the work has not finished. */
gmp_status gmp_sync(gmp_handle h, void *stream, double timeout_s);

/* Message for the last non-OK status on this handle (never NULL). */
const char *gmp_last_error(gmp_handle h);

/* Number of kernels this handle has launched so far (diagnostics). */
int64_t gmp_kernel_launches(gmp_handle h);

/* Stage timing (diagnostics, not part of the method).  With enable != 0 the
 * featurize calls record CUDA events on the caller's stream around
 *   stage 0: neighbor search (binning, count, fill),
 *   stage 1: the forward (feature) kernel,
 *   stage 2: the backward kernel of gmp_featurize_vjp, or the Jacobian
 *            kernel of gmp_featurize_grad,
 *   stage 3: double-float refinement of ill-conditioned features;
 * gmp_profile_read synchronises those events and writes, per stage, the
 * summed milliseconds and the number of stage executions since the last
 * read (arrays of length n_stages <= 4), then clears the counters. */
gmp_status gmp_profile(gmp_handle h, int enable);
gmp_status gmp_profile_read(gmp_handle h, double *ms, int64_t *count, int n_stages);

/* Release the handle and its device memory. */
void gmp_destroy(gmp_handle h);

/* Throughput probes of CUDA device `device` at its present clocks
 * (diagnostics, about 30 ms): FP32 FMA rate with scalar FMAs and with packed
 * FP32-pair FMAs (TFLOP/s, 2 FLOP per FMA), and the SFU's ex2 rate (10^12
 * per second).  Each probe runs independent dependency chains on every
 * resident thread.  Needs no handle; GMP_ERR_CUDA if a launch fails. */
gmp_status gmp_probe_peaks(int device, double *fma_tflops, double *fma2_tflops, double *ex2_tops);

/* Measured evaluation of a tensor-core recast of the moment contraction
 * (the per-center sum over pairs of R_{l,sigma} S_c, section Overview's
 * multipole moments; diagnostics, about 100 ms): the same 16-sigma x
 * 64-slot contraction over 16-pair shared-memory tiles (orders 0..6) run
 * (a) as the forward kernel runs it, packed FP32-pair FMAs with a TwoSum
 * fold per tile, and (b) on the tensor cores, mma.sync m16n8k8 with TF32
 * operands split hi + lo and three products per tile (hi*hi, hi*lo,
 * lo*hi), FP32 accumulators folded by TwoSum per tile.  result[n_result],
 * n_result >= GMP_PROBE_CONTRACT_N, host array, four versions v =
 * FP32 (16 warps per SM), TF32x3 (16 warps per SM, 128 registers),
 * TF32x3 (8 warps per SM, up to 255 registers), TF32x3 on tiles stored
 * already split (16 warps per SM):
 *   [v]      10^9 pairs/s
 *   [4 + v]  largest error of a 144-pair sum relative to its
 *            cancellation-free scale (sum of |R S|), against FP64
 *   [8 + v]  registers per thread
 * Needs no handle; GMP_ERR_CUDA if a launch fails. */
#define GMP_PROBE_CONTRACT_N 12
gmp_status gmp_probe_contraction(int device, double *result, int32_t n_result);

/* Measured evaluation of the backward kernel's per-pair adjoint
 * contraction (paper Examples: the derivatives of the features,
 * calc_derivatives; per pair lam_k = sum_s Lam[s][k] R_{s,l(k)} and its
 * radial derivative counterpart, 16 sigmas x 49 components x 2) on the
 * 5th-generation tensor cores against the FP32 scheme the backward kernel
 * runs, on seeded data.  tcgen05 version: 128 pairs per tile on the MMA's
 * M rows (one per tensor-memory lane), K = 16 sigmas, N = 32 columns per
 * order, kind::tf32 with hi/lo operand splits (3 MMAs per product),
 * operands in shared memory, accumulators in tensor memory, bounded
 * mbarrier waits.  Writes GMP_PROBE_BWD_CONTRACT_N doubles into the host
 * array `result`: [0] FP32 scheme, 10^9 pairs/s; [1] tcgen05, 10^9
 * pairs/s; [2] [3] FP32 max error of lam / lamd over 128 pairs against
 * FP64, relative to each sum's cancellation-free scale; [4] [5] the same
 * for tcgen05; [6] [7] registers per thread of the two kernels; [8]
 * nonzero if a tcgen05 wait ran out (its results are then incomplete).
 * Needs no handle; GMP_ERR_CUDA if a launch fails.  The library's kernels
 * do not use the tcgen05 version. */
#define GMP_PROBE_BWD_CONTRACT_N 9
gmp_status gmp_probe_backward_contraction(int device, double *result, int32_t n_result);

#ifdef __cplusplus
}
#endif

#endif /* GMP_H_ */
