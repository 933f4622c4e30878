/*
 * FP64 CPU oracle for Gaussian Multipole (GMP) features and their position
 * derivatives.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the
 * CPU-baseline leg of the benchmark call it; the product path never does.
 * It shares no code, header, table or constant with the CUDA path.
 *
 * What is computed (GMP-Featurizer, arXiv 2303.12980):
 *   - features of the local electron density around every atom position
 *     (Summary; Statement of Needs: density approximated by a multipole
 *     expansion of per-atom Gaussian densities);
 *   - probes = MCSH angular functions of order l times Gaussian radial
 *     functions of width sigma; the feature set is the Cartesian product of
 *     orders and sigmas, order-major; order -1 is the local density itself,
 *     one feature, sigma ignored (Examples);
 *   - periodic crystals, molecules and clusters, given lattice vectors and
 *     positions (Statement of Needs; Overview);
 *   - derivatives of the features with respect to atom positions
 *     (Examples, calc_derivatives / feature_primes).
 * The paper defers the formulas to its GMP reference; the definitions used
 * here are written out step by step below, each step in plain FP64 with no
 * blocking, fusion or reordering:
 *   1. neighbor images: all (j, n in Z^3, n_k = 0 on non-periodic axes) with
 *      d = (x_j - x_i) + ((n1 a1 + n2 a2) + n3 a3) and
 *      dx*dx + dy*dy + dz*dz < rc*rc (left to right, no FMA contraction);
 *   2. MCSH polynomial S_abc(r) = (-1)^l r^(2l+1) d^a/dx^a d^b/dy^b d^c/dz^c (1/r),
 *      generated from Q = 1 by Q <- r^2 dQ/dv - (2k+1) v Q, integer
 *      coefficients;
 *   3. overlap of one density primitive c exp(-alpha |r-d|^2) with the probe
 *      N_sigma S_abc(r) exp(-r^2/(2 sigma^2)), N_sigma = (2 pi sigma^2)^(-3/2):
 *      Gaussian product theorem, then the Gaussian expectation of each
 *      monomial of S_abc from 1-D moments m_{n+1} = P m_n + n/(2 gamma) m_{n-1}
 *      (an image at d = 0, the center's own atom, adds exactly 0 to the
 *      orders l >= 1: S_abc is harmonic without a constant term);
 *   4. moments mu_{l,sigma,abc}(i) = plain FP64 sum over pairs and primitives;
 *   5. feature f_{l,sigma} = sum_abc l!/(a! b! c!) mu_abc^2 (order -1: the
 *      density sum_pairs sum_k c_k exp(-alpha_k |d|^2));
 *   6. derivative: d/dd of step 3 = 2 alpha (E[X S(X)] - d E[S(X)]) K, one
 *      monomial order higher; chain rule through step 5; images of the same
 *      atom are summed, and the center's own block is minus the sum of the
 *      others (images of the center do not move relative to it).
 * Build with -ffp-contract=off (no FMA contraction) so step 1 is bit-stable.
 *
 * Accuracy of step 3: the monomial sum cancels when the product Gaussian's
 * variance 1/(2 gamma) is large against its centre P = (alpha/gamma) d
 * (narrow probes, small density exponents, high orders): the moments are
 * ~var^(l/2) while the harmonic combination leaves ~|P|^l.  The FP64 error
 * of a moment is then a few units of 2^-53 of the sum of the magnitudes it
 * adds (K |coef| a_p a_q a_s, a_n the moments of the same recursion with
 * |P|), not of its own value.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_LMAX 6                 /* highest MCSH order supported            */
#define OR_PD 9                   /* dense poly index bound (degree <= 8)    */
#define OR_MAXCOMP 28             /* (l+1)(l+2)/2 at l = 6                   */

typedef struct {
  int32_t n_struct;
  const int64_t *atom_off;  /* [n_struct+1]                                  */
  const double *pos;        /* [N,3] raw Cartesian positions, Angstrom        */
  const double *cell;       /* [n_struct,3,3], rows are lattice vectors       */
  const uint8_t *pbc;       /* [n_struct,3]                                   */
  const int32_t *species;   /* [N], 0..n_elements-1                           */
  int32_t n_elements;
  const int32_t *gauss_off; /* [n_elements+1] into coef/exp                    */
  const double *gauss_coef; /* c_k: rho_e(r) = sum_k c_k exp(-alpha_k r^2)    */
  const double *gauss_exp;  /* alpha_k, Angstrom^-2                           */
  int32_t n_orders;
  const int32_t *orders;    /* each -1..6                                      */
  int32_t n_sigmas;
  const double *sigmas;     /* Angstrom                                        */
  double cutoff;            /* Angstrom                                        */
} oracle_problem;

/* ------------------------------------------------------------------ */
/* Step 2: MCSH polynomials from repeated differentiation of 1/r.      */
/* ------------------------------------------------------------------ */

typedef struct {
  int deg;                  /* total degree; -1 for the zero polynomial      */
  int64_t c[OR_PD][OR_PD];  /* c[p][q] multiplies x^p y^q z^(deg-p-q)        */
} opoly;

static void opoly_zero(opoly *P, int deg) {
  memset(P, 0, sizeof(*P));
  P->deg = deg;
}

/* d/dv of a homogeneous polynomial, v = 0 (x), 1 (y), 2 (z). */
static void opoly_deriv(const opoly *P, int v, opoly *out) {
  opoly_zero(out, P->deg - 1);
  for (int p = 0; p <= P->deg; ++p)
    for (int q = 0; p + q <= P->deg; ++q) {
      int s = P->deg - p - q;
      int64_t k = P->c[p][q];
      if (!k) continue;
      if (v == 0 && p > 0) out->c[p - 1][q] += k * p;
      if (v == 1 && q > 0) out->c[p][q - 1] += k * q;
      if (v == 2 && s > 0) out->c[p][q] += k * s;
    }
}

/* r^2 * P, degree + 2 (P may be the zero polynomial of degree deg). */
static void opoly_mul_r2(const opoly *P, opoly *out) {
  opoly_zero(out, P->deg + 2);
  for (int p = 0; p <= P->deg; ++p)
    for (int q = 0; p + q <= P->deg; ++q) {
      int64_t k = P->c[p][q];
      if (!k) continue;
      out->c[p + 2][q] += k;  /* x^2 */
      out->c[p][q + 2] += k;  /* y^2 */
      out->c[p][q] += k;      /* z^2: same (p,q), s grows by 2 */
    }
}

/* v * P, degree + 1. */
static void opoly_mul_axis(const opoly *P, int v, opoly *out) {
  opoly_zero(out, P->deg + 1);
  for (int p = 0; p <= P->deg; ++p)
    for (int q = 0; p + q <= P->deg; ++q) {
      int64_t k = P->c[p][q];
      if (!k) continue;
      if (v == 0) out->c[p + 1][q] += k;
      else if (v == 1) out->c[p][q + 1] += k;
      else out->c[p][q] += k;
    }
}

/* S_abc = (-1)^l r^(2l+1) d^a_x d^b_y d^c_z (1/r) as integer polynomial.
 * Writing the k-th derivative of 1/r as Q_k r^-(2k+1):
 *   d/dv [Q r^-(2k+1)] = (r^2 dQ/dv - (2k+1) v Q) r^-(2k+3). */
static void mcsh_poly(int a, int b, int c, opoly *S) {
  opoly Q, dQ, t1, t2;
  opoly_zero(&Q, 0);
  Q.c[0][0] = 1;
  int axes[3 * OR_LMAX], n = 0;
  for (int i = 0; i < a; ++i) axes[n++] = 0;
  for (int i = 0; i < b; ++i) axes[n++] = 1;
  for (int i = 0; i < c; ++i) axes[n++] = 2;
  for (int k = 0; k < n; ++k) {
    int v = axes[k];
    opoly_deriv(&Q, v, &dQ);
    opoly_mul_r2(&dQ, &t1);         /* degree k+1 */
    opoly_mul_axis(&Q, v, &t2);     /* degree k+1 */
    opoly_zero(&Q, k + 1);
    for (int p = 0; p < OR_PD; ++p)
      for (int q = 0; q < OR_PD; ++q)
        Q.c[p][q] = t1.c[p][q] - (int64_t)(2 * k + 1) * t2.c[p][q];
  }
  *S = Q;
  if (n & 1)
    for (int p = 0; p < OR_PD; ++p)
      for (int q = 0; q < OR_PD; ++q) S->c[p][q] = -S->c[p][q];
}

/* Component order inside order l: a from l down to 0, then b from l-a down
 * to 0, c = l-a-b.  l=1: x, y, z.  l=2: xx, xy, xz, yy, yz, zz. */
static int mcsh_components(int l, int *A, int *B, int *C) {
  int n = 0;
  for (int a = l; a >= 0; --a)
    for (int b = l - a; b >= 0; --b) {
      A[n] = a; B[n] = b; C[n] = l - a - b; ++n;
    }
  return n;
}

static double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

/* Sparse form of one component's polynomial, used by the feature loops. */
typedef struct {
  int a, b, c, nterm;
  double w;                       /* l!/(a! b! c!)                          */
  double coef[OR_MAXCOMP];
  int p[OR_MAXCOMP], q[OR_MAXCOMP], s[OR_MAXCOMP];
} ocomp;

typedef struct {
  int ncomp[OR_LMAX + 1];
  ocomp comp[OR_LMAX + 1][OR_MAXCOMP];
} otable;

static void build_table(otable *T) {
  for (int l = 0; l <= OR_LMAX; ++l) {
    int A[OR_MAXCOMP], B[OR_MAXCOMP], C[OR_MAXCOMP];
    int nc = mcsh_components(l, A, B, C);
    T->ncomp[l] = nc;
    for (int ci = 0; ci < nc; ++ci) {
      opoly S;
      mcsh_poly(A[ci], B[ci], C[ci], &S);
      ocomp *o = &T->comp[l][ci];
      o->a = A[ci]; o->b = B[ci]; o->c = C[ci];
      o->w = factorial(l) / (factorial(A[ci]) * factorial(B[ci]) * factorial(C[ci]));
      o->nterm = 0;
      for (int p = 0; p <= l; ++p)
        for (int q = 0; p + q <= l; ++q)
          if (S.c[p][q]) {
            o->coef[o->nterm] = (double)S.c[p][q];
            o->p[o->nterm] = p; o->q[o->nterm] = q; o->s[o->nterm] = l - p - q;
            ++o->nterm;
          }
    }
  }
}

/* Exported for the table pins: writes the integer coefficients of S_abc as
 * a dense [(l+1) x (l+1)] array indexed [p][q] (z power = l-p-q). */
int oracle_mcsh_poly(int a, int b, int c, int64_t *out) {
  int l = a + b + c;
  if (a < 0 || b < 0 || c < 0 || l > OR_LMAX) return -1;
  opoly S;
  mcsh_poly(a, b, c, &S);
  for (int p = 0; p <= l; ++p)
    for (int q = 0; q <= l; ++q) out[p * (l + 1) + q] = (p + q <= l) ? S.c[p][q] : 0;
  return 0;
}

int oracle_max_order(void) { return OR_LMAX; }

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Step 1: neighbor images.                                             */
/* ------------------------------------------------------------------ */

static int struct_of(const oracle_problem *P, int64_t i) {
  int lo = 0, hi = P->n_struct - 1;
  while (lo < hi) {                      /* last s with atom_off[s] <= i */
    int mid = (lo + hi + 1) / 2;
    if (P->atom_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

/* 3x3 inverse by cofactors; returns 0 if singular. */
static int inv3(const double *A, double *Ai) {
  double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
               A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (det == 0.0 || !isfinite(det)) return 0;
  Ai[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  Ai[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  Ai[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  Ai[3] = (A[5] * A[6] - A[3] * A[8]) / det;
  Ai[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  Ai[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  Ai[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  Ai[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  Ai[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  return 1;
}

typedef struct {
  int32_t j;
  int32_t n[3];
  double d[3];
} opair;

/* All neighbor images of center i, in order (j ascending, then n1, n2, n3
 * ascending).  Image bounds per periodic axis k: with b_k the k-th column
 * of inv(cell) and df = frac_j - frac_i, any image within rc satisfies
 * |df_k + n_k| <= rc |b_k|; the loop takes one extra image on each side. */
static int64_t list_neighbors_at(const oracle_problem *P, int s, const double *xi, opair **out,
                                 int64_t *cap);

static int64_t list_neighbors(const oracle_problem *P, int64_t i, opair **out, int64_t *cap) {
  return list_neighbors_at(P, struct_of(P, i), P->pos + 3 * i, out, cap);
}

/* The same enumeration around an arbitrary point xi of structure s (the
 * center need not be an atom): d = (x_j - xi) + ((n1 a1 + n2 a2) + n3 a3). */
static int64_t list_neighbors_at(const oracle_problem *P, int s, const double *xi, opair **out,
                                 int64_t *cap) {
  const double *A = P->cell + 9 * s;
  const uint8_t *pb = P->pbc + 3 * s;
  int periodic = pb[0] || pb[1] || pb[2];
  double Ai[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  double reach[3] = {0, 0, 0};
  if (periodic) {
    if (!inv3(A, Ai)) return -1;
    for (int k = 0; k < 3; ++k) {
      double bk = sqrt(Ai[k] * Ai[k] + Ai[3 + k] * Ai[3 + k] + Ai[6 + k] * Ai[6 + k]);
      reach[k] = P->cutoff * bk;
    }
  }
  const double rc2 = P->cutoff * P->cutoff;
  double fi[3];
  for (int k = 0; k < 3; ++k) fi[k] = xi[0] * Ai[k] + xi[1] * Ai[3 + k] + xi[2] * Ai[6 + k];
  int64_t cnt = 0;
  for (int64_t j = P->atom_off[s]; j < P->atom_off[s + 1]; ++j) {
    const double *xj = P->pos + 3 * j;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) {
      if (!pb[k]) continue;
      double fj = xj[0] * Ai[k] + xj[1] * Ai[3 + k] + xj[2] * Ai[6 + k];
      double df = fj - fi[k];
      lo[k] = (int)floor(-reach[k] - df) - 1;
      hi[k] = (int)ceil(reach[k] - df) + 1;
    }
    for (int n1 = lo[0]; n1 <= hi[0]; ++n1)
      for (int n2 = lo[1]; n2 <= hi[1]; ++n2)
        for (int n3 = lo[2]; n3 <= hi[2]; ++n3) {
          double d[3];
          for (int k = 0; k < 3; ++k) {
            double shift = ((double)n1 * A[k] + (double)n2 * A[3 + k]) + (double)n3 * A[6 + k];
            d[k] = (xj[k] - xi[k]) + shift;
          }
          double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          if (!(r2 < rc2)) continue;
          if (cnt == *cap) {
            *cap = *cap ? 2 * *cap : 256;
            *out = (opair *)realloc(*out, (size_t)*cap * sizeof(opair));
          }
          opair *o = &(*out)[cnt++];
          o->j = (int32_t)j;
          o->n[0] = n1; o->n[1] = n2; o->n[2] = n3;
          o->d[0] = d[0]; o->d[1] = d[1]; o->d[2] = d[2];
        }
  }
  return cnt;
}

/* Number of neighbor images of each listed center (or -1 on a singular
 * periodic cell). */
int oracle_neighbor_counts(const oracle_problem *P, int64_t n_centers, const int64_t *centers,
                           int64_t *counts) {
  int bad = 0;
#pragma omp parallel
  {
    opair *buf = NULL;
    int64_t cap = 0;
#pragma omp for schedule(dynamic, 4)
    for (int64_t t = 0; t < n_centers; ++t) {
      counts[t] = list_neighbors(P, centers[t], &buf, &cap);
      if (counts[t] < 0) bad = 1;
    }
    free(buf);
  }
  return bad ? -1 : 0;
}

/* Neighbor lists of the listed centers, concatenated in center order;
 * offsets from oracle_neighbor_counts.  shift is [.,3]; d is [.,3]. */
int oracle_neighbor_lists(const oracle_problem *P, int64_t n_centers, const int64_t *centers,
                          const int64_t *offsets, int32_t *j_out, int32_t *shift_out,
                          double *d_out) {
  int bad = 0;
#pragma omp parallel
  {
    opair *buf = NULL;
    int64_t cap = 0;
#pragma omp for schedule(dynamic, 4)
    for (int64_t t = 0; t < n_centers; ++t) {
      int64_t m = list_neighbors(P, centers[t], &buf, &cap);
      if (m < 0 || m != offsets[t + 1] - offsets[t]) { bad = 1; continue; }
      for (int64_t u = 0; u < m; ++u) {
        int64_t o = offsets[t] + u;
        j_out[o] = buf[u].j;
        for (int k = 0; k < 3; ++k) {
          shift_out[3 * o + k] = buf[u].n[k];
          d_out[3 * o + k] = buf[u].d[k];
        }
      }
    }
    free(buf);
  }
  return bad ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Step 3: one pair's overlap integrals with every probe component.     */
/* ------------------------------------------------------------------ */

/* 1-D moments E[X^n], X ~ Normal(mean P, variance 1/(2 gamma)), n = 0..nmax. */
static void gauss_moments(double P, double gamma, int nmax, double *m) {
  double var = 0.5 / gamma;
  m[0] = 1.0;
  if (nmax >= 1) m[1] = P;
  for (int n = 1; n < nmax; ++n) m[n + 1] = P * m[n] + n * var * m[n - 1];
}

typedef struct {
  const oracle_problem *P;
  otable T;
  int F;                 /* number of features                              */
  int n_sig;
  int lmax;              /* highest non-negative order requested (-1: none) */
  int ncol;              /* (sum over requested l >= 0 of ncomp) * n_sig    */
  int col_off[16];       /* per order slot: first column of that order      */
  int has_density;
} octx;

static int ctx_init(octx *X, const oracle_problem *P) {
  X->P = P;
  build_table(&X->T);
  X->n_sig = P->n_sigmas;
  X->F = 0;
  X->lmax = -1;
  X->ncol = 0;
  X->has_density = 0;
  if (P->n_orders > 16) return -1;
  for (int o = 0; o < P->n_orders; ++o) {
    int l = P->orders[o];
    if (l < -1 || l > OR_LMAX) return -1;
    if (l == -1) { X->F += 1; X->has_density = 1; X->col_off[o] = -1; continue; }
    X->F += P->n_sigmas;
    if (l > X->lmax) X->lmax = l;
    X->col_off[o] = X->ncol;
    X->ncol += X->T.ncomp[l] * P->n_sigmas;
  }
  return 0;
}

/* Column of (order slot o, sigma s, component c). */
static inline int col_of(const octx *X, int o, int s, int c) {
  int l = X->P->orders[o];
  return X->col_off[o] + s * X->T.ncomp[l] + c;
}

/* Per-pair moment contributions t[col] (summed over the neighbor's
 * primitives) and, if dt != NULL, their derivatives dt[col][3] w.r.t. d.
 * Also the density term rho (order -1) and its gradient drho[3]. */
static void pair_terms(const octx *X, int e, const double d[3], double *t, double *dt,
                       double *rho, double *drho) {
  const oracle_problem *P = X->P;
  const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  memset(t, 0, sizeof(double) * X->ncol);
  if (dt) memset(dt, 0, sizeof(double) * 3 * X->ncol);
  *rho = 0.0;
  if (drho) drho[0] = drho[1] = drho[2] = 0.0;
  const int nmax = (X->lmax < 0 ? 0 : X->lmax) + 1;
  double mx[OR_LMAX + 3], my[OR_LMAX + 3], mz[OR_LMAX + 3];
  for (int k = P->gauss_off[e]; k < P->gauss_off[e + 1]; ++k) {
    const double alpha = P->gauss_exp[k], c = P->gauss_coef[k];
    /* order -1: the density of this primitive at the center */
    double g = c * exp(-alpha * r2);
    *rho += g;
    if (drho) /* d/dd exp(-alpha |d|^2) = -2 alpha d exp(-alpha |d|^2) */
      for (int a = 0; a < 3; ++a) drho[a] += -2.0 * alpha * d[a] * g;
    if (X->lmax < 0) continue;
    for (int s = 0; s < X->n_sig; ++s) {
      const double sig = P->sigmas[s];
      const double beta = 1.0 / (2.0 * sig * sig);
      const double gamma = alpha + beta;
      const double Nsig = pow(2.0 * M_PI * sig * sig, -1.5);
      /* Gaussian product theorem: exp(-beta r^2) exp(-alpha |r-d|^2)
       *   = exp(-(alpha beta/gamma)|d|^2) exp(-gamma |r - Pc|^2), Pc = (alpha/gamma) d */
      const double K = c * Nsig * pow(M_PI / gamma, 1.5) * exp(-(alpha * beta / gamma) * r2);
      double Pc[3] = {alpha / gamma * d[0], alpha / gamma * d[1], alpha / gamma * d[2]};
      gauss_moments(Pc[0], gamma, nmax, mx);
      gauss_moments(Pc[1], gamma, nmax, my);
      gauss_moments(Pc[2], gamma, nmax, mz);
      for (int o = 0; o < P->n_orders; ++o) {
        int l = P->orders[o];
        if (l < 0) continue;
        /* A neighbor image at d = 0 (the center's own atom) is a density
         * centred on the probe: its overlap with an order l >= 1 probe is
         * exactly 0 (S_abc is harmonic with no constant term, and a Gaussian
         * average of a harmonic polynomial is its value at the Gaussian's
         * centre, here the origin).  The monomial route of step 3 would
         * leave FP64 cancellation residue of ~2^-53 of its term magnitudes
         * instead; the derivative there is kept (the center's own images
         * never enter a gradient). */
        if (l >= 1 && r2 == 0.0 && !dt) continue;
        for (int ci = 0; ci < X->T.ncomp[l]; ++ci) {
          const ocomp *cp = &X->T.comp[l][ci];
          double v = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
          for (int u = 0; u < cp->nterm; ++u) {
            int p = cp->p[u], q = cp->q[u], r = cp->s[u];
            v += cp->coef[u] * mx[p] * my[q] * mz[r];
            if (dt) {
              jx += cp->coef[u] * mx[p + 1] * my[q] * mz[r];
              jy += cp->coef[u] * mx[p] * my[q + 1] * mz[r];
              jz += cp->coef[u] * mx[p] * my[q] * mz[r + 1];
            }
          }
          int col = col_of(X, o, s, ci);
          if (!(l >= 1 && r2 == 0.0)) t[col] += K * v;
          if (dt) {
            /* d/dd exp(-alpha|r-d|^2) = 2 alpha (r - d) exp(...):
             * d I/dd = 2 alpha K (E[X S(X)] - d E[S(X)]) */
            dt[3 * col + 0] += 2.0 * alpha * K * (jx - d[0] * v);
            dt[3 * col + 1] += 2.0 * alpha * K * (jy - d[1] * v);
            dt[3 * col + 2] += 2.0 * alpha * K * (jz - d[2] * v);
          }
        }
      }
    }
  }
}

/* ------------------------------------------------------------------ */
/* Steps 4-5: features of listed centers.                               */
/* ------------------------------------------------------------------ */

/* feat[t*F + f]: features; fabs[t*F + f] (optional): the same reduction
 * applied to the sums of |per-pair contribution| (the cancellation-free
 * scale of each feature); mu (optional): [n_centers, ncol] moments. */
static int features_impl(const oracle_problem *P, int64_t n_centers, const int64_t *centers,
                         const double *points, const int32_t *point_struct, double *feat,
                         double *fabs_out, double *mu_out);

int oracle_features(const oracle_problem *P, int64_t n_centers, const int64_t *centers,
                    double *feat, double *fabs_out, double *mu_out) {
  return features_impl(P, n_centers, centers, NULL, NULL, feat, fabs_out, mu_out);
}

/* Features at reference points (the paper's Overview section: the probes may
 * be centred on arbitrary points of a structure): points [n,3], point_struct [n]. */
int oracle_point_features(const oracle_problem *P, int64_t n_points, const double *points,
                          const int32_t *point_struct, double *feat, double *fabs_out) {
  return features_impl(P, n_points, NULL, points, point_struct, feat, fabs_out, NULL);
}

static int features_impl(const oracle_problem *P, int64_t n_centers, const int64_t *centers,
                         const double *points, const int32_t *point_struct, double *feat,
                         double *fabs_out, double *mu_out) {
  octx X;
  if (ctx_init(&X, P)) return -1;
  int bad = 0;
#pragma omp parallel
  {
    opair *buf = NULL;
    int64_t cap = 0;
    double *mu = (double *)calloc((size_t)X.ncol + 1, sizeof(double));
    double *ab = (double *)calloc((size_t)X.ncol + 1, sizeof(double));
    double *t = (double *)calloc((size_t)X.ncol + 1, sizeof(double));
#pragma omp for schedule(dynamic, 1)
    for (int64_t ti = 0; ti < n_centers; ++ti) {
      int64_t m = points ? list_neighbors_at(P, point_struct[ti], points + 3 * ti, &buf, &cap)
                         : list_neighbors(P, centers[ti], &buf, &cap);
      if (m < 0) { bad = 1; continue; }
      memset(mu, 0, sizeof(double) * X.ncol);
      memset(ab, 0, sizeof(double) * X.ncol);
      double rho = 0.0, rho_abs = 0.0;
      for (int64_t u = 0; u < m; ++u) {
        double r;
        pair_terms(&X, P->species[buf[u].j], buf[u].d, t, NULL, &r, NULL);
        for (int cI = 0; cI < X.ncol; ++cI) { mu[cI] += t[cI]; ab[cI] += fabs(t[cI]); }
        rho += r;
        rho_abs += fabs(r);
      }
      double *fo = feat + ti * X.F;
      double *fa = fabs_out ? fabs_out + ti * X.F : NULL;
      int f = 0;
      for (int o = 0; o < P->n_orders; ++o) {
        int l = P->orders[o];
        if (l < 0) {
          fo[f] = rho;
          if (fa) fa[f] = rho_abs;
          ++f;
          continue;
        }
        for (int s = 0; s < X.n_sig; ++s, ++f) {
          double acc = 0.0, acca = 0.0;
          for (int ci = 0; ci < X.T.ncomp[l]; ++ci) {
            int col = col_of(&X, o, s, ci);
            acc += X.T.comp[l][ci].w * mu[col] * mu[col];
            acca += X.T.comp[l][ci].w * ab[col] * ab[col];
          }
          fo[f] = acc;
          if (fa) fa[f] = acca;
        }
      }
      if (mu_out) memcpy(mu_out + ti * X.ncol, mu, sizeof(double) * X.ncol);
    }
    free(buf); free(mu); free(ab); free(t);
  }
  return bad ? -1 : 0;
}

int oracle_num_features(const oracle_problem *P) {
  octx X;
  if (ctx_init(&X, P)) return -1;
  return X.F;
}

int oracle_num_moment_columns(const oracle_problem *P) {
  octx X;
  if (ctx_init(&X, P)) return -1;
  return X.ncol;
}

/* Step 3 per pair, for inspection: the pairs of center i in list order
 * (oracle_neighbor_lists), each pair's moment contributions t[pair][col]
 * and their derivatives dt[pair][col][3] with respect to d.  m is the
 * pair count from oracle_neighbor_counts. */
int oracle_pair_terms(const oracle_problem *P, int64_t i, int64_t m, double *t_out, double *dt_out) {
  octx X;
  if (ctx_init(&X, P)) return -1;
  opair *buf = NULL;
  int64_t cap = 0;
  int64_t got = list_neighbors(P, i, &buf, &cap);
  if (got != m) { free(buf); return -1; }
  for (int64_t u = 0; u < m; ++u) {
    double r, dr[3];
    pair_terms(&X, P->species[buf[u].j], buf[u].d, t_out + u * X.ncol, dt_out + 3 * u * X.ncol, &r, dr);
  }
  free(buf);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Step 6: Jacobian rows d f_i / d x_j.                                 */
/* ------------------------------------------------------------------ */

/* Number of distinct neighbor atoms (the center included) of each center. */
int oracle_jacobian_counts(const oracle_problem *P, int64_t n_centers, const int64_t *centers,
                           int64_t *counts) {
  int bad = 0;
#pragma omp parallel
  {
    opair *buf = NULL;
    int64_t cap = 0;
#pragma omp for schedule(dynamic, 4)
    for (int64_t t = 0; t < n_centers; ++t) {
      int64_t m = list_neighbors(P, centers[t], &buf, &cap);
      if (m < 0) { bad = 1; counts[t] = 0; continue; }
      int64_t u = 0;
      for (int64_t a = 0; a < m; ++a)
        if (a == 0 || buf[a].j != buf[a - 1].j) ++u;
      counts[t] = u;
    }
    free(buf);
  }
  return bad ? -1 : 0;
}

/* For each listed center i: distinct neighbor atoms j (ascending) and the
 * blocks jac[., F, 3] = d f_i / d x_j.  Offsets from oracle_jacobian_counts.
 * jac_abs (optional) [., F]: the cancellation-free scale of each block,
 * sum over the block's pairs and components of 2 w_c A_c |d t_c / d d|
 * with A_c = sum over pairs of |t_c| (same for the center's own block,
 * summed over the other atoms' pairs); the scale against which an entry counts as near zero. */
int oracle_jacobian_rows(const oracle_problem *P, int64_t n_centers, const int64_t *centers,
                         const int64_t *offsets, int32_t *j_out, double *jac, double *jac_abs) {
  octx X;
  if (ctx_init(&X, P)) return -1;
  const int F = X.F;
  int bad = 0;
#pragma omp parallel
  {
    opair *buf = NULL;
    int64_t cap = 0;
    double *mu = (double *)calloc((size_t)X.ncol + 1, sizeof(double));
    double *t = (double *)calloc((size_t)X.ncol + 1, sizeof(double));
    double *dt = (double *)calloc(3 * (size_t)X.ncol + 1, sizeof(double));
    double *g = (double *)calloc(3 * (size_t)F, sizeof(double));   /* df/dd of one pair */
    double *self = (double *)calloc(3 * (size_t)F, sizeof(double));
    double *ab = (double *)calloc((size_t)X.ncol + 1, sizeof(double));
    double *ga = (double *)calloc((size_t)F, sizeof(double));
    double *self_abs = (double *)calloc((size_t)F, sizeof(double));
#pragma omp for schedule(dynamic, 1)
    for (int64_t ti = 0; ti < n_centers; ++ti) {
      const int64_t i = centers[ti];
      int64_t m = list_neighbors(P, i, &buf, &cap);
      if (m < 0) { bad = 1; continue; }
      /* forward moments of this center */
      memset(mu, 0, sizeof(double) * X.ncol);
      memset(ab, 0, sizeof(double) * X.ncol);
      for (int64_t u = 0; u < m; ++u) {
        double r;
        pair_terms(&X, P->species[buf[u].j], buf[u].d, t, NULL, &r, NULL);
        for (int cI = 0; cI < X.ncol; ++cI) { mu[cI] += t[cI]; ab[cI] += fabs(t[cI]); }
      }
      memset(self, 0, sizeof(double) * 3 * F);
      memset(self_abs, 0, sizeof(double) * F);
      int64_t row = offsets[ti] - 1, self_row = -1;
      for (int64_t u = 0; u < m; ++u) {
        if (u == 0 || buf[u].j != buf[u - 1].j) {
          ++row;
          if (row >= offsets[ti + 1]) { bad = 1; break; }
          j_out[row] = buf[u].j;
          memset(jac + row * 3 * F, 0, sizeof(double) * 3 * F);
          if (jac_abs) memset(jac_abs + row * F, 0, sizeof(double) * F);
          if (buf[u].j == i) self_row = row;
        }
        double r, dr[3];
        pair_terms(&X, P->species[buf[u].j], buf[u].d, t, dt, &r, dr);
        /* chain rule: df_{l,s}/dd = sum_c 2 w_c mu_c dmu_c/dd */
        int f = 0;
        for (int o = 0; o < P->n_orders; ++o) {
          int l = P->orders[o];
          if (l < 0) {
            for (int a = 0; a < 3; ++a) g[3 * f + a] = dr[a];
            ga[f] = sqrt(dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2]);
            ++f;
            continue;
          }
          for (int s = 0; s < X.n_sig; ++s, ++f) {
            double gx = 0.0, gy = 0.0, gz = 0.0, gabs = 0.0;
            for (int ci = 0; ci < X.T.ncomp[l]; ++ci) {
              int col = col_of(&X, o, s, ci);
              double wmu2 = 2.0 * X.T.comp[l][ci].w * mu[col];
              gx += wmu2 * dt[3 * col + 0];
              gy += wmu2 * dt[3 * col + 1];
              gz += wmu2 * dt[3 * col + 2];
              gabs += 2.0 * X.T.comp[l][ci].w * ab[col] *
                      sqrt(dt[3 * col] * dt[3 * col] + dt[3 * col + 1] * dt[3 * col + 1] +
                           dt[3 * col + 2] * dt[3 * col + 2]);
            }
            g[3 * f + 0] = gx; g[3 * f + 1] = gy; g[3 * f + 2] = gz;
            ga[f] = gabs;
          }
        }
        /* d = x_j - x_i + shift: +g onto atom j; -g onto the center unless
         * j is the center itself (its images move with it). */
        double *blk = jac + row * 3 * F;
        for (int q = 0; q < 3 * F; ++q) blk[q] += g[q];
        if (jac_abs)
          for (int q = 0; q < F; ++q) jac_abs[row * F + q] += ga[q];
        if (buf[u].j != i) {
          for (int q = 0; q < 3 * F; ++q) self[q] -= g[q];
          for (int q = 0; q < F; ++q) self_abs[q] += ga[q];
        }
      }
      if (self_row >= 0) {
        /* the center's own images cancel in pairs (d and -d) */
        double *blk = jac + self_row * 3 * F;
        memcpy(blk, self, sizeof(double) * 3 * F);
        if (jac_abs) memcpy(jac_abs + self_row * F, self_abs, sizeof(double) * F);
      } else {
        bad = 1;
      }
    }
    free(buf); free(mu); free(t); free(dt); free(g); free(self); free(ab); free(ga); free(self_abs);
  }
  return bad ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Strain derivative (virial).                                          */
/* ------------------------------------------------------------------ */

/* L = sum_i sum_f g[i,f] f_i.  Under a homogeneous strain x -> (I + eps) x
 * applied to positions and lattice vectors alike, every pair displacement
 * becomes (I + eps) d, so per structure s
 *   W[s][a][b] = dL/d eps_ab = sum over the pairs of s of (dL/dd)_a d_b,
 *   dL/dd = sum_f g[i,f] d f_i / d d   (the per-pair chain rule of the
 * Jacobian rows above).  W_abs (optional) [s][a][b]: the cancellation-free
 * scale sum over pairs of |g| . |d f/d d| |d_b|. */
int oracle_virial(const oracle_problem *P, const double *gcoef, double *W, double *W_abs) {
  octx X;
  if (ctx_init(&X, P)) return -1;
  const int F = X.F;
  const int64_t N = P->atom_off[P->n_struct];
  memset(W, 0, sizeof(double) * 9 * P->n_struct);
  if (W_abs) memset(W_abs, 0, sizeof(double) * 9 * P->n_struct);
  int bad = 0;
#pragma omp parallel
  {
    opair *buf = NULL;
    int64_t cap = 0;
    double *mu = (double *)calloc((size_t)X.ncol + 1, sizeof(double));
    double *ab = (double *)calloc((size_t)X.ncol + 1, sizeof(double));
    double *t = (double *)calloc((size_t)X.ncol + 1, sizeof(double));
    double *dt = (double *)calloc(3 * (size_t)X.ncol + 1, sizeof(double));
    double *Wt = (double *)calloc(9 * (size_t)P->n_struct, sizeof(double));
    double *Wa = (double *)calloc(9 * (size_t)P->n_struct, sizeof(double));
#pragma omp for schedule(dynamic, 1)
    for (int64_t i = 0; i < N; ++i) {
      int64_t m = list_neighbors(P, i, &buf, &cap);
      if (m < 0) { bad = 1; continue; }
      const int s = struct_of(P, i);
      const double *gi = gcoef + i * F;
      memset(mu, 0, sizeof(double) * X.ncol);
      memset(ab, 0, sizeof(double) * X.ncol);
      for (int64_t u = 0; u < m; ++u) {
        double r;
        pair_terms(&X, P->species[buf[u].j], buf[u].d, t, NULL, &r, NULL);
        for (int cI = 0; cI < X.ncol; ++cI) { mu[cI] += t[cI]; ab[cI] += fabs(t[cI]); }
      }
      for (int64_t u = 0; u < m; ++u) {
        double r, dr[3];
        pair_terms(&X, P->species[buf[u].j], buf[u].d, t, dt, &r, dr);
        double v[3] = {0.0, 0.0, 0.0}, vabs = 0.0;
        int f = 0;
        for (int o = 0; o < P->n_orders; ++o) {
          int l = P->orders[o];
          if (l < 0) {
            for (int a = 0; a < 3; ++a) v[a] += gi[f] * dr[a];
            vabs += fabs(gi[f]) * sqrt(dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2]);
            ++f;
            continue;
          }
          for (int sg = 0; sg < X.n_sig; ++sg, ++f) {
            for (int ci = 0; ci < X.T.ncomp[l]; ++ci) {
              int col = col_of(&X, o, sg, ci);
              double wmu2 = 2.0 * X.T.comp[l][ci].w * mu[col];
              for (int a = 0; a < 3; ++a) v[a] += gi[f] * wmu2 * dt[3 * col + a];
              vabs += fabs(gi[f]) * 2.0 * X.T.comp[l][ci].w * ab[col] *
                      sqrt(dt[3 * col] * dt[3 * col] + dt[3 * col + 1] * dt[3 * col + 1] +
                           dt[3 * col + 2] * dt[3 * col + 2]);
            }
          }
        }
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            Wt[9 * s + 3 * a + b] += v[a] * buf[u].d[b];
            Wa[9 * s + 3 * a + b] += vabs * fabs(buf[u].d[b]);
          }
      }
    }
#pragma omp critical
    {
      for (int64_t k = 0; k < 9 * (int64_t)P->n_struct; ++k) {
        W[k] += Wt[k];
        if (W_abs) W_abs[k] += Wa[k];
      }
    }
    free(buf); free(mu); free(ab); free(t); free(dt); free(Wt); free(Wa);
  }
  return bad ? -1 : 0;
}
