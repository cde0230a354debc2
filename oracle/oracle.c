/*
 * oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for cluster-TEBD.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA path.
 *
 * Everything is double precision complex, single-threaded, unblocked.  Each
 * function cites the passage of the paper (arXiv 2502.19289) it restates.
 *
 * Conventions (the same interface conventions the product documents):
 *   - qubits 0..n-1; big-endian basis: qubit 0 is the most significant bit
 *     (|x> = |x_0> (x) |x_1> (x) ..., Sec. IV.A);
 *   - bond b (0..n) sits left of qubit b; chi[0] = chi[n] = 1;
 *   - site q is a row-major (chi[q], 2, chi[q+1]) complex tensor;
 *   - the MPS is kept in right-canonical Vidal form: right isometries B_q
 *     plus the bond spectra lambda_b (reading of Sec. II.C and Sec. V for
 *     several clusters updated independently; see the cluster update below).
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 */
#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-2)
#define ORC_ERR_STATE (-6)

/* gate codes: the shared input format (see synth/__init__.py) */
enum {
  K_H = 1, K_X, K_Y, K_Z, K_S, K_T, K_P, K_X14, K_SQW,
  K_CNOT = 10, K_CY, K_CZ, K_SWAP, K_CH, K_CS, K_CT, K_SQSWAP, K_CP
};

/* ------------------------------------------------------------------------ */
/* App. A: gate matrices.  Two-qubit matrices are indexed 2*x_first+x_second */
/* (first listed qubit = control = most significant).                        */
/* ------------------------------------------------------------------------ */
static int gate_matrix(int kind, double param, cplx *g) {
  const double r2 = 1.0 / sqrt(2.0);
  const cplx I1 = I;
  const cplx w8 = cexp(I1 * M_PI / 4.0); /* e^{i pi/4} */
  switch (kind) {
    case K_H: g[0] = r2; g[1] = r2; g[2] = r2; g[3] = -r2; return 2;
    case K_X: g[0] = 0; g[1] = 1; g[2] = 1; g[3] = 0; return 2;
    case K_Y: g[0] = 0; g[1] = -I1; g[2] = I1; g[3] = 0; return 2;
    case K_Z: g[0] = 1; g[1] = 0; g[2] = 0; g[3] = -1; return 2;
    case K_S: g[0] = 1; g[1] = 0; g[2] = 0; g[3] = I1; return 2;      /* P(pi/2) */
    case K_T: g[0] = 1; g[1] = 0; g[2] = 0; g[3] = w8; return 2;      /* P(pi/4) */
    case K_P: g[0] = 1; g[1] = 0; g[2] = 0; g[3] = cexp(I1 * param); return 2;
    case K_X14: {                                                      /* X^(1/4) */
      cplx ph = cexp(I1 * M_PI / 8.0);
      double c = cos(M_PI / 8.0), s = sin(M_PI / 8.0);
      g[0] = ph * c; g[1] = -I1 * ph * s; g[2] = -I1 * ph * s; g[3] = ph * c;
      return 2;
    }
    case K_SQW:
      /* principal square root of W=(X+Y)/sqrt2; the printed matrix has the
         sign of the exponent flipped and is not unitary (App. A reading). */
      g[0] = r2 * w8; g[1] = -I1 * r2; g[2] = r2; g[3] = r2 * w8; return 2;
    default: break;
  }
  for (int i = 0; i < 16; i++) g[i] = 0;
  g[0] = 1; g[5] = 1;
  switch (kind) {
    case K_CNOT: g[11] = 1; g[14] = 1; return 4;
    case K_CY: g[11] = -I1; g[14] = I1; return 4;
    case K_CZ: g[10] = 1; g[15] = -1; return 4;
    case K_SWAP: g[5] = 0; g[6] = 1; g[9] = 1; g[15] = 1; return 4;
    case K_CH: g[10] = r2; g[11] = r2; g[14] = r2; g[15] = -r2; return 4;
    case K_CS: g[10] = 1; g[15] = I1; return 4;                        /* C-P(pi/2) */
    case K_CT: g[10] = 1; g[15] = w8; return 4;
    case K_CP: g[10] = 1; g[15] = cexp(I1 * param); return 4;
    case K_SQSWAP:
      g[5] = 0.5 * (1 + I1); g[6] = 0.5 * (1 - I1);
      g[9] = 0.5 * (1 - I1); g[10] = 0.5 * (1 + I1); g[15] = 1; return 4;
    default: return 0;
  }
}

int orc_gate_matrix(int kind, double param, double *out) {
  cplx g[16];
  int d = gate_matrix(kind, param, g);
  if (!d) return ORC_ERR_ARG;
  for (int i = 0; i < d * d; i++) { out[2 * i] = creal(g[i]); out[2 * i + 1] = cimag(g[i]); }
  return d;
}

/* ------------------------------------------------------------------------ */
/* Sec. II.A: a gate belongs to the earliest layer after the last gate on any */
/* of its qubits.  Layers are 1-indexed.  Returns the number of layers.       */
/* ------------------------------------------------------------------------ */
int orc_asap(int n, int ng, const int *g5, int *layer) {
  int *last = calloc((size_t)n, sizeof(int));
  int nl = 0;
  if (!last) return ORC_ERR_OOM;
  for (int i = 0; i < ng; i++) {
    const int *g = g5 + 5 * i;
    int L = 0;
    for (int t = 0; t < g[0]; t++) {
      int q = g[1 + t];
      if (q < 0 || q >= n) { free(last); return ORC_ERR_ARG; }
      if (last[q] > L) L = last[q];
    }
    L += 1;
    layer[i] = L;
    for (int t = 0; t < g[0]; t++) last[g[1 + t]] = L;
    if (L > nl) nl = L;
  }
  free(last);
  return nl;
}

/* ------------------------------------------------------------------------ */
/* Sec. III.A, Eqs. 6-8: cluster partition for one cluster-TEBD iteration.    */
/* bond[b] (b = 1..n-1) marks the bond left of qubit b (paper's entry b-1 in  */
/* 1-indexed notation).  A run of marked bonds b1..b2 is a cluster of qubits  */
/* b1-1..b2, k = b2-b1+2 (size q_n - q_1 + 2), bounded by chi[b1-1] and       */
/* chi[b2+1] (the off-by-one reading of the external bond indices).          */
/* The iteration contracts up to the last layer L* for which every cluster    */
/* satisfies log2(2^k chi_L chi_R) <= Q_max (Eq. 7), k <= k_max, and the      */
/* number of layers in the step is <= L_max (Eq. 8; l_max <= 0 = unbounded).  */
/* ------------------------------------------------------------------------ */
static int runs_ok(int n, const unsigned char *bond, const long long *chi, int q_max, int k_max) {
  int b = 1;
  while (b <= n - 1) {
    if (!bond[b]) { b++; continue; }
    int b1 = b;
    while (b <= n - 1 && bond[b]) b++;
    int b2 = b - 1;
    int k = b2 - b1 + 2;
    if (k_max > 0 && k > k_max) return 0;
    if (k > 100) return 0;
    unsigned __int128 size = ((unsigned __int128)1 << k) *
                             (unsigned __int128)chi[b1 - 1] * (unsigned __int128)chi[b2 + 1];
    unsigned __int128 lim = (q_max >= 120) ? ~(unsigned __int128)0 : ((unsigned __int128)1 << q_max);
    if (size > lim) return 0;
  }
  return 1;
}

int orc_partition(int n, int ng, const int *g5, const int *layer, int n_layers, int start,
                  const long long *chi, int q_max, int l_max, int k_max,
                  int *out_q0, int *out_k, int cap, int *n_out, int *stop) {
  unsigned char *bond = calloc((size_t)n + 1, 1), *tent = calloc((size_t)n + 1, 1);
  int Lstar = start, rc = ORC_OK;
  if (!bond || !tent) { free(bond); free(tent); return ORC_ERR_OOM; }
  for (int L = start + 1; L <= n_layers; L++) {
    if (l_max > 0 && L - start > l_max) break;
    memcpy(tent, bond, (size_t)n + 1);
    for (int i = 0; i < ng; i++) {
      const int *g = g5 + 5 * i;
      if (layer[i] != L || g[0] < 2) continue;
      int lo = g[1], hi = g[1];
      for (int t = 1; t < g[0]; t++) { if (g[1 + t] < lo) lo = g[1 + t]; if (g[1 + t] > hi) hi = g[1 + t]; }
      if (hi - lo != g[0] - 1) { rc = ORC_ERR_ARG; goto done; } /* not contiguous */
      for (int b = lo + 1; b <= hi; b++) tent[b] = 1;
    }
    if (!runs_ok(n, tent, chi, q_max, k_max)) break;
    memcpy(bond, tent, (size_t)n + 1);
    Lstar = L;
  }
  if (Lstar == start && start < n_layers) { rc = ORC_ERR_STATE; goto done; }
  {
    int nc = 0, b = 1;
    while (b <= n - 1) {
      if (!bond[b]) { b++; continue; }
      int b1 = b;
      while (b <= n - 1 && bond[b]) b++;
      if (nc < cap) { out_q0[nc] = b1 - 1; out_k[nc] = b - 1 - b1 + 2; }
      nc++;
    }
    *n_out = nc;
    if (nc > cap) rc = ORC_ERR_ARG;
  }
  *stop = Lstar;
done:
  free(bond); free(tent);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. II.A: state-vector simulation, gates applied in time order.          */
/* ------------------------------------------------------------------------ */
static void apply_gate_vec(int nq, cplx *psi, int gnq, const int *lq, const cplx *g) {
  const int dim = 1 << gnq;
  const long long N = 1LL << nq;
  long long mask = 0;
  int pos[3];
  for (int t = 0; t < gnq; t++) { pos[t] = nq - 1 - lq[t]; mask |= 1LL << pos[t]; }
  cplx v[8], w[8];
  long long idx[8];
  for (long long base = 0; base < N; base++) {
    if (base & mask) continue;
    for (int x = 0; x < dim; x++) {
      long long i = base;
      for (int t = 0; t < gnq; t++)
        if ((x >> (gnq - 1 - t)) & 1) i |= 1LL << pos[t];
      idx[x] = i;
      v[x] = psi[i];
    }
    for (int a = 0; a < dim; a++) {
      cplx acc = 0;
      for (int b = 0; b < dim; b++) acc += g[a * dim + b] * v[b];
      w[a] = acc;
    }
    for (int x = 0; x < dim; x++) psi[idx[x]] = w[x];
  }
}

int orc_statevector(int n, int ng, const int *g5, const double *params, double *psi_out) {
  if (n > 26) return ORC_ERR_ARG;
  long long N = 1LL << n;
  cplx *psi = calloc((size_t)N, sizeof(cplx));
  if (!psi) return ORC_ERR_OOM;
  psi[0] = 1;
  for (int i = 0; i < ng; i++) {
    const int *g = g5 + 5 * i;
    cplx m[16];
    int d = gate_matrix(g[4], params[i], m);
    if (!d || (d == 2) != (g[0] == 1)) { free(psi); return ORC_ERR_ARG; }
    apply_gate_vec(n, psi, g[0], g + 1, m);
  }
  for (long long i = 0; i < N; i++) { psi_out[2 * i] = creal(psi[i]); psi_out[2 * i + 1] = cimag(psi[i]); }
  free(psi);
  return ORC_OK;
}

/* U_c: ordered product of the gates in layers (lo, hi] acting inside the     */
/* qubit window [q0, q0+k) -- the exactly contracted cluster (Sec. III.A).     */
/* Row-major 2^k x 2^k, big-endian over the window (q0 is the MSB).            */
static int cluster_unitary(int q0, int k, int ng, const int *g5, const double *params,
                           const int *layer, int lo, int hi, cplx *U) {
  const int D = 1 << k;
  cplx *col = malloc(sizeof(cplx) * (size_t)D);
  if (!col) return ORC_ERR_OOM;
  for (int i = 0; i < D * D; i++) U[i] = 0;
  for (int i = 0; i < D; i++) U[i * D + i] = 1;
  for (int i = 0; i < ng; i++) {
    if (layer[i] <= lo || layer[i] > hi) continue;
    const int *g = g5 + 5 * i;
    int in = 0, lq[3];
    for (int t = 0; t < g[0]; t++) {
      lq[t] = g[1 + t] - q0;
      if (lq[t] >= 0 && lq[t] < k) in++;
    }
    if (in == 0) continue;
    if (in != g[0]) { free(col); return ORC_ERR_ARG; } /* gate straddles the window */
    cplx m[16];
    if (!gate_matrix(g[4], params[i], m)) { free(col); return ORC_ERR_ARG; }
    for (int c = 0; c < D; c++) {
      for (int r = 0; r < D; r++) col[r] = U[r * D + c];
      apply_gate_vec(k, col, g[0], lq, m);
      for (int r = 0; r < D; r++) U[r * D + c] = col[r];
    }
  }
  free(col);
  return ORC_OK;
}

int orc_cluster_unitary(int q0, int k, int ng, const int *g5, const double *params,
                        const int *layer, int lo, int hi, double *out) {
  const int D = 1 << k;
  cplx *U = malloc(sizeof(cplx) * (size_t)D * D);
  if (!U) return ORC_ERR_OOM;
  int rc = cluster_unitary(q0, k, ng, g5, params, layer, lo, hi, U);
  for (int i = 0; i < D * D; i++) { out[2 * i] = creal(U[i]); out[2 * i + 1] = cimag(U[i]); }
  free(U);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Truncated SVD building block (Fig. 3): one-sided Jacobi (Hestenes),       */
/* LAPACK-free.  Orthogonalises the columns of A (rows x cols, column-major), */
/* accumulating the rotations in V so that A_in V = A_out.                    */
/* ------------------------------------------------------------------------ */
static void hestenes(int rows, int cols, cplx *A, cplx *V) {
  const double tol = 1e-15 * sqrt((double)(rows > 1 ? rows : 1));
  /* A column whose norm is below eps * ||A||_F is a numerical zero: it adds */
  /* at most that much to any singular value, and rotating against it is     */
  /* meaningless.  Its inner products can be subnormal, and the phase        */
  /* gamma / |gamma| of a subnormal gamma is not of unit modulus, which would */
  /* make V non-unitary.  Such pairs are skipped.                            */
  double fro = 0;
  for (size_t i = 0; i < (size_t)rows * cols; i++) fro += creal(A[i]) * creal(A[i]) + cimag(A[i]) * cimag(A[i]);
  const double zero2 = DBL_EPSILON * DBL_EPSILON * fro;
  for (int i = 0; i < cols * cols; i++) V[i] = 0;
  for (int i = 0; i < cols; i++) V[i * cols + i] = 1;
  for (int sweep = 0; sweep < 80; sweep++) {
    int rotated = 0;
    for (int p = 0; p < cols - 1; p++) {
      for (int q = p + 1; q < cols; q++) {
        cplx *ap = A + (size_t)p * rows, *aq = A + (size_t)q * rows;
        double alpha = 0, beta = 0;
        cplx gamma = 0;
        for (int i = 0; i < rows; i++) {
          alpha += creal(ap[i]) * creal(ap[i]) + cimag(ap[i]) * cimag(ap[i]);
          beta += creal(aq[i]) * creal(aq[i]) + cimag(aq[i]) * cimag(aq[i]);
          gamma += conj(ap[i]) * aq[i];
        }
        double g = cabs(gamma);
        if (g == 0.0 || alpha <= zero2 || beta <= zero2 || g <= tol * sqrt(alpha * beta)) continue;
        rotated = 1;
        cplx ph = conj(gamma / g); /* e^{-i phi} */
        double zeta = (beta - alpha) / (2.0 * g);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int i = 0; i < rows; i++) {
          cplx x = ap[i], y = aq[i] * ph;
          ap[i] = c * x - s * y;
          aq[i] = s * x + c * y;
        }
        cplx *vp = V + (size_t)p * cols, *vq = V + (size_t)q * cols;
        for (int i = 0; i < cols; i++) {
          cplx x = vp[i], y = vq[i] * ph;
          vp[i] = c * x - s * y;
          vq[i] = s * x + c * y;
        }
      }
    }
    if (!rotated) break;
  }
}

static double colnorm(int rows, const cplx *a) {
  double s = 0;
  for (int i = 0; i < rows; i++) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
  return sqrt(s);
}

/* order[] = indices sorted by value descending (stable insertion sort). */
static void argsort_desc(int n, const double *v, int *order) {
  for (int i = 0; i < n; i++) order[i] = i;
  for (int i = 1; i < n; i++) {
    int o = order[i], j = i - 1;
    while (j >= 0 && v[order[j]] < v[o]) { order[j + 1] = order[j]; j--; }
    order[j + 1] = o;
  }
}

/* Singular values (descending) and right singular vectors of M (m x n,
   row-major).  p = min(m,n) values; Y is n x p row-major with column mu the
   right singular vector of s[mu].  For m < n the Jacobi runs on M^dagger,
   whose orthogonalised columns are the right vectors scaled by s. */
static int svd_right(int m, int n, const cplx *M, double *s, cplx *Y) {
  int p = m < n ? m : n;
  if (m >= n) {
    cplx *A = malloc(sizeof(cplx) * (size_t)m * n), *V = malloc(sizeof(cplx) * (size_t)n * n);
    double *sv = malloc(sizeof(double) * (size_t)n);
    int *ord = malloc(sizeof(int) * (size_t)n);
    if (!A || !V || !sv || !ord) { free(A); free(V); free(sv); free(ord); return ORC_ERR_OOM; }
    for (int i = 0; i < m; i++)
      for (int c = 0; c < n; c++) A[(size_t)c * m + i] = M[(size_t)i * n + c];
    hestenes(m, n, A, V);
    for (int c = 0; c < n; c++) sv[c] = colnorm(m, A + (size_t)c * m);
    argsort_desc(n, sv, ord);
    for (int mu = 0; mu < p; mu++) {
      s[mu] = sv[ord[mu]];
      for (int r = 0; r < n; r++) Y[(size_t)r * p + mu] = V[(size_t)ord[mu] * n + r];
    }
    free(A); free(V); free(sv); free(ord);
  } else {
    cplx *A = malloc(sizeof(cplx) * (size_t)m * n), *V = malloc(sizeof(cplx) * (size_t)m * m);
    double *sv = malloc(sizeof(double) * (size_t)m);
    int *ord = malloc(sizeof(int) * (size_t)m);
    if (!A || !V || !sv || !ord) { free(A); free(V); free(sv); free(ord); return ORC_ERR_OOM; }
    for (int i = 0; i < m; i++)
      for (int c = 0; c < n; c++) A[(size_t)i * n + c] = conj(M[(size_t)i * n + c]);
    hestenes(n, m, A, V);
    for (int i = 0; i < m; i++) sv[i] = colnorm(n, A + (size_t)i * n);
    argsort_desc(m, sv, ord);
    for (int mu = 0; mu < p; mu++) {
      double sig = sv[ord[mu]];
      s[mu] = sig;
      for (int r = 0; r < n; r++)
        Y[(size_t)r * p + mu] = sig > 0 ? A[(size_t)ord[mu] * n + r] / sig : 0;
    }
    free(A); free(V); free(sv); free(ord);
  }
  return ORC_OK;
}

int orc_svd(int m, int n, const double *Mri, double *s, double *Yri) {
  int p = m < n ? m : n;
  cplx *M = malloc(sizeof(cplx) * (size_t)m * n), *Y = malloc(sizeof(cplx) * (size_t)n * p);
  if (!M || !Y) { free(M); free(Y); return ORC_ERR_OOM; }
  for (size_t i = 0; i < (size_t)m * n; i++) M[i] = Mri[2 * i] + I * Mri[2 * i + 1];
  int rc = svd_right(m, n, M, s, Y);
  for (size_t i = 0; i < (size_t)n * p; i++) { Yri[2 * i] = creal(Y[i]); Yri[2 * i + 1] = cimag(Y[i]); }
  free(M); free(Y);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Truncation rule (Sec. II.B, Fig. 3), in the discarded-weight reading:      */
/* r = smallest r >= 1 with sum_{mu>r} s^2 <= eta * sum s^2 (eta = 0 keeps    */
/* everything), values s <= floor * s_1 are numerical zeros and are dropped,  */
/* and r <= chi_max.                                                          */
/* ------------------------------------------------------------------------ */
static int truncation_rank(int p, const double *s, int chi_max, double eta, double floor_rel) {
  double W = 0;
  for (int i = 0; i < p; i++) W += s[i] * s[i];
  int r = p;
  if (eta > 0) {
    double tail = 0;
    r = 1;
    for (int i = p - 1; i >= 1; i--) {
      tail += s[i] * s[i];
      if (tail > eta * W) { r = i + 1; break; }
    }
  }
  int nz = 0;
  for (int i = 0; i < p; i++) if (s[i] > floor_rel * s[0]) nz++;
  if (nz < r) r = nz;
  if (r > chi_max) r = chi_max;
  if (r < 1) r = 1;
  return r;
}

/* ------------------------------------------------------------------------ */
/* MPS store                                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int n;
  long long *chi;
  cplx **site;
  double **lam;
  double *log;   /* split records, 9 doubles each */
  int nlog, caplog;
  int nstep;
  double logF;
} orc_mps;

static void log_split(orc_mps *h, int q0, int k, int bond, int m, int n, int r, double f, double W) {
  if (h->nlog == h->caplog) {
    int nc = h->caplog ? 2 * h->caplog : 256;
    double *nl = realloc(h->log, sizeof(double) * 9 * (size_t)nc);
    if (!nl) return;
    h->log = nl; h->caplog = nc;
  }
  double *e = h->log + 9 * (size_t)h->nlog++;
  e[0] = h->nstep; e[1] = q0; e[2] = k; e[3] = bond; e[4] = m; e[5] = n; e[6] = r; e[7] = f; e[8] = W;
}

orc_mps *orc_mps_new(int n) {
  orc_mps *h = calloc(1, sizeof(orc_mps));
  if (!h) return NULL;
  h->n = n;
  h->chi = calloc((size_t)n + 1, sizeof(long long));
  h->site = calloc((size_t)n, sizeof(cplx *));
  h->lam = calloc((size_t)n + 1, sizeof(double *));
  for (int b = 0; b <= n; b++) { h->chi[b] = 1; h->lam[b] = malloc(sizeof(double)); h->lam[b][0] = 1; }
  for (int q = 0; q < n; q++) { h->site[q] = calloc(2, sizeof(cplx)); h->site[q][0] = 1; } /* |0> */
  return h;
}

void orc_mps_free(orc_mps *h) {
  if (!h) return;
  for (int q = 0; q < h->n; q++) free(h->site[q]);
  for (int b = 0; b <= h->n; b++) free(h->lam[b]);
  free(h->site); free(h->lam); free(h->chi); free(h->log); free(h);
}

int orc_mps_set_site(orc_mps *h, int q, long long cl, long long cr, const double *ri) {
  if (q < 0 || q >= h->n) return ORC_ERR_ARG;
  cplx *s = malloc(sizeof(cplx) * (size_t)(cl * 2 * cr));
  if (!s) return ORC_ERR_OOM;
  for (long long i = 0; i < cl * 2 * cr; i++) s[i] = ri[2 * i] + I * ri[2 * i + 1];
  free(h->site[q]);
  h->site[q] = s;
  h->chi[q] = cl; h->chi[q + 1] = cr;
  return ORC_OK;
}

int orc_mps_set_lambda(orc_mps *h, int b, long long c, const double *v) {
  if (b < 0 || b > h->n) return ORC_ERR_ARG;
  double *l = malloc(sizeof(double) * (size_t)c);
  if (!l) return ORC_ERR_OOM;
  memcpy(l, v, sizeof(double) * (size_t)c);
  free(h->lam[b]);
  h->lam[b] = l;
  h->chi[b] = c;
  return ORC_OK;
}

void orc_mps_get_chi(const orc_mps *h, long long *out) { memcpy(out, h->chi, sizeof(long long) * (size_t)(h->n + 1)); }

void orc_mps_get_site(const orc_mps *h, int q, double *out) {
  long long sz = h->chi[q] * 2 * h->chi[q + 1];
  for (long long i = 0; i < sz; i++) { out[2 * i] = creal(h->site[q][i]); out[2 * i + 1] = cimag(h->site[q][i]); }
}

void orc_mps_get_lambda(const orc_mps *h, int b, double *out) { memcpy(out, h->lam[b], sizeof(double) * (size_t)h->chi[b]); }
double orc_mps_logF(const orc_mps *h) { return h->logF; }
int orc_mps_nlog(const orc_mps *h) { return h->nlog; }
void orc_mps_get_log(const orc_mps *h, double *out) { memcpy(out, h->log, sizeof(double) * 9 * (size_t)h->nlog); }
int orc_mps_nstep(const orc_mps *h) { return h->nstep; }

/* G5 reading: a one-qubit gate outside every cluster acts on its site's     */
/* physical index directly; unitary, so right-canonicity is preserved.       */
static void apply_1q_site(orc_mps *h, int q, const cplx *u) {
  long long cl = h->chi[q], cr = h->chi[q + 1];
  cplx *s = h->site[q];
  for (long long a = 0; a < cl; a++)
    for (long long b = 0; b < cr; b++) {
      cplx x0 = s[(a * 2 + 0) * cr + b], x1 = s[(a * 2 + 1) * cr + b];
      s[(a * 2 + 0) * cr + b] = u[0] * x0 + u[1] * x1;
      s[(a * 2 + 1) * cr + b] = u[2] * x0 + u[3] * x1;
    }
}

int orc_apply_1q(orc_mps *h, int q, const double *ri) {
  cplx u[4];
  for (int i = 0; i < 4; i++) u[i] = ri[2 * i] + I * ri[2 * i + 1];
  apply_1q_site(h, q, u);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* One cluster update, Sec. III.A: exact contraction of the cluster (merge    */
/* of its k sites with U_c applied to the physical indices), then successive  */
/* truncated SVDs back into k sites (Fig. 2, Fig. 3), per-split fidelity f_j  */
/* (Eq. 4, with squares), accumulated into log F (Eq. 5).                     */
/*                                                                            */
/* Gauge (the paper leaves it open when several clusters are contracted       */
/* independently): sites are right isometries B and bonds carry spectra       */
/* lambda, so theta = diag(lambda_L) * (B_q ... B_{q+k-1}) holds the Schmidt   */
/* weights.  Splits go right to left; each new right site is Y^dagger (a      */
/* right isometry); the remainder is carried *unweighted* (R = Mbar * Y_r) so  */
/* the leftmost site never divides by lambda_L.  Kept values are renormalised  */
/* to unit weight; the discarded weight is accounted for by f_j.              */
/* ------------------------------------------------------------------------ */
static int cluster_update(orc_mps *h, int q0, int k, const cplx *U, int chi_max, double eta,
                          double floor_rel, double *f_out, int *r_out) {
  const int n = h->n;
  if (q0 < 0 || k < 1 || q0 + k > n) return ORC_ERR_ARG;
  const long long cL = h->chi[q0], cR = h->chi[q0 + k];
  const long long D = 1LL << k;
  /* merge: T (rows x cur) <- T * B_{q0+j} viewed as (cur x 2 chi') */
  long long rows = cL * 2, cur = h->chi[q0 + 1];
  cplx *T = malloc(sizeof(cplx) * (size_t)(rows * cur));
  if (!T) return ORC_ERR_OOM;
  memcpy(T, h->site[q0], sizeof(cplx) * (size_t)(rows * cur));
  for (int j = 1; j < k; j++) {
    long long nxt = h->chi[q0 + j + 1];
    cplx *T2 = calloc((size_t)(rows * 2 * nxt), sizeof(cplx));
    if (!T2) { free(T); return ORC_ERR_OOM; }
    const cplx *B = h->site[q0 + j];
    for (long long i = 0; i < rows; i++)
      for (long long c = 0; c < cur; c++) {
        cplx t = T[i * cur + c];
        if (t == 0) continue;
        for (long long o = 0; o < 2 * nxt; o++) T2[i * 2 * nxt + o] += t * B[c * 2 * nxt + o];
      }
    free(T);
    T = T2;
    rows *= 2;
    cur = nxt;
  }
  /* T is theta_bar (cL, 2^k, cR); apply U on the physical multi-index */
  cplx *R = calloc((size_t)(cL * D * cR), sizeof(cplx));
  if (!R) { free(T); return ORC_ERR_OOM; }
  for (long long a = 0; a < cL; a++)
    for (long long sp = 0; sp < D; sp++)
      for (long long s = 0; s < D; s++) {
        cplx u = U[sp * D + s];
        if (u == 0) continue;
        const cplx *src = T + (a * D + s) * cR;
        cplx *dst = R + (a * D + sp) * cR;
        for (long long b = 0; b < cR; b++) dst[b] += u * src[b];
      }
  free(T);
  /* successive splits, right to left */
  long long rdim = cR;
  const double *lamL = h->lam[q0];
  for (int j = k - 1; j >= 1; j--) {
    long long m = cL << j, nn = 2 * rdim;
    long long p = m < nn ? m : nn;
    cplx *M = malloc(sizeof(cplx) * (size_t)(m * nn));
    double *s = malloc(sizeof(double) * (size_t)p);
    cplx *Y = malloc(sizeof(cplx) * (size_t)(nn * p));
    if (!M || !s || !Y) { free(M); free(s); free(Y); free(R); return ORC_ERR_OOM; }
    for (long long i = 0; i < m; i++) {
      double w = lamL[i >> j];
      for (long long c = 0; c < nn; c++) M[i * nn + c] = w * R[i * nn + c];
    }
    int rc = svd_right((int)m, (int)nn, M, s, Y);
    if (rc) { free(M); free(s); free(Y); free(R); return rc; }
    double W = 0, kept = 0;
    for (long long i = 0; i < p; i++) W += s[i] * s[i];
    int r = truncation_rank((int)p, s, chi_max, eta, floor_rel);
    for (int i = 0; i < r; i++) kept += s[i] * s[i];
    double f = W > 0 ? kept / W : 1.0;
    double nrm = sqrt(kept);
    int bnd = q0 + j;
    /* new right site B_{q0+j} = (Y_r)^dagger as (r, 2, rdim) */
    cplx *B = malloc(sizeof(cplx) * (size_t)(r * nn));
    double *lam = malloc(sizeof(double) * (size_t)r);
    cplx *Rn = calloc((size_t)(m * r), sizeof(cplx));
    if (!B || !lam || !Rn) { free(M); free(s); free(Y); free(R); free(B); free(lam); free(Rn); return ORC_ERR_OOM; }
    for (int mu = 0; mu < r; mu++) {
      for (long long c = 0; c < nn; c++) B[mu * nn + c] = conj(Y[c * p + mu]);
      lam[mu] = s[mu] / nrm;
    }
    /* unweighted remainder R_new = Rbar * Y_r / sqrt(kept) */
    for (long long i = 0; i < m; i++)
      for (long long c = 0; c < nn; c++) {
        cplx x = R[i * nn + c];
        if (x == 0) continue;
        for (int mu = 0; mu < r; mu++) Rn[i * r + mu] += x * Y[c * p + mu];
      }
    for (long long i = 0; i < m * r; i++) Rn[i] /= nrm;
    free(h->site[bnd]); h->site[bnd] = B;
    free(h->lam[bnd]); h->lam[bnd] = lam;
    h->chi[bnd] = r;
    if (f_out) f_out[k - 1 - j] = f;
    if (r_out) r_out[k - 1 - j] = r;
    h->logF += log(f);
    log_split(h, q0, k, bnd, (int)m, (int)nn, r, f, W);
    free(M); free(s); free(Y); free(R);
    R = Rn;
    rdim = r;
  }
  free(h->site[q0]);
  h->site[q0] = R; /* (cL * 2) x rdim == (cL, 2, chi[q0+1]) */
  return ORC_OK;
}

int orc_cluster_update(orc_mps *h, int q0, int k, const double *Uri, int chi_max, double eta,
                       double floor_rel, double *f_out, int *r_out) {
  const long long D = 1LL << k;
  cplx *U = malloc(sizeof(cplx) * (size_t)(D * D));
  if (!U) return ORC_ERR_OOM;
  for (long long i = 0; i < D * D; i++) U[i] = Uri[2 * i] + I * Uri[2 * i + 1];
  int rc = cluster_update(h, q0, k, U, chi_max, eta, floor_rel, f_out, r_out);
  free(U);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. III.A, full iteration loop: partition -> contract every cluster up to */
/* L* -> decompose -> restart from the new MPS until all gates are applied.   */
/* With l_max = 1 and k_max = 2 this is standard TEBD (Sec. II.C) in the same */
/* gauge: one layer per iteration, one split per two-qubit gate.             */
/* ------------------------------------------------------------------------ */
int orc_run(orc_mps *h, int ng, const int *g5, const double *params, int chi_max, double eta,
            int q_max, int l_max, int k_max, double floor_rel) {
  const int n = h->n;
  int *layer = malloc(sizeof(int) * (size_t)(ng > 0 ? ng : 1));
  int *cq = malloc(sizeof(int) * (size_t)n), *ck = malloc(sizeof(int) * (size_t)n);
  unsigned char *inc = malloc((size_t)n);
  int rc = ORC_OK;
  if (!layer || !cq || !ck || !inc) { rc = ORC_ERR_OOM; goto out; }
  int nl = orc_asap(n, ng, g5, layer);
  if (nl < 0) { rc = nl; goto out; }
  int start = 0;
  while (start < nl) {
    int nc = 0, stop = 0;
    rc = orc_partition(n, ng, g5, layer, nl, start, h->chi, q_max, l_max, k_max, cq, ck, n, &nc, &stop);
    if (rc) goto out;
    memset(inc, 0, (size_t)n);
    for (int c = 0; c < nc; c++)
      for (int t = 0; t < ck[c]; t++) inc[cq[c] + t] = 1;
    /* singletons: product of their one-qubit gates in layer order */
    for (int i = 0; i < ng; i++) {
      if (layer[i] <= start || layer[i] > stop) continue;
      const int *g = g5 + 5 * i;
      if (g[0] != 1 || inc[g[1]]) continue;
      cplx u[16];
      if (gate_matrix(g[4], params[i], u) != 2) { rc = ORC_ERR_ARG; goto out; }
      apply_1q_site(h, g[1], u);
    }
    for (int c = 0; c < nc; c++) {
      const long long D = 1LL << ck[c];
      cplx *U = malloc(sizeof(cplx) * (size_t)(D * D));
      if (!U) { rc = ORC_ERR_OOM; goto out; }
      rc = cluster_unitary(cq[c], ck[c], ng, g5, params, layer, start, stop, U);
      if (!rc) rc = cluster_update(h, cq[c], ck[c], U, chi_max, eta, floor_rel, NULL, NULL);
      free(U);
      if (rc) goto out;
    }
    h->nstep++;
    start = stop;
  }
out:
  free(layer); free(cq); free(ck); free(inc);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Observables                                                                */
/* ------------------------------------------------------------------------ */
/* <x|psi> = B_0[0,x_0,:] B_1[:,x_1,:] ... (lambda_0 = [1]) */
int orc_amplitude(const orc_mps *h, const unsigned char *bits, double *out) {
  long long c = 1;
  cplx *v = malloc(sizeof(cplx)), *w;
  if (!v) return ORC_ERR_OOM;
  v[0] = 1;
  for (int q = 0; q < h->n; q++) {
    long long cr = h->chi[q + 1];
    w = calloc((size_t)cr, sizeof(cplx));
    if (!w) { free(v); return ORC_ERR_OOM; }
    for (long long a = 0; a < c; a++)
      for (long long b = 0; b < cr; b++) w[b] += v[a] * h->site[q][(a * 2 + bits[q]) * cr + b];
    free(v);
    v = w;
    c = cr;
  }
  out[0] = creal(v[0]); out[1] = cimag(v[0]);
  free(v);
  return ORC_OK;
}

int orc_to_statevector(const orc_mps *h, double *out) {
  if (h->n > 24) return ORC_ERR_ARG;
  long long rows = 1, c = 1;
  cplx *v = malloc(sizeof(cplx));
  if (!v) return ORC_ERR_OOM;
  v[0] = 1;
  for (int q = 0; q < h->n; q++) {
    long long cr = h->chi[q + 1];
    cplx *w = calloc((size_t)(rows * 2 * cr), sizeof(cplx));
    if (!w) { free(v); return ORC_ERR_OOM; }
    for (long long i = 0; i < rows; i++)
      for (long long a = 0; a < c; a++) {
        cplx x = v[i * c + a];
        for (long long o = 0; o < 2 * cr; o++) w[i * 2 * cr + o] += x * h->site[q][a * 2 * cr + o];
      }
    free(v);
    v = w;
    rows *= 2;
    c = cr;
  }
  for (long long i = 0; i < rows; i++) { out[2 * i] = creal(v[i]); out[2 * i + 1] = cimag(v[i]); }
  free(v);
  return ORC_OK;
}

/* <a|b> by left-to-right transfer matrices; Eq. 3 is |<a|b>|^2. */
int orc_overlap(const orc_mps *a, const orc_mps *b, double *out) {
  if (a->n != b->n) return ORC_ERR_ARG;
  long long ca = 1, cb = 1;
  cplx *E = malloc(sizeof(cplx));
  if (!E) return ORC_ERR_OOM;
  E[0] = 1;
  for (int q = 0; q < a->n; q++) {
    long long ra = a->chi[q + 1], rb = b->chi[q + 1];
    cplx *F = calloc((size_t)(ra * rb), sizeof(cplx));
    cplx *G = calloc((size_t)(ca * rb), sizeof(cplx));
    if (!F || !G) { free(E); free(F); free(G); return ORC_ERR_OOM; }
    for (int s = 0; s < 2; s++) {
      memset(G, 0, sizeof(cplx) * (size_t)(ca * rb));
      for (long long i = 0; i < ca; i++)
        for (long long j = 0; j < cb; j++) {
          cplx e = E[i * cb + j];
          if (e == 0) continue;
          for (long long y = 0; y < rb; y++) G[i * rb + y] += e * b->site[q][(j * 2 + s) * rb + y];
        }
      for (long long i = 0; i < ca; i++)
        for (long long x = 0; x < ra; x++) {
          cplx av = conj(a->site[q][(i * 2 + s) * ra + x]);
          if (av == 0) continue;
          for (long long y = 0; y < rb; y++) F[x * rb + y] += av * G[i * rb + y];
        }
    }
    free(E); free(G);
    E = F;
    ca = ra; cb = rb;
  }
  out[0] = creal(E[0]); out[1] = cimag(E[0]);
  free(E);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Stabilizer tableau (Clifford circuits, Sec. IV.A; Gottesman-Knill): the X/Z */
/* bits of the n stabilizer generators under conjugation (signs are not       */
/* needed for entanglement).  S_b = rank_GF(2)(generators restricted to qubits */
/* 0..b-1) - b, so an untruncated MPS has chi_b = 2^{S_b} (Eq. 1).             */
/* ------------------------------------------------------------------------ */
int orc_stab_entropy(int n, int ng, const int *g5, int *S_out) {
  const int W = (n + 63) / 64;
  uint64_t *x = calloc((size_t)n * W, 8), *z = calloc((size_t)n * W, 8);
  if (!x || !z) { free(x); free(z); return ORC_ERR_OOM; }
#define BIT(a, r, q) ((a[(size_t)(r) * W + (q) / 64] >> ((q) % 64)) & 1ULL)
#define FLIP(a, r, q) (a[(size_t)(r) * W + (q) / 64] ^= 1ULL << ((q) % 64))
  for (int i = 0; i < n; i++) FLIP(z, i, i);
  for (int gi = 0; gi < ng; gi++) {
    const int *g = g5 + 5 * gi;
    int k = g[4], a = g[1], b = g[2];
    for (int r = 0; r < n; r++) {
      uint64_t xa = BIT(x, r, a), za = BIT(z, r, a), xb = 0, zb = 0;
      if (g[0] == 2) { xb = BIT(x, r, b); zb = BIT(z, r, b); }
      uint64_t nxa = xa, nza = za, nxb = xb, nzb = zb;
      switch (k) {
        case K_H: nxa = za; nza = xa; break;
        case K_S: nza = za ^ xa; break;
        case K_X: case K_Y: case K_Z: break;
        case K_CNOT: nxb = xb ^ xa; nza = za ^ zb; break;
        case K_CZ: nza = za ^ xb; nzb = zb ^ xa; break;
        case K_CY: /* S_t^dag, CNOT, S_t on the bits */
          zb ^= xb; nxb = xb ^ xa; nza = za ^ zb; nzb = zb ^ nxb; break;
        case K_SWAP: nxa = xb; nza = zb; nxb = xa; nzb = za; break;
        default: free(x); free(z); return ORC_ERR_ARG; /* not Clifford */
      }
      if (nxa != xa) FLIP(x, r, a);
      if (nza != za) FLIP(z, r, a);
      if (g[0] == 2) {
        if (nxb != BIT(x, r, b)) FLIP(x, r, b);
        if (nzb != BIT(z, r, b)) FLIP(z, r, b);
      }
    }
  }
  /* rank of the n x 2b matrix for each bond b */
  const int W2 = (2 * n + 63) / 64;
  uint64_t *Mb = malloc((size_t)n * W2 * 8);
  if (!Mb) { free(x); free(z); return ORC_ERR_OOM; }
  S_out[0] = 0;
  S_out[n] = 0;
  for (int bnd = 1; bnd < n; bnd++) {
    memset(Mb, 0, (size_t)n * W2 * 8);
    for (int r = 0; r < n; r++)
      for (int q = 0; q < bnd; q++) {
        if (BIT(x, r, q)) Mb[(size_t)r * W2 + q / 64] |= 1ULL << (q % 64);
        if (BIT(z, r, q)) Mb[(size_t)r * W2 + (bnd + q) / 64] |= 1ULL << ((bnd + q) % 64);
      }
    int rank = 0;
    for (int col = 0; col < 2 * bnd && rank < n; col++) {
      int piv = -1;
      for (int r = rank; r < n; r++)
        if ((Mb[(size_t)r * W2 + col / 64] >> (col % 64)) & 1ULL) { piv = r; break; }
      if (piv < 0) continue;
      if (piv != rank)
        for (int w = 0; w < W2; w++) {
          uint64_t t = Mb[(size_t)piv * W2 + w];
          Mb[(size_t)piv * W2 + w] = Mb[(size_t)rank * W2 + w];
          Mb[(size_t)rank * W2 + w] = t;
        }
      for (int r = 0; r < n; r++)
        if (r != rank && ((Mb[(size_t)r * W2 + col / 64] >> (col % 64)) & 1ULL))
          for (int w = 0; w < W2; w++) Mb[(size_t)r * W2 + w] ^= Mb[(size_t)rank * W2 + w];
      rank++;
    }
    S_out[bnd] = rank - bnd;
  }
#undef BIT
#undef FLIP
  free(Mb); free(x); free(z);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Rank-predictor network reference (not in the paper): F -> H1 -> H2 -> NB   */
/* with ReLU, mean softmax cross-entropy.  Parameters packed as               */
/* W1 (H1 x F), b1, W2 (H2 x H1), b2, W3 (NB x H2), b3, row-major.            */
/* ------------------------------------------------------------------------ */
static void mlp_fwd1(int F, int H1, int H2, int NB, const double *P, const double *x,
                     double *h1, double *h2, double *lo) {
  const double *W1 = P, *b1 = W1 + H1 * F, *W2 = b1 + H1, *b2 = W2 + H2 * H1, *W3 = b2 + H2, *b3 = W3 + NB * H2;
  for (int i = 0; i < H1; i++) {
    double a = b1[i];
    for (int j = 0; j < F; j++) a += W1[i * F + j] * x[j];
    h1[i] = a > 0 ? a : 0;
  }
  for (int i = 0; i < H2; i++) {
    double a = b2[i];
    for (int j = 0; j < H1; j++) a += W2[i * H1 + j] * h1[j];
    h2[i] = a > 0 ? a : 0;
  }
  for (int i = 0; i < NB; i++) {
    double a = b3[i];
    for (int j = 0; j < H2; j++) a += W3[i * H2 + j] * h2[j];
    lo[i] = a;
  }
}

int orc_mlp_forward(int B, int F, int H1, int H2, int NB, const double *P, const double *X, double *logits) {
  double *h1 = malloc(sizeof(double) * (size_t)H1), *h2 = malloc(sizeof(double) * (size_t)H2);
  if (!h1 || !h2) { free(h1); free(h2); return ORC_ERR_OOM; }
  for (int b = 0; b < B; b++) mlp_fwd1(F, H1, H2, NB, P, X + (size_t)b * F, h1, h2, logits + (size_t)b * NB);
  free(h1); free(h2);
  return ORC_OK;
}

int orc_mlp_loss_grad(int B, int F, int H1, int H2, int NB, const double *P, const double *X,
                      const int *y, double *loss, double *G) {
  const int np = H1 * F + H1 + H2 * H1 + H2 + NB * H2 + NB;
  const double *W2 = P + H1 * F + H1, *W3 = W2 + H2 * H1 + H2;
  double *gW1 = G, *gb1 = gW1 + H1 * F, *gW2 = gb1 + H1, *gb2 = gW2 + H2 * H1, *gW3 = gb2 + H2, *gb3 = gW3 + NB * H2;
  double *h1 = malloc(sizeof(double) * (size_t)H1), *h2 = malloc(sizeof(double) * (size_t)H2);
  double *lo = malloc(sizeof(double) * (size_t)NB), *d3 = malloc(sizeof(double) * (size_t)NB);
  double *d2 = malloc(sizeof(double) * (size_t)H2), *d1 = malloc(sizeof(double) * (size_t)H1);
  if (!h1 || !h2 || !lo || !d3 || !d2 || !d1) { free(h1); free(h2); free(lo); free(d3); free(d2); free(d1); return ORC_ERR_OOM; }
  memset(G, 0, sizeof(double) * (size_t)np);
  double L = 0;
  for (int b = 0; b < B; b++) {
    const double *x = X + (size_t)b * F;
    mlp_fwd1(F, H1, H2, NB, P, x, h1, h2, lo);
    double mx = lo[0], se = 0;
    for (int i = 1; i < NB; i++) if (lo[i] > mx) mx = lo[i];
    for (int i = 0; i < NB; i++) se += exp(lo[i] - mx);
    L += log(se) + mx - lo[y[b]];
    for (int i = 0; i < NB; i++) d3[i] = (exp(lo[i] - mx) / se - (i == y[b] ? 1.0 : 0.0)) / B;
    for (int i = 0; i < NB; i++) {
      gb3[i] += d3[i];
      for (int j = 0; j < H2; j++) gW3[i * H2 + j] += d3[i] * h2[j];
    }
    for (int j = 0; j < H2; j++) {
      double a = 0;
      for (int i = 0; i < NB; i++) a += W3[i * H2 + j] * d3[i];
      d2[j] = h2[j] > 0 ? a : 0;
    }
    for (int i = 0; i < H2; i++) {
      gb2[i] += d2[i];
      for (int j = 0; j < H1; j++) gW2[i * H1 + j] += d2[i] * h1[j];
    }
    for (int j = 0; j < H1; j++) {
      double a = 0;
      for (int i = 0; i < H2; i++) a += W2[i * H1 + j] * d2[i];
      d1[j] = h1[j] > 0 ? a : 0;
    }
    for (int i = 0; i < H1; i++) {
      gb1[i] += d1[i];
      for (int j = 0; j < F; j++) gW1[i * F + j] += d1[i] * x[j];
    }
  }
  *loss = L / B;
  free(h1); free(h2); free(lo); free(d3); free(d2); free(d1);
  return ORC_OK;
}
