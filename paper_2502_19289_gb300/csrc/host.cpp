// host.cpp -- C ABI entry points and host orchestration of the cluster update.
//
// Host-side pieces (bit-exact, deterministic): earliest-layer assignment
// (Sec. II.A), the cluster partition with the Eq. 7 / Eq. 8 stop rule
// (Sec. III.A), gate matrices (App. A) and the cluster unitaries.  The device
// pieces (merge, U, Gram, eigen-solve, truncation, write-back) are launched
// here, batched over all clusters of an iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/ctebd.h"
#include "internal.h"

using namespace ctebd;
using cd = std::complex<double>;

static thread_local std::string g_err;
static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
#define CUDA_TRY(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(CTEBD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
  } while (0)
#define TRY(call)              \
  do {                         \
    int rc_ = (call);          \
    if (rc_ != CTEBD_OK) return rc_; \
  } while (0)

void ctebd::set_last_error(const std::string& msg) { g_err = msg; }

extern "C" int ctebd_last_error(char* buf, size_t n) {
  if (!buf || n == 0) return CTEBD_ERR_ARG;
  std::snprintf(buf, n, "%s", g_err.c_str());
  return CTEBD_OK;
}

// ---------------------------------------------------------------------------
// App. A gate matrices (row-major, first listed qubit = MSB / control)
// ---------------------------------------------------------------------------
static int gate_dim(int kind, double param, cd* g) {
  const double r2 = 1.0 / std::sqrt(2.0);
  const cd i1(0, 1), w8 = std::polar(1.0, M_PI / 4);
  auto set2 = [&](cd a, cd b, cd c, cd d) { g[0] = a; g[1] = b; g[2] = c; g[3] = d; return 2; };
  switch (kind) {
    case CTEBD_H: return set2(r2, r2, r2, -r2);
    case CTEBD_X: return set2(0., 1., 1., 0.);
    case CTEBD_Y: return set2(0., -i1, i1, 0.);
    case CTEBD_Z: return set2(1., 0., 0., -1.);
    case CTEBD_S: return set2(1., 0., 0., i1);
    case CTEBD_T: return set2(1., 0., 0., w8);
    case CTEBD_P: return set2(1., 0., 0., std::polar(1.0, param));
    case CTEBD_X14: {
      const cd ph = std::polar(1.0, M_PI / 8);
      const double c = std::cos(M_PI / 8), s = std::sin(M_PI / 8);
      return set2(ph * c, -i1 * ph * s, -i1 * ph * s, ph * c);
    }
    case CTEBD_SQW: return set2(r2 * w8, -i1 * r2, r2, r2 * w8);  // principal root of (X+Y)/sqrt2
    default: break;
  }
  for (int i = 0; i < 16; i++) g[i] = 0;
  for (int i = 0; i < 4; i++) g[5 * i] = 1;
  switch (kind) {
    case CTEBD_CNOT: g[10] = 0; g[15] = 0; g[11] = 1; g[14] = 1; return 4;
    case CTEBD_CY: g[10] = 0; g[15] = 0; g[11] = -i1; g[14] = i1; return 4;
    case CTEBD_CZ: g[15] = -1; return 4;
    case CTEBD_SWAP: g[5] = 0; g[10] = 0; g[6] = 1; g[9] = 1; return 4;
    case CTEBD_CH: g[10] = r2; g[11] = r2; g[14] = r2; g[15] = -r2; return 4;
    case CTEBD_CS: g[15] = i1; return 4;
    case CTEBD_CT: g[15] = w8; return 4;
    case CTEBD_CP: g[15] = std::polar(1.0, param); return 4;
    case CTEBD_SQSWAP:
      g[5] = 0.5 * (1. + i1); g[6] = 0.5 * (1. - i1); g[9] = 0.5 * (1. - i1); g[10] = 0.5 * (1. + i1);
      return 4;
    default: return 0;
  }
}

// ---------------------------------------------------------------------------
// Sec. II.A layering, Sec. III.A partition
// ---------------------------------------------------------------------------
extern "C" int assign_layers(ctebd_gate* gates, int n_gates, int n_qubits, int* n_layers) {
  if (n_gates < 0 || n_qubits <= 0 || (n_gates > 0 && !gates)) return fail(CTEBD_ERR_ARG, "assign_layers: bad args");
  std::vector<int> last(n_qubits, 0);
  int nl = 0;
  for (int i = 0; i < n_gates; i++) {
    ctebd_gate& g = gates[i];
    if (g.n_q < 1 || g.n_q > 3) return fail(CTEBD_ERR_ARG, "assign_layers: n_q out of range");
    int L = 0;
    for (int t = 0; t < g.n_q; t++) {
      if (g.q[t] < 0 || g.q[t] >= n_qubits) return fail(CTEBD_ERR_ARG, "assign_layers: qubit out of range");
      L = std::max(L, last[g.q[t]]);
    }
    g.layer = L + 1;
    for (int t = 0; t < g.n_q; t++) last[g.q[t]] = g.layer;
    nl = std::max(nl, g.layer);
  }
  if (n_layers) *n_layers = nl;
  return CTEBD_OK;
}

// A run of entangled bonds [b1, b2] is a cluster of qubits b1-1..b2 (Eq. 6:
// 2^k chi[b1-1] chi[b2+1] with k = b2 - b1 + 2).
static bool clusters_fit(const std::vector<char>& bond, int n, const int* chi, int q_max, int k_max) {
  int b = 1;
  while (b <= n - 1) {
    if (!bond[b]) { ++b; continue; }
    const int b1 = b;
    while (b <= n - 1 && bond[b]) ++b;
    const int k = b - b1 + 1;
    if (k_max > 0 && k > k_max) return false;
    // log2(2^k chi_L chi_R) <= q_max, compared exactly in integers
    if (k > q_max) return false;
    const unsigned long long budget = q_max - k >= 63 ? ~0ULL : (1ULL << (q_max - k));
    const unsigned long long cl = (unsigned long long)chi[b1 - 1], cr = (unsigned long long)chi[b];
    if (cl > budget || cr > budget / cl) return false;
  }
  return true;
}

// True when the gates are in non-decreasing layer order (then the gates of a
// layer range are one contiguous run, found by binary search).
static bool layer_sorted(const ctebd_gate* gates, int n_gates) {
  for (int i = 1; i < n_gates; i++)
    if (gates[i].layer < gates[i - 1].layer) return false;
  return true;
}

// Indices of the gates in layers (lo, hi], in layer order and, within a
// layer, in the given order.
static void gates_in_layers(const ctebd_gate* gates, int n_gates, int lo, int hi, std::vector<int>& idx) {
  idx.clear();
  if (layer_sorted(gates, n_gates)) {
    const ctebd_gate* b = std::lower_bound(gates, gates + n_gates, lo + 1,
                                           [](const ctebd_gate& g, int L) { return g.layer < L; });
    for (const ctebd_gate* g = b; g < gates + n_gates && g->layer <= hi; ++g) idx.push_back((int)(g - gates));
    return;
  }
  for (int i = 0; i < n_gates; i++)
    if (gates[i].layer > lo && gates[i].layer <= hi) idx.push_back(i);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return gates[a].layer < gates[b].layer; });
}

extern "C" int cluster_partition(const ctebd_gate* gates, int n_gates, int layer_start, const int* chi,
                                 const ctebd_config* cfg, ctebd_cluster* out, int cap, int* n_out,
                                 int* layer_stop) {
  if (!cfg || !chi || !n_out || !layer_stop || n_gates < 0 || (n_gates && !gates))
    return fail(CTEBD_ERR_ARG, "cluster_partition: null argument");
  const int n = cfg->n_qubits;
  int n_layers = 0;
  for (int i = 0; i < n_gates; i++) n_layers = std::max(n_layers, gates[i].layer);
  // the gates after layer_start in layer order
  std::vector<int> order;
  gates_in_layers(gates, n_gates, layer_start, n_layers, order);
  std::vector<char> bond(n + 1, 0), tent;
  int stop = layer_start;
  size_t pos = 0;
  for (int L = layer_start + 1; L <= n_layers; L++) {
    if (cfg->l_max > 0 && L - layer_start > cfg->l_max) break;
    tent = bond;
    while (pos < order.size() && gates[order[pos]].layer == L) {
      const ctebd_gate& g = gates[order[pos++]];
      if (g.n_q < 2) continue;
      int lo = g.q[0], hi = g.q[0];
      for (int t = 1; t < g.n_q; t++) { lo = std::min(lo, g.q[t]); hi = std::max(hi, g.q[t]); }
      if (hi - lo != g.n_q - 1 || lo < 0 || hi >= n)
        return fail(CTEBD_ERR_ARG, "cluster_partition: multi-qubit gate on non-adjacent qubits (route it first)");
      for (int b = lo + 1; b <= hi; b++) tent[b] = 1;
    }
    if (!clusters_fit(tent, n, chi, cfg->q_max, cfg->k_max)) break;
    bond.swap(tent);
    stop = L;
  }
  if (stop == layer_start && layer_start < n_layers)
    return fail(CTEBD_ERR_STATE, "cluster_partition: no layer fits Q_max / k_max (check preconditions)");
  int nc = 0, b = 1;
  while (b <= n - 1) {
    if (!bond[b]) { ++b; continue; }
    const int b1 = b;
    while (b <= n - 1 && bond[b]) ++b;
    if (nc < cap && out) {
      out[nc].q0 = b1 - 1;
      out[nc].k = b - b1 + 1;
      out[nc].layer_lo = layer_start;
      out[nc].layer_hi = stop;
      for (int j = 0; j < 11; j++) out[nc].rank_hint[j] = 0;
    }
    ++nc;
  }
  *n_out = nc;
  *layer_stop = stop;
  if (nc > cap) return fail(CTEBD_ERR_ARG, "cluster_partition: cap too small");
  return CTEBD_OK;
}

// M <- G M for a gate on window qubits lq of a row-major 2^k x 2^k matrix:
// the gate mixes whole rows (the row index is big-endian over the window: the
// window's first qubit is the most significant bit, and bit t of a gate's
// own index belongs to its qubit lq[gnq - 1 - t]), so each update streams
// contiguous rows.  A gate whose
// matrix is a permutation (X, CNOT, SWAP) moves rows, a diagonal one scales
// them (rows with factor 1 are skipped), any other one takes the full sums.
// Complex products are written out in real arithmetic.
static void gate_on_rows(int k, cd* M, int gnq, const int* lq, const cd* g, std::vector<cd>& tmp) {
  const long long D = 1LL << k;
  const int dim = 1 << gnq;
  long long mask = 0;
  int pos[3];
  for (int t = 0; t < gnq; t++) { pos[t] = k - 1 - lq[t]; mask |= 1LL << pos[t]; }
  bool diag = true, perm = true;
  int src[8];
  for (int a = 0; a < dim; a++) {
    int ones = 0;
    src[a] = -1;
    for (int c = 0; c < dim; c++) {
      const cd v = g[a * dim + c];
      if (a != c && v != cd(0.0)) diag = false;
      if (v == cd(1.0)) { ones++; src[a] = c; }
      else if (v != cd(0.0)) perm = false;
    }
    if (ones != 1) perm = false;
  }
  if ((long long)tmp.size() < dim * D) tmp.resize(dim * D);
  double* row[8];
  for (long long base = 0; base < D; base++) {
    if (base & mask) continue;
    for (int x = 0; x < dim; x++) {
      long long i = base;
      for (int t = 0; t < gnq; t++) if ((x >> (gnq - 1 - t)) & 1) i |= 1LL << pos[t];
      row[x] = reinterpret_cast<double*>(M + i * D);
    }
    if (diag) {
      for (int a = 0; a < dim; a++) {
        const double gr = g[a * dim + a].real(), gi = g[a * dim + a].imag();
        if (gr == 1.0 && gi == 0.0) continue;
        double* r = row[a];
        for (long long j = 0; j < D; j++) {
          const double xr = r[2 * j], xi = r[2 * j + 1];
          r[2 * j] = gr * xr - gi * xi;
          r[2 * j + 1] = gr * xi + gi * xr;
        }
      }
      continue;
    }
    if (perm) {
      for (int a = 0; a < dim; a++)
        if (src[a] != a) std::memcpy(tmp.data() + a * D, row[src[a]], sizeof(cd) * D);
      for (int a = 0; a < dim; a++)
        if (src[a] != a) std::memcpy(row[a], tmp.data() + a * D, sizeof(cd) * D);
      continue;
    }
    double gr[64], gi[64];
    for (int e = 0; e < dim * dim; e++) { gr[e] = g[e].real(); gi[e] = g[e].imag(); }
    for (long long j = 0; j < D; j++) {
      double xr[8], xi[8];
      for (int c = 0; c < dim; c++) { xr[c] = row[c][2 * j]; xi[c] = row[c][2 * j + 1]; }
      for (int a = 0; a < dim; a++) {
        double sr = 0, si = 0;
        for (int c = 0; c < dim; c++) {
          sr += gr[a * dim + c] * xr[c] - gi[a * dim + c] * xi[c];
          si += gr[a * dim + c] * xi[c] + gi[a * dim + c] * xr[c];
        }
        row[a][2 * j] = sr;
        row[a][2 * j + 1] = si;
      }
    }
  }
}

extern "C" int cluster_unitary(const ctebd_gate* gates, int n_gates, const ctebd_cluster* c, double* U) {
  if (!c || !U || c->k < 1 || c->k > 12) return fail(CTEBD_ERR_ARG, "cluster_unitary: bad args");
  const int k = c->k;
  const long long D = 1LL << k;
  std::vector<cd> M(D * D, 0.0), tmp;
  for (long long i = 0; i < D; i++) M[i * D + i] = 1;
  std::vector<int> order;
  gates_in_layers(gates, n_gates, c->layer_lo, c->layer_hi, order);
  for (int gi : order) {
    const ctebd_gate& g = gates[gi];
    int lq[3], inside = 0;
    for (int t = 0; t < g.n_q; t++) {
      lq[t] = g.q[t] - c->q0;
      inside += (lq[t] >= 0 && lq[t] < k);
    }
    if (!inside) continue;
    if (inside != g.n_q) return fail(CTEBD_ERR_ARG, "cluster_unitary: gate straddles the cluster");
    cd gm[16];
    const int d = gate_dim(g.kind, g.param, gm);
    if (!d || (d == 2) != (g.n_q == 1)) return fail(CTEBD_ERR_ARG, "cluster_unitary: unknown gate kind");
    gate_on_rows(k, M.data(), g.n_q, lq, gm, tmp);
  }
  for (long long i = 0; i < D * D; i++) { U[2 * i] = M[i].real(); U[2 * i + 1] = M[i].imag(); }
  return CTEBD_OK;
}

// ---------------------------------------------------------------------------
// Device staging of small descriptor arrays (pinned host -> device, bump)
// ---------------------------------------------------------------------------
struct Staging {
  unsigned char* h = nullptr;
  unsigned char* d = nullptr;
  size_t cap = 0, off = 0;
  cudaStream_t s = nullptr;
  int init(size_t c, cudaStream_t st) {
    s = st;
    cap = c;
    CUDA_TRY(cudaMallocHost(&h, cap));
    CUDA_TRY(cudaMalloc(&d, cap));
    return CTEBD_OK;
  }
  void release() {
    if (h) cudaFreeHost(h);
    if (d) cudaFree(d);
    h = d = nullptr;
  }
  // Callers reset only after a stream synchronisation.
  void reset() { off = 0; }
  template <typename T>
  int push(const T* src, size_t count, const T** out) {
    const size_t bytes = sizeof(T) * std::max<size_t>(count, 1);
    const size_t need = (bytes + 255) & ~size_t(255);
    if (off + need > cap) {
      CUDA_TRY(cudaStreamSynchronize(s));
      off = 0;
      if (need > cap) return fail(CTEBD_ERR_OOM, "staging buffer too small");
    }
    std::memcpy(h + off, src, sizeof(T) * count);
    CUDA_TRY(cudaMemcpyAsync(d + off, h + off, sizeof(T) * count, cudaMemcpyHostToDevice, s));
    *out = reinterpret_cast<const T*>(d + off);
    off += need;
    return CTEBD_OK;
  }
};

// ---------------------------------------------------------------------------
// MPS handle
// ---------------------------------------------------------------------------
struct Work {
  int q0, k, chiL, chiR;
  void* bufA = nullptr;  // theta' / Mbar / remainder
  void* bufB = nullptr;  // merge ping-pong / Mbar*V
  size_t bufElems = 0;
  void* G = nullptr;
  void* V = nullptr;
  void* W = nullptr;     // refinement accumulator
  void* J = nullptr;
  void* T = nullptr;     // scratch of the tensor-core Jacobi round update (FP32)
  size_t eigElems = 0, jElems = 0;
  double* rho = nullptr;   // nmax weights, then nmax squared column norms of V
  int* perm = nullptr;
  double* res = nullptr; // [0..7] select results, [8] ||M||^2, [12..15] int status
  // sketched split (FP32, sketch enabled): Y and Q (m x l), B^H and Q_B (n x l),
  // FP64 Cholesky work (2 l^2 complex128) and the triangular factor X (l x l)
  void* Ys = nullptr;
  void* Qs = nullptr;
  void* Bs = nullptr;
  void* QB = nullptr;
  void* CW = nullptr;
  void* X = nullptr;
  size_t nmax = 0;
  int rdim = 0;          // current right dimension during splitting
  int hint[12] = {0};    // rank hints per internal bond (<= 0: none)
  bool owned = false;    // buffers allocated individually (apply_cluster path)
};

// ---------------------------------------------------------------------------
// Per-kernel-class CUDA-event timing on the library's stream (off by
// default) and launch counting (always on).  Flops and bytes are the
// algorithmic amounts of each launch (complex MAC = 8 real flops).
// ---------------------------------------------------------------------------
enum KernelKind {
  KK_GEMM_MERGE, KK_GEMM_U, KK_GEMM_GRAM, KK_GEMM_PROJ, KK_EIG_INIT, KK_EIG_INNER, KK_EIG_APPLY,
  KK_COLNORM, KK_SELECT, KK_GATHER, KK_ONEQ, KK_AMP, KK_GEMM_SKETCH, KK_CHOL, KK_MLP, KK_COUNT
};
static const char* kKindNames[KK_COUNT] = {
  "gemm_merge", "gemm_apply_u", "gemm_gram", "gemm_project", "eig_init", "eig_inner", "eig_apply",
  "colnorm", "select", "gather", "apply_1q", "amplitude", "gemm_sketch", "cholqr", "mlp_forward"};

struct Prof {
  bool on = false;
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  double launches[KK_COUNT] = {0}, ms[KK_COUNT] = {0}, flops[KK_COUNT] = {0}, bytes[KK_COUNT] = {0};
  double tc[KK_COUNT] = {0};   // launches of the class that ran on the tensor cores
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void reset() {
    for (int i = 0; i < KK_COUNT; i++) launches[i] = ms[i] = flops[i] = bytes[i] = tc[i] = 0;
  }
  // fold finished records into the accumulators (caller synchronised)
  void drain() {
    for (auto& r : recs) {
      float t = 0;
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.kind] += t;
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
  }
  void release() {
    drain();
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
  }
};

struct ProfScope {
  Prof& p;
  cudaStream_t s;
  int kind;
  cudaEvent_t b = nullptr;
  ProfScope(Prof& pr, cudaStream_t st, int k, double fl, double by) : p(pr), s(st), kind(k) {
    p.launches[k] += 1;
    p.flops[k] += fl;
    p.bytes[k] += by;
    if (p.on) {
      cudaEvent_t a = p.get();
      b = p.get();
      cudaEventRecord(a, s);
      p.recs.push_back({k, a, b});
    }
  }
  ~ProfScope() {
    if (b) cudaEventRecord(b, s);
  }
};

struct ctebd_mps {
  ctebd_config cfg{};
  int n = 0;
  bool fp64 = true;
  size_t esz = 16;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<int> chi;
  std::vector<void*> site;
  std::vector<size_t> site_cap;
  std::vector<double*> lam;
  int lam_cap = 0;
  double logF = 0;
  std::vector<double> splitlog;
  std::vector<double> splitlog2;   // per split: sketched, eigen-dim, rank before cap, hint,
                                   // Jacobi sweeps of pass 1 and pass 2
  double sk_stats[2] = {0, 0};     // sketched splits attempted, fallen back
  double solve_stats[2] = {0, 0};  // refinement passes accepted at the sweep cap, their
                                   // largest last-sweep moved weight (relative to the trace)
  uint64_t nstep = 0;
  float* mlp = nullptr;            // rank predictor parameters (device)
  int* tc_err = nullptr;           // tensor-core completion-wait timeout flag (device)
  double* eig_scr = nullptr;       // eigen-solve counters and pair flags (high-water)
  size_t eig_scr_cap = 0;          // in doubles
  unsigned char* pack_scr = nullptr;   // packed tensor-core GEMM operands (high-water)
  size_t pack_cap = 0;                 // in bytes
  cudaStream_t side = nullptr;     // second branch of the device-side sweep graphs
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  void* arena = nullptr;
  size_t arena_cap = 0;
  Staging stage;
  double* h_res = nullptr;       // pinned results of select (8 per problem)
  size_t h_res_cap = 0;
  std::map<int, Work> pending;
  Prof prof;
};

static int ensure_site(ctebd_mps* m, int q, size_t elems) {
  if (m->site_cap[q] >= elems) return CTEBD_OK;
  if (m->site[q]) CUDA_TRY(cudaFreeAsync(m->site[q], m->stream));
  m->site[q] = nullptr;
  CUDA_TRY(cudaMallocAsync(&m->site[q], std::max<size_t>(elems, 1) * m->esz, m->stream));
  m->site_cap[q] = elems;
  return CTEBD_OK;
}

extern "C" int mps_create(const ctebd_config* cfg, void* cuda_stream, ctebd_mps** out) {
  if (!cfg || !out) return fail(CTEBD_ERR_ARG, "mps_create: null argument");
  if (cfg->n_qubits < 1 || cfg->chi_max < 1 || cfg->chi_max > 2048)
    return fail(CTEBD_ERR_ARG, "mps_create: n_qubits >= 1 and 1 <= chi_max <= 2048 required");
  if (cfg->precision != CTEBD_FP64 && cfg->precision != CTEBD_FP32)
    return fail(CTEBD_ERR_ARG, "mps_create: precision must be CTEBD_FP64 or CTEBD_FP32");
  if (cfg->k_max == 1) return fail(CTEBD_ERR_ARG, "mps_create: k_max must be >= 2 (or <= 0)");
  int lg = 0;
  while ((1 << lg) < cfg->chi_max) lg++;
  if (cfg->q_max < 2 + 2 * lg)
    return fail(CTEBD_ERR_ARG, "mps_create: q_max >= 2 + 2 log2(chi_max) required (Eq. 7 must admit one layer)");
  if (!(cfg->cutoff >= 0.0) || cfg->cutoff >= 1.0) return fail(CTEBD_ERR_ARG, "mps_create: 0 <= cutoff < 1");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
    return fail(CTEBD_ERR_CUDA, "mps_create: no CUDA device");
  ctebd_mps* m = new ctebd_mps();
  m->cfg = *cfg;
  m->n = cfg->n_qubits;
  m->fp64 = cfg->precision == CTEBD_FP64;
  m->esz = m->fp64 ? 16 : 8;
  if (cuda_stream) {
    m->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete m;
      return fail(CTEBD_ERR_CUDA, "mps_create: stream");
    }
    m->own_stream = true;
  }
  m->chi.assign(m->n + 1, 1);
  m->site.assign(m->n, nullptr);
  m->site_cap.assign(m->n, 0);
  m->lam_cap = cfg->chi_max;
  m->lam.assign(m->n + 1, nullptr);
  int rc = m->stage.init(8 << 20, m->stream);
  if (rc) { mps_destroy(m); return rc; }
  if (cudaMallocHost(&m->h_res, 16 * sizeof(double) * 4096) != cudaSuccess) { mps_destroy(m); return fail(CTEBD_ERR_OOM, "pinned"); }
  m->h_res_cap = 4096;
  std::vector<double> one(1, 1.0);
  for (int b = 0; b <= m->n; b++) {
    if (cudaMalloc(&m->lam[b], sizeof(double) * m->lam_cap) != cudaSuccess) { mps_destroy(m); return fail(CTEBD_ERR_OOM, "lambda"); }
    cudaMemcpyAsync(m->lam[b], one.data(), sizeof(double), cudaMemcpyHostToDevice, m->stream);
  }
  // |0> on every site: (1, 2, 1) tensor [1, 0]
  std::vector<double> zero_state(4, 0.0);
  zero_state[0] = 1.0;
  for (int q = 0; q < m->n; q++) {
    if (ensure_site(m, q, 2) != CTEBD_OK) { mps_destroy(m); return CTEBD_ERR_OOM; }
    if (m->fp64) {
      cudaMemcpyAsync(m->site[q], zero_state.data(), 32, cudaMemcpyHostToDevice, m->stream);
    } else {
      float z[4] = {1.f, 0.f, 0.f, 0.f};
      cudaMemcpyAsync(m->site[q], z, 16, cudaMemcpyHostToDevice, m->stream);
    }
  }
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) { mps_destroy(m); return fail(CTEBD_ERR_CUDA, "mps_create: init"); }
  *out = m;
  return CTEBD_OK;
}

static std::vector<std::pair<void**, size_t>> work_buffers(const ctebd_mps* m, Work& w);

extern "C" int mps_destroy(ctebd_mps* m) {
  if (!m) return CTEBD_ERR_ARG;
  if (m->stream) cudaStreamSynchronize(m->stream);
  for (auto& kv : m->pending) {
    Work& w = kv.second;
    if (w.owned)
      for (auto& pb : work_buffers(m, w)) if (*pb.first) cudaFree(*pb.first);
  }
  for (void* p : m->site) if (p) cudaFree(p);
  for (double* p : m->lam) if (p) cudaFree(p);
  if (m->arena) cudaFree(m->arena);
  if (m->mlp) cudaFree(m->mlp);
  if (m->tc_err) cudaFree(m->tc_err);
  if (m->eig_scr) cudaFree(m->eig_scr);
  if (m->pack_scr) cudaFree(m->pack_scr);
  if (m->h_res) cudaFreeHost(m->h_res);
  m->stage.release();
  m->prof.release();
  if (m->side) cudaStreamDestroy(m->side);
  if (m->fork_ev) cudaEventDestroy(m->fork_ev);
  if (m->join_ev) cudaEventDestroy(m->join_ev);
  if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
  delete m;
  return CTEBD_OK;
}

// ---------------------------------------------------------------------------
// Batched pieces
// ---------------------------------------------------------------------------
// tensor-core GEMM policy: 0 never, 1 for FP32 calls above a work threshold,
// 2 for every FP32 call (process-wide; ctebd_set_tensor_cores)
static int g_tc_mode = 1;

extern "C" int ctebd_set_tensor_cores(int mode) {
  if (mode < 0 || mode > 2) return fail(CTEBD_ERR_ARG, "ctebd_set_tensor_cores: mode 0, 1 or 2");
  g_tc_mode = mode;
  return CTEBD_OK;
}

// grow the eigen-solve scratch to at least n doubles (synchronises only when it grows)
static int ensure_eig_scratch(ctebd_mps* m, size_t n) {
  if (n <= m->eig_scr_cap) return CTEBD_OK;
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  if (m->eig_scr) CUDA_TRY(cudaFree(m->eig_scr));
  m->eig_scr = nullptr;
  m->eig_scr_cap = 0;
  const size_t want = n + n / 2 + 1024;
  if (cudaMalloc(&m->eig_scr, sizeof(double) * want) != cudaSuccess) {
    cudaGetLastError();
    return fail(CTEBD_ERR_OOM, "eigen-solve scratch");
  }
  m->eig_scr_cap = want;
  return CTEBD_OK;
}

// grow the packed-operand scratch to at least n bytes (synchronises only when it grows)
static int ensure_pack_scratch(ctebd_mps* m, size_t n) {
  if (n <= m->pack_cap) return CTEBD_OK;
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  if (m->pack_scr) CUDA_TRY(cudaFree(m->pack_scr));
  m->pack_scr = nullptr;
  m->pack_cap = 0;
  const size_t want = n + n / 4;
  if (cudaMalloc(&m->pack_scr, want) != cudaSuccess) {
    cudaGetLastError();
    return fail(CTEBD_ERR_OOM, "packed GEMM operands of " + std::to_string(want >> 20) + " MiB");
  }
  m->pack_cap = want;
  return CTEBD_OK;
}

// the device flag that a tensor-core kernel sets when a bounded wait expires
static int ensure_tc_err(ctebd_mps* m) {
  if (m->tc_err) return CTEBD_OK;
  CUDA_TRY(cudaMalloc(&m->tc_err, sizeof(int)));
  CUDA_TRY(cudaMemsetAsync(m->tc_err, 0, sizeof(int), m->stream));
  return CTEBD_OK;
}

static size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static double gemm_flops(const GemmProb& g) { return 8.0 * g.M * g.N * (double)g.K * g.batch; }

static double gemm_bytes(const GemmProb& g, size_t esz) {
  return ((double)g.M * g.K * (g.sA ? g.batch : 1) + (double)g.K * g.N * (g.sB ? g.batch : 1) +
          (double)g.M * g.N * g.batch) * esz;
}

// one grouped launch of probs on the tensor cores (tc) or the SIMT kernel
static int launch_gemm_group(ctebd_mps* m, const std::vector<GemmProb>& probs, int kind, bool tc) {
  if (probs.empty()) return CTEBD_OK;
  double fl = 0, by = 0;
  for (const GemmProb& g : probs) {
    fl += gemm_flops(g);
    by += gemm_bytes(g, m->esz);
  }
  if (tc) {
    // tensor cores: the operands of a run of problems are packed into the
    // scratch (at most kPackGroup bytes per run, or one problem), then
    // multiplied; consecutive runs reuse the scratch in stream order
    constexpr size_t kPackGroup = (size_t)8 << 30;
    TRY(ensure_tc_err(m));
    ProfScope ps(m->prof, m->stream, kind, fl, by);
    for (size_t i0 = 0; i0 < probs.size();) {
      size_t bytes = 0, i1 = i0;
      while (i1 < probs.size()) {
        const size_t b = round_up(tc_packed_bytes(probs[i1]), 256);
        if (i1 > i0 && bytes + b > kPackGroup) break;
        bytes += b;
        i1++;
      }
      TRY(ensure_pack_scratch(m, bytes));
      const int np = (int)(i1 - i0);
      std::vector<PackedProb> pp(np);
      std::vector<long long> poff(np + 1, 0), toff(np + 1, 0);
      unsigned char* p = m->pack_scr;
      for (int i = 0; i < np; i++) {
        PackedProb& q = pp[i];
        q.g = probs[i0 + i];
        tc_packed_shape(q.g, q.tilesM, q.tilesN, q.chunks);
        q.pa = reinterpret_cast<float*>(p);
        q.pb = reinterpret_cast<float*>(p + tc_packed_a_bytes(q.g));
        p += round_up(tc_packed_bytes(q.g), 256);
        poff[i + 1] = poff[i] + tc_packed_pack_blocks(q.g);
        toff[i + 1] = toff[i] + tc_packed_tiles(q.g);
      }
      const PackedProb* dpp;
      const long long *dpo, *dto;
      TRY(m->stage.push(pp.data(), pp.size(), &dpp));
      TRY(m->stage.push(poff.data(), poff.size(), &dpo));
      TRY(m->stage.push(toff.data(), toff.size(), &dto));
      m->prof.tc[kind] += 1;
      CUDA_TRY(launch_tc_packed(dpp, dpo, dto, np, poff.back(), toff.back(), m->tc_err, m->stream));
      i0 = i1;
    }
    return CTEBD_OK;
  }
  std::vector<long long> off(probs.size() + 1, 0);
  for (size_t i = 0; i < probs.size(); i++) off[i + 1] = off[i] + gemm_tiles(probs[i], m->fp64);
  const GemmProb* dp;
  const long long* doff;
  TRY(m->stage.push(probs.data(), probs.size(), &dp));
  TRY(m->stage.push(off.data(), off.size(), &doff));
  ProfScope ps(m->prof, m->stream, kind, fl, by);
  cudaError_t e = m->fp64 ? launch_gemm<double>(dp, doff, (int)probs.size(), off.back(), m->stream)
                          : launch_gemm<float>(dp, doff, (int)probs.size(), off.back(), m->stream);
  CUDA_TRY(e);
  return CTEBD_OK;
}

// Size policy (mode 1): a group of at least 2 GFLOP goes to the tensor cores,
// except its problems with fewer than 64 rows -- the tensor-core tile is 128
// rows -- which run on the SIMT kernel in a second launch.
static int run_gemms(ctebd_mps* m, const std::vector<GemmProb>& probs, int kind) {
  if (probs.empty()) return CTEBD_OK;
  if (m->fp64 || g_tc_mode == 0) return launch_gemm_group(m, probs, kind, false);
  if (g_tc_mode == 2) return launch_gemm_group(m, probs, kind, true);
  double fl = 0;
  for (const GemmProb& g : probs) fl += gemm_flops(g);
  if (fl < 2e9) return launch_gemm_group(m, probs, kind, false);
  std::vector<GemmProb> tc, simt;
  for (const GemmProb& g : probs) (g.M >= 64 ? tc : simt).push_back(g);
  TRY(launch_gemm_group(m, tc, kind, true));
  return launch_gemm_group(m, simt, kind, false);
}

// sizes of one cluster's work buffers
static void work_sizes(const ctebd_mps* m, Work& w) {
  const int k = w.k, q0 = w.q0;
  size_t big = (size_t)w.chiL * ((size_t)1 << k) * w.chiR;
  size_t rows = (size_t)w.chiL * 2;
  for (int j = 1; j < k; j++) {  // merge intermediates
    big = std::max(big, rows * (size_t)m->chi[q0 + j]);
    rows *= 2;
  }
  // split level shapes: the Gram of the split at bond q0 + j is n x n with
  // n = 2 r, r the rank kept at bond q0 + j + 1 (chi_R for the first split,
  // j = k - 1), and r <= min(chi_max, chi_L 2^(j+1), chi_R 2^(k-j-1)) (the
  // ranks of the matrices split there)
  size_t nmax = 2 * (size_t)w.chiR;
  for (int j = 1; j < k - 1; j++)
    nmax = std::max(nmax, 2 * std::min({(size_t)m->cfg.chi_max, (size_t)w.chiL << (j + 1),
                                        (size_t)w.chiR << (k - j - 1)}));
  const int JB = eig_block(m->fp64);
  const size_t npad = round_up(nmax, 2 * JB);
  w.bufElems = big;
  w.nmax = nmax;
  w.eigElems = npad * npad;
  w.jElems = std::max(npad * 2 * JB, ((size_t)1 << k) * ((size_t)1 << k));
}

// every device buffer of a work item: (pointer slot, bytes)
static std::vector<std::pair<void**, size_t>> work_buffers(const ctebd_mps* m, Work& w) {
  std::vector<std::pair<void**, size_t>> b = {
      {&w.bufA, w.bufElems * m->esz}, {&w.bufB, w.bufElems * m->esz}, {&w.G, w.eigElems * m->esz},
      {&w.V, w.eigElems * m->esz},    {&w.W, w.eigElems * m->esz},    {&w.J, w.jElems * m->esz},
      {(void**)&w.rho, w.nmax * 16},   {(void**)&w.perm, w.nmax * 4},  {(void**)&w.res, 256}};
  if (!m->fp64) b.push_back({&w.T, w.eigElems * m->esz});
  if (!m->fp64 && m->cfg.sketch_oversample > 0) {
    b.push_back({&w.Ys, w.bufElems / 2 * m->esz});
    b.push_back({&w.Qs, w.bufElems / 2 * m->esz});
    b.push_back({&w.Bs, w.eigElems / 2 * m->esz});
    b.push_back({&w.QB, w.eigElems / 2 * m->esz});
    b.push_back({&w.CW, w.eigElems * 16});
    b.push_back({&w.X, w.eigElems / 4 * m->esz});
  }
  return b;
}

static int carve_work(ctebd_mps* m, std::vector<Work>& ws) {
  size_t total = 0;
  auto al = [](size_t b) { return round_up(std::max<size_t>(b, 16), 256); };
  for (auto& w : ws) {
    work_sizes(m, w);
    for (auto& pb : work_buffers(m, w)) total += al(pb.second);
  }
  if (total > m->arena_cap) {
    CUDA_TRY(cudaStreamSynchronize(m->stream));
    if (m->arena) CUDA_TRY(cudaFree(m->arena));
    m->arena = nullptr;
    m->arena_cap = 0;
    const size_t want = total + total / 4;
    if (cudaMalloc(&m->arena, want) != cudaSuccess) {
      cudaGetLastError();
      return fail(CTEBD_ERR_OOM, "workspace arena of " + std::to_string(want >> 20) + " MiB");
    }
    m->arena_cap = want;
  }
  unsigned char* p = (unsigned char*)m->arena;
  for (auto& w : ws)
    for (auto& pb : work_buffers(m, w)) {
      *pb.first = p;
      p += al(pb.second);
    }
  return CTEBD_OK;
}

static int alloc_owned(ctebd_mps* m, Work& w) {
  work_sizes(m, w);
  for (auto& pb : work_buffers(m, w))
    if (cudaMallocAsync(pb.first, std::max<size_t>(pb.second, 16), m->stream) != cudaSuccess)
      return fail(CTEBD_ERR_OOM, "work buffer");
  w.owned = true;
  return CTEBD_OK;
}

static void free_owned(ctebd_mps* m, Work& w) {
  if (!w.owned) return;
  for (auto& pb : work_buffers(m, w))
    if (*pb.first) cudaFreeAsync(*pb.first, m->stream);
  w.owned = false;
}

// merge k sites and apply U: theta' ends in bufA (Sec. III.A exact contraction)
static int merge_apply(ctebd_mps* m, std::vector<Work>& ws, const std::vector<const double*>& Us) {
  const int kmax = [&] { int x = 0; for (auto& w : ws) x = std::max(x, w.k); return x; }();
  std::vector<void*> cur(ws.size()), other(ws.size());
  for (size_t i = 0; i < ws.size(); i++) { cur[i] = nullptr; }
  // level j: T_{j} = T_{j-1} * B_{q0+j}; T_0 = site q0
  for (int j = 1; j < kmax; j++) {
    std::vector<GemmProb> probs;
    for (size_t i = 0; i < ws.size(); i++) {
      Work& w = ws[i];
      if (j >= w.k) continue;
      const int rows = w.chiL << j;  // rows of T_{j-1} viewed (chiL 2^j) x chi[q0+j]
      const int kdim = m->chi[w.q0 + j];
      const int ncol = 2 * m->chi[w.q0 + j + 1];
      void* dst = (cur[i] == w.bufA) ? w.bufB : w.bufA;
      GemmProb p{};
      p.M = rows; p.N = ncol; p.K = kdim; p.batch = 1;
      p.A = cur[i] ? cur[i] : m->site[w.q0]; p.lda = kdim; p.opA = 0;
      p.B = m->site[w.q0 + j]; p.ldb = ncol; p.opB = 0;
      p.C = dst; p.ldc = ncol; p.alpha = 1.0;
      probs.push_back(p);
      cur[i] = dst;
    }
    TRY(run_gemms(m, probs, KK_GEMM_MERGE));
  }
  // U (host c128) -> device run precision, then theta' = U theta per left index
  std::vector<GemmProb> probs;
  std::vector<ApplyUProb> small;
  long long max_cols = 0;
  double u_flops = 0, u_bytes = 0;
  for (size_t i = 0; i < ws.size(); i++) {
    Work& w = ws[i];
    const long long D = 1LL << w.k;
    const double* dU;
    TRY(m->stage.push(Us[i], (size_t)(2 * D * D), &dU));
    void* src = cur[i] ? cur[i] : m->site[w.q0];
    // convert U into the spare half of the non-source buffer's tail: use J scratch
    void* Ud = w.J;
    if ((size_t)(D * D) > w.jElems) return fail(CTEBD_ERR_ARG, "cluster too large for U scratch");
    cudaError_t e = m->fp64 ? launch_convert_from_c128<double>(dU, Ud, D * D, m->stream)
                            : launch_convert_from_c128<float>(dU, Ud, D * D, m->stream);
    CUDA_TRY(e);
    void* dst = (src == w.bufA) ? w.bufB : w.bufA;
    if (D <= 16) {   // small clusters: streaming transform of the (a, b) columns
      ApplyUProb u{};
      u.U = Ud; u.src = src; u.dst = dst; u.chiL = w.chiL; u.chiR = w.chiR; u.D = (int)D;
      small.push_back(u);
      max_cols = std::max(max_cols, (long long)w.chiL * w.chiR);
      u_flops += 8.0 * D * D * w.chiL * (double)w.chiR;
      u_bytes += 2.0 * D * w.chiL * (double)w.chiR * m->esz;
      if (dst != w.bufA) std::swap(w.bufA, w.bufB);
      continue;
    }
    GemmProb p{};
    p.M = (int)D; p.N = w.chiR; p.K = (int)D; p.batch = w.chiL;
    p.A = Ud; p.lda = (int)D; p.opA = 0; p.sA = 0;
    p.B = src; p.ldb = w.chiR; p.opB = 0; p.sB = D * w.chiR;
    p.C = dst; p.ldc = w.chiR; p.sC = D * w.chiR; p.alpha = 1.0;
    probs.push_back(p);
    if (dst != w.bufA) {
      // keep theta' in bufA: swap the roles of the two buffers for this work item
      std::swap(w.bufA, w.bufB);
    }
  }
  if (!small.empty()) {
    const ApplyUProb* dsu;
    TRY(m->stage.push(small.data(), small.size(), &dsu));
    ProfScope ps(m->prof, m->stream, KK_GEMM_U, u_flops, u_bytes);
    CUDA_TRY(m->fp64 ? launch_apply_u<double>(dsu, (int)small.size(), max_cols, m->stream)
                     : launch_apply_u<float>(dsu, (int)small.size(), max_cols, m->stream));
  }
  TRY(run_gemms(m, probs, KK_GEMM_U));
  for (auto& w : ws) w.rdim = w.chiR;
  return CTEBD_OK;
}

// ---------------------------------------------------------------------------
// Split pieces (one level = one bond per active cluster).  A problem's
// eigen-dimension ne is its column count n (full split) or the sketch size l
// (sketched split: Rayleigh-Ritz on the range of M^H Q).
// ---------------------------------------------------------------------------
struct Level {
  std::vector<int> act;                        // indices into ws
  std::vector<int> mm, nn, npad, shift;        // M-bar rows / cols, padded cols, lambda shift
  std::vector<int> ne, nepad, nbv, vld;        // eigen-dimension, padded, blocks, ld of V
  std::vector<char> sk;                        // sketched
  std::vector<int> sw1, sw2;                   // Jacobi sweeps of pass 1 / pass 2
};

static void level_set_full(Level& L, int a, int JB) {
  L.sk[a] = 0;
  L.ne[a] = L.nn[a];
  L.nepad[a] = L.npad[a];
  L.nbv[a] = L.npad[a] / JB;
  L.vld[a] = L.npad[a];
}

// G = Z^H diag(lambda_L^2) Z over the m rows of Z (ne columns, row-major)
static int level_gram(ctebd_mps* m, std::vector<Work>& ws, const Level& L, const std::vector<int>& sel,
                      const std::vector<const void*>& Z) {
  std::vector<GemmProb> probs;
  for (size_t i = 0; i < sel.size(); i++) {
    const int a = sel[i];
    Work& w = ws[L.act[a]];
    CUDA_TRY(cudaMemsetAsync(w.G, 0, (size_t)L.nepad[a] * L.nepad[a] * m->esz, m->stream));
    GemmProb p{};
    p.M = L.ne[a]; p.N = L.ne[a]; p.K = L.mm[a]; p.batch = 1;
    p.A = Z[i]; p.lda = L.ne[a]; p.opA = 1;
    p.B = Z[i]; p.ldb = L.ne[a]; p.opB = 0;
    p.C = w.G; p.ldc = L.nepad[a];
    p.kw = m->lam[w.q0];
    p.kw_shift = L.shift[a];
    p.alpha = 1.0;
    probs.push_back(p);
  }
  return run_gemms(m, probs, KK_GEMM_GRAM);
}

// Batched block-Jacobi on every G of the selection; rotations accumulate
// into acc[i] (set to identity first).  floor_factor scales the absolute
// rotation floor eps * trace(G): 1 for a Gram computed from Mbar (absolute
// rounding), ~0 for a Gram of already rotated columns (relative accuracy).
// ---------------------------------------------------------------------------
// Device-side sweep loop: one CUDA graph with a WHILE conditional node whose
// body is the rounds of one sweep (inner + apply per round) followed by the
// sweep-end kernel, which folds the counters, retires converged problems and
// sets the loop condition.  One launch and one host read per eigen-solve
// instead of a host round trip per sweep.  Used when per-launch profiling is
// off, by default for batches at least kGraphMinBlocks blocks wide
// (ctebd_set_sweep_graphs; process-wide): a narrower batch converges in a few
// short sweeps, and building and instantiating its graph costs more than the
// host round trips it saves.
// ---------------------------------------------------------------------------
static int g_sweep_graphs = 1;   // 0 never, 1 wide batches, 2 always
constexpr int kGraphMinBlocks = 16;
static int g_max_sweeps = 60;

namespace ctebd {
int max_jacobi_sweeps() { return g_max_sweeps; }
}  // namespace ctebd

extern "C" int ctebd_set_max_sweeps(int n) {
  if (n < 1 || n > 1000) return fail(CTEBD_ERR_ARG, "ctebd_set_max_sweeps: 1..1000");
  g_max_sweeps = n;
  return CTEBD_OK;
}

extern "C" int ctebd_max_sweeps(void) { return g_max_sweeps; }

extern "C" int ctebd_set_sweep_graphs(int mode) {
  if (mode < 0 || mode > 2) return fail(CTEBD_ERR_ARG, "ctebd_set_sweep_graphs: 0, 1 or 2");
  g_sweep_graphs = mode;
  return CTEBD_OK;
}

// The problems are split into two halves captured on two streams: the graph
// body holds two independent chains of round launches (joined before the
// sweep-end kernel), so one half's latency-bound inner kernels can run while
// the other half's apply kernels do.
// Batches of more than kSweepCompact problems at least kCompactMinBlocks
// blocks wide get a second chain of round launches over a compact copy of the
// problems still active (grid y = kSweepCompact): the last sweeps of such a
// batch typically rotate one or two problems, and the full grids'
// early-exiting CTAs then cost more than the work.  Narrower batches keep the
// single chain: there the extra graph bodies cost more to build than the tail.
constexpr int kSweepCompact = 8, kCompactMinBlocks = 32;

static int run_sweep_graph(ctebd_mps* m, EigProb* dep, int na, const std::vector<int>& nbs, double* d_cum,
                           int max_sweeps, bool tc_apply, EigProb* d_compact, int* d_mode) {
  const bool f64 = m->fp64;
  if (!m->side) {
    CUDA_TRY(cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&m->fork_ev, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&m->join_ev, cudaEventDisableTiming));
  }
  const int na0 = na > 1 ? (na + 1) / 2 : na, na1 = na - na0;
  int nb0 = 2, nb1 = 2;
  for (int i = 0; i < na; i++) (i < na0 ? nb0 : nb1) = std::max(i < na0 ? nb0 : nb1, nbs[i]);
  const int max_nb = std::max(nb0, nb1);
  const int JB = eig_block(f64);
  const bool compact = na > kSweepCompact && max_nb >= kCompactMinBlocks && d_compact && d_mode;
  auto chain = [&](EigProb* d, int n, int mnb, cudaStream_t s) -> cudaError_t {
    cudaError_t le = cudaSuccess;
    for (int t = 0; t < mnb - 1 && le == cudaSuccess; t++) {
      le = f64 ? launch_eig_inner<double>(d, n, mnb, t, s) : launch_eig_inner<float>(d, n, mnb, t, s);
      if (le != cudaSuccess) break;
      if (tc_apply) le = launch_eig_apply_tc(d, n, mnb, mnb * JB, t, m->tc_err, s);
      else le = f64 ? launch_eig_apply<double>(d, n, mnb, t, s) : launch_eig_apply<float>(d, n, mnb, t, s);
    }
    return le;
  };
  // both halves of the batch, the second on the side stream (fork / join)
  auto full_chains = [&]() -> cudaError_t {
    cudaError_t le = cudaSuccess;
    if (na1 > 0) {
      le = cudaEventRecord(m->fork_ev, m->stream);
      if (le == cudaSuccess) le = cudaStreamWaitEvent(m->side, m->fork_ev, 0);
      if (le == cudaSuccess) le = chain(dep + na0, na1, nb1, m->side);
      if (le == cudaSuccess) le = cudaEventRecord(m->join_ev, m->side);
    }
    if (le == cudaSuccess) le = chain(dep, na0, nb0, m->stream);
    if (le == cudaSuccess && na1 > 0) le = cudaStreamWaitEvent(m->stream, m->join_ev, 0);
    return le;
  };
  // capture fn's launches on the handle's stream into graph gr after deps
  auto capture = [&](cudaGraph_t gr, const cudaGraphNode_t* deps, size_t nd, auto fn) -> cudaError_t {
    cudaError_t ce = cudaStreamBeginCaptureToGraph(m->stream, gr, deps, nullptr, nd, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return ce;
    const cudaError_t le = fn();
    cudaGraph_t out = nullptr;
    ce = cudaStreamEndCapture(m->stream, &out);
    return le != cudaSuccess ? le : ce;
  };
  auto add_if = [&](cudaGraph_t parent, const cudaGraphNode_t* dep_node, cudaGraphConditionalHandle hh,
                    cudaGraphNode_t* out_node, cudaGraph_t* out_body) -> cudaError_t {
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hh;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    const cudaError_t ce = cudaGraphAddNode(out_node, parent, dep_node, nullptr, dep_node ? 1 : 0, &ip);
    if (ce == cudaSuccess) *out_body = ip.conditional.phGraph_out[0];
    return ce;
  };
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  cudaGraphConditionalHandle h{};
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
  }
  if (e == cudaSuccess && !compact) {
    e = capture(cp.conditional.phGraph_out[0], nullptr, 0, [&]() -> cudaError_t {
      cudaError_t le = full_chains();
      if (le == cudaSuccess)
        le = launch_sweep_end(dep, na, d_cum, d_cum + 4 * na, max_sweeps, h, nullptr, 0, nullptr, m->stream);
      return le;
    });
  } else if (e == cudaSuccess) {
    // body: sweep_begin -> IF compact { one chain } -> IF full { both halves } -> sweep_end
    cudaGraph_t body = cp.conditional.phGraph_out[0], bc = nullptr, bf = nullptr;
    cudaGraphConditionalHandle hc{}, hf{};
    cudaGraphNode_t n_begin = nullptr, n_c = nullptr, n_f = nullptr;
    e = cudaGraphConditionalHandleCreate(&hc, body, 0, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hf, body, 0, 0);
    if (e == cudaSuccess) e = capture(body, nullptr, 0, [&]() { return launch_sweep_begin(d_mode, hc, hf, m->stream); });
    if (e == cudaSuccess) {
      size_t nn = 1;
      e = cudaGraphGetNodes(body, &n_begin, &nn);
      if (e == cudaSuccess && nn != 1) e = cudaErrorUnknown;
    }
    if (e == cudaSuccess) e = add_if(body, &n_begin, hc, &n_c, &bc);
    if (e == cudaSuccess) e = capture(bc, nullptr, 0, [&]() { return chain(d_compact, kSweepCompact, max_nb, m->stream); });
    if (e == cudaSuccess) e = add_if(body, &n_c, hf, &n_f, &bf);
    if (e == cudaSuccess) e = capture(bf, nullptr, 0, full_chains);
    if (e == cudaSuccess)
      e = capture(body, &n_f, 1, [&]() {
        return launch_sweep_end(dep, na, d_cum, d_cum + 4 * na, max_sweeps, h, d_compact, kSweepCompact, d_mode,
                                m->stream);
      });
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(ex, m->stream);
  if (ex) cudaGraphExecDestroy(ex);   // freed once the launch completes
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(CTEBD_ERR_CUDA, std::string("sweep graph: ") + cudaGetErrorString(e));
  }
  return CTEBD_OK;
}

static int level_eig(ctebd_mps* m, std::vector<Work>& ws, const Level& L, const std::vector<int>& sel,
                     const std::vector<void*>& acc, double floor_factor, double rel_skip,
                     std::vector<int>& sweeps, bool use_cut = false) {
  const bool f64 = m->fp64;
  const int JB = eig_block(f64);
  const int na = (int)sel.size();
  if (na == 0) return CTEBD_OK;
  std::vector<EigProb> eps(na);
  int max_npad = 0, max_nb = 0;
  for (int i = 0; i < na; i++) {
    max_npad = std::max(max_npad, L.nepad[sel[i]]);
    max_nb = std::max(max_nb, L.nbv[sel[i]]);
  }
  const int maxh = std::max(1, max_nb / 2);
  // FP32 round updates on the tensor cores only when the tensor-core policy
  // forces every FP32 product onto them (ctebd_set_tensor_cores(2)): measured
  // on 2048-wide batches, the CUDA-core round update is faster (the tile
  // products' operand staging is latency-bound at K = 64)
  const bool tc_apply = !f64 && g_tc_mode == 2;
  // per problem 4 counters (zeroed every sweep), then per problem the trace,
  // then maxh pair flags per problem; then the device-side loop's cumulative
  // counters (3 per problem + the sweep count), in the handle's high-water
  // scratch (no allocation once it has grown)
  const size_t n_mv = (size_t)na * maxh;   // per problem and pair slot: moved weight of the sweep
  const size_t n_dbl = 5 * (size_t)na + n_mv + ((size_t)na * maxh + 1) / 2;
  const size_t n_cum = 4 * (size_t)na + 1;
  // the sweep graph's compact descriptor copies and chain selector
  const size_t n_cmp = (kSweepCompact * sizeof(EigProb) + sizeof(double)) / sizeof(double) + 1;
  TRY(ensure_eig_scratch(m, n_dbl + n_cum + n_cmp));
  double* d_off = m->eig_scr;
  double* d_cum = m->eig_scr + n_dbl;
  EigProb* d_compact = reinterpret_cast<EigProb*>(m->eig_scr + n_dbl + n_cum);
  int* d_mode = reinterpret_cast<int*>(d_compact + kSweepCompact);
  double* d_mv = d_off + 5 * na;
  int* d_flag = reinterpret_cast<int*>(d_mv + n_mv);
  for (int i = 0; i < na; i++) {
    const int a = sel[i];
    Work& w = ws[L.act[a]];
    eps[i].G = w.G; eps[i].V = acc[i]; eps[i].J = w.J;
    eps[i].npad = L.nepad[a]; eps[i].nb = L.nbv[a]; eps[i].active = 1; eps[i].nact = L.ne[a];
    eps[i].off = d_off + 4 * i;
    eps[i].scale = d_off + 4 * na + i;
    eps[i].floor_factor = floor_factor;
    eps[i].jflag = d_flag + (size_t)i * maxh;
    eps[i].rel_skip = rel_skip;
    eps[i].T = w.T;
    if (tc_apply && !w.T) return fail(CTEBD_ERR_STATE, "internal: no round-update scratch");
    if (use_cut) {   // columns sorted by the previous pass: [lo, hi) around the cut
      eps[i].move_rel = 1e-13;
      // a sweep that moves at most this much weight in all ends the solve:
      // far below the 1e-5 target on f, and below a hundredth of the cutoff
      eps[i].move_tol = m->cfg.cutoff > 0 ? std::min(1e-10, 1e-2 * m->cfg.cutoff) : 1e-10;
      eps[i].mv = d_mv + (size_t)i * maxh;
      eps[i].cut_lo = (int)m->h_res[16 * a + 6];
      eps[i].cut_hi = std::max(1, (int)m->h_res[16 * a + 7]);
    }
  }
  if (tc_apply) TRY(ensure_tc_err(m));
  const EigProb* dep;
  TRY(m->stage.push(eps.data(), eps.size(), &dep));
  {
    ProfScope ps(m->prof, m->stream, KK_EIG_INIT, 0, 0);
    CUDA_TRY(f64 ? launch_eig_init<double>(dep, na, max_npad, m->stream)
                 : launch_eig_init<float>(dep, na, max_npad, m->stream));
    CUDA_TRY(f64 ? launch_eig_trace<double>(dep, na, m->stream) : launch_eig_trace<float>(dep, na, m->stream));
  }
  const int max_sweeps = g_max_sweeps;
  // A refinement pass whose last sweep moved at most kCapAccept of the trace
  // is accepted at the sweep cap (the split's f is then exact to about that
  // level, far below 1e-5) and counted in solve_stats; anything else left
  // rotating is an error.
  constexpr double kCapAccept = 1e-8;
  auto capped = [&](int i, double moved) {
    if (!use_cut || !(moved <= kCapAccept)) return false;
    m->solve_stats[0] += 1;
    m->solve_stats[1] = std::max(m->solve_stats[1], moved);
    (void)i;
    return true;
  };
  auto not_converged = [&](int count, double moved) {
    char tail[96];
    snprintf(tail, sizeof tail, " (%s pass; the last sweep moved up to %.2e of the trace)",
             use_cut ? "refinement" : "first", moved);
    return fail(CTEBD_ERR_NUMERIC, "Jacobi eigen-solve: " + std::to_string(count) + " of " +
                                       std::to_string(na) + " problems still rotating after " +
                                       std::to_string(max_sweeps) + " sweeps" + tail);
  };
  if (!m->prof.on && (g_sweep_graphs == 2 || (g_sweep_graphs == 1 && max_nb >= kGraphMinBlocks))) {
    // cumulative counters (rotations, applied flops, sweeps per problem) + sweep count
    CUDA_TRY(cudaMemsetAsync(d_cum, 0, sizeof(double) * n_cum, m->stream));
    CUDA_TRY(cudaMemsetAsync(d_off, 0, sizeof(double) * 4 * na, m->stream));
    CUDA_TRY(cudaMemsetAsync(d_mv, 0, sizeof(double) * n_mv, m->stream));
    CUDA_TRY(cudaMemsetAsync(d_mode, 0, sizeof(int), m->stream));   // first sweep: the full chain
    CUDA_TRY(eig_prepare(f64));
    if (tc_apply) CUDA_TRY(eig_apply_tc_prepare());
    std::vector<int> nbs(na);
    for (int i = 0; i < na; i++) nbs[i] = eps[i].nb;
    const int rc = run_sweep_graph(m, const_cast<EigProb*>(dep), na, nbs, d_cum, max_sweeps, tc_apply, d_compact,
                                   d_mode);
    std::vector<double> hc(n_cum, 0.0);
    std::vector<EigProb> fin(na);   // descriptors after the loop: active = still rotating
    if (rc == CTEBD_OK) {
      CUDA_TRY(cudaMemcpyAsync(hc.data(), d_cum, sizeof(double) * n_cum, cudaMemcpyDeviceToHost, m->stream));
      CUDA_TRY(cudaMemcpyAsync(fin.data(), dep, sizeof(EigProb) * na, cudaMemcpyDeviceToHost, m->stream));
      CUDA_TRY(cudaStreamSynchronize(m->stream));
    }
    TRY(rc);
    // launches: every sweep runs both halves' rounds (counted as for one batch)
    const double rounds = hc[4 * na] * (max_nb - 1);
    m->prof.launches[KK_EIG_INNER] += hc[4 * na] * (max_nb > 2 ? max_nb : 1);   // + the one-pair launch
    m->prof.launches[KK_EIG_APPLY] += rounds * (tc_apply ? 2 : 1);
    if (tc_apply) m->prof.tc[KK_EIG_APPLY] += rounds * 2;
    for (int i = 0; i < na; i++) {
      // inner-solve work: 14 flops per element pair, 3 vectors of length 2JB per rotation
      m->prof.flops[KK_EIG_INNER] += hc[4 * i] * 42.0 * (2 * JB);
      m->prof.flops[KK_EIG_APPLY] += hc[4 * i + 1];
      sweeps[sel[i]] += (int)hc[4 * i + 2];
    }
    int left = 0;
    double moved = 0;
    for (int i = 0; i < na; i++)
      if (fin[i].active && !capped(i, hc[4 * i + 3])) { left++; moved = std::max(moved, hc[4 * i + 3]); }
    if (left) return not_converged(left, moved);
    return CTEBD_OK;
  }
  std::vector<double> hoff(5 * na + n_mv);   // counters, the traces, the moved weights
  std::vector<double> last_moved(na, 0.0);
  std::vector<int> sweeps0(na);
  for (int i = 0; i < na; i++) sweeps0[i] = sweeps[sel[i]];
  for (int sweep = 0; sweep < max_sweeps; sweep++) {
    CUDA_TRY(cudaMemsetAsync(d_off, 0, sizeof(double) * 4 * na, m->stream));
    CUDA_TRY(cudaMemsetAsync(d_mv, 0, sizeof(double) * n_mv, m->stream));
    double fap_sweep = 0, bap_sweep = 0;
    for (int t = 0; t < max_nb - 1; t++) {
      double bin = 0;
      const double D = 2.0 * JB;
      for (int i = 0; i < na; i++) {
        const int a = sel[i];
        if (!eps[i].active || t >= L.nbv[a] - 1) continue;
        const double h = L.nbv[a] / 2, np2 = (double)L.nepad[a] * L.nepad[a];
        bin += 2 * h * D * D * m->esz;                                 // read blocks, write J
        fap_sweep += 8.0 * (2 * h * (h + 1) / 2 + h * h) * D * D * D;  // J^H G J (upper tiles), V J
        bap_sweep += (4 * np2 + h * D * D) * m->esz;                   // G, V read+write, J read
      }
      {
        ProfScope ps(m->prof, m->stream, KK_EIG_INNER, 0, bin);
        m->prof.launches[KK_EIG_INNER] += eig_inner_launches(max_nb, t) - 1;
        CUDA_TRY(f64 ? launch_eig_inner<double>(dep, na, max_nb, t, m->stream)
                     : launch_eig_inner<float>(dep, na, max_nb, t, m->stream));
      }
      {
        // flops and bytes are added after the sweep from the tiles actually updated
        ProfScope ps(m->prof, m->stream, KK_EIG_APPLY, 0, 0);
        if (tc_apply) {
          m->prof.launches[KK_EIG_APPLY] += 1;   // two launches (phases) per round
          m->prof.tc[KK_EIG_APPLY] += 2;
          CUDA_TRY(launch_eig_apply_tc(dep, na, max_nb, max_npad, t, m->tc_err, m->stream));
        } else {
          CUDA_TRY(f64 ? launch_eig_apply<double>(dep, na, max_nb, t, m->stream)
                       : launch_eig_apply<float>(dep, na, max_nb, t, m->stream));
        }
      }
    }
    CUDA_TRY(cudaMemcpyAsync(hoff.data(), d_off, sizeof(double) * (5 * na + n_mv), cudaMemcpyDeviceToHost,
                             m->stream));
    CUDA_TRY(cudaStreamSynchronize(m->stream));
    bool any = false;
    double fap_done = 0;
    for (int i = 0; i < na; i++) {
      if (eps[i].active) sweeps[sel[i]] += 1;
      // inner-solve work: 14 flops per element pair, 3 vectors of length 2JB per rotation
      m->prof.flops[KK_EIG_INNER] += hoff[4 * i + 1] * 42.0 * (2 * JB);
      fap_done += hoff[4 * i + 2];
      if (!eps[i].active) continue;
      // same rules as the device-side loop's k_sweep_end
      double mw = 0;   // summed in slot order, as on the device
      for (int k = 0; k < eps[i].nb / 2; k++) mw += hoff[5 * na + (size_t)i * maxh + k];
      const double moved = mw / hoff[4 * na + i];
      if (eps[i].cut_hi > 0 && eps[i].move_tol > 0 && sweeps[sel[i]] - sweeps0[i] >= 6 && moved > 0.9 * last_moved[i])
        eps[i].cut_hi = 0;
      last_moved[i] = moved;
      const bool settled = eps[i].move_tol > 0 && moved <= eps[i].move_tol;
      if (hoff[4 * i] == 0.0 || settled) eps[i].active = 0; else any = true;
    }
    m->prof.flops[KK_EIG_APPLY] += fap_done;
    if (fap_sweep > 0) m->prof.bytes[KK_EIG_APPLY] += bap_sweep * (fap_done / fap_sweep);
    if (!any) break;
    m->stage.reset();
    TRY(m->stage.push(eps.data(), eps.size(), &dep));
  }
  int left = 0;
  double moved = 0;
  for (int i = 0; i < na; i++)
    if (eps[i].active && !capped(i, last_moved[i])) { left++; moved = std::max(moved, last_moved[i]); }
  if (left) return not_converged(left, moved);
  return CTEBD_OK;
}

// Rfull = Mbar V (bufB, m x ne), rho = weighted column norms, truncation
// select (with the total weight ||M||^2 for sketched problems); results to host
static int level_project_select(ctebd_mps* m, std::vector<Work>& ws, const Level& L,
                                const std::vector<int>& sel) {
  const bool f64 = m->fp64;
  const double floor_rel = f64 ? 1e-13 : 1e-6;
  const int na = (int)sel.size();
  if (na == 0) return CTEBD_OK;
  std::vector<GemmProb> probs;
  int max_n = 0, max_m = 0;
  for (int a : sel) {
    Work& w = ws[L.act[a]];
    GemmProb p{};
    p.M = L.mm[a]; p.N = L.ne[a]; p.K = L.nn[a]; p.batch = 1;
    p.A = w.bufA; p.lda = L.nn[a]; p.opA = 0;
    p.B = w.V; p.ldb = L.vld[a]; p.opB = 0;
    p.C = w.bufB; p.ldc = L.ne[a]; p.alpha = 1.0;
    probs.push_back(p);
    CUDA_TRY(cudaMemsetAsync(w.rho, 0, sizeof(double) * L.ne[a], m->stream));
    CUDA_TRY(cudaMemsetAsync(w.rho + w.nmax, 0, sizeof(double) * L.ne[a], m->stream));
    max_n = std::max(max_n, L.ne[a]);
    max_m = std::max(max_m, std::max(L.mm[a], L.nn[a]));
  }
  TRY(run_gemms(m, probs, KK_GEMM_PROJ));
  {
    // problems 0..na-1: weighted column norms of Rfull (rho); na..2na-1:
    // squared column norms of V (vn), which normalise rho and the write-back
    std::vector<const void*> R(2 * na);
    std::vector<const double*> Lm(2 * na);
    std::vector<double*> rho(2 * na);
    std::vector<int> mm(2 * na), nn(2 * na), sh(2 * na), ld(2 * na);
    double by = 0;
    for (int i = 0; i < na; i++) {
      const int a = sel[i];
      Work& w = ws[L.act[a]];
      R[i] = w.bufB; Lm[i] = m->lam[w.q0]; rho[i] = w.rho;
      mm[i] = L.mm[a]; nn[i] = L.ne[a]; sh[i] = L.shift[a]; ld[i] = L.ne[a];
      R[na + i] = w.V; Lm[na + i] = nullptr; rho[na + i] = w.rho + w.nmax;
      mm[na + i] = L.nn[a]; nn[na + i] = L.ne[a]; sh[na + i] = 0; ld[na + i] = L.vld[a];
      by += ((double)L.mm[a] + L.nn[a]) * L.ne[a] * m->esz;
    }
    const void* const* dR; const int *dm, *dn, *dsh, *dld; const double* const* dL; double* const* drho;
    TRY(m->stage.push(R.data(), 2 * na, (const void* const**)&dR));
    TRY(m->stage.push(mm.data(), 2 * na, &dm));
    TRY(m->stage.push(nn.data(), 2 * na, &dn));
    TRY(m->stage.push(sh.data(), 2 * na, &dsh));
    TRY(m->stage.push(ld.data(), 2 * na, &dld));
    TRY(m->stage.push(Lm.data(), 2 * na, (const double* const**)&dL));
    TRY(m->stage.push(rho.data(), 2 * na, (double* const**)&drho));
    ProfScope ps(m->prof, m->stream, KK_COLNORM, 0, by);
    CUDA_TRY(f64 ? launch_colnorm_batch<double>(dR, dm, dn, dld, dL, dsh, drho, 2 * na, max_n, max_m, m->stream)
                 : launch_colnorm_batch<float>(dR, dm, dn, dld, dL, dsh, drho, 2 * na, max_n, max_m, m->stream));
    CUDA_TRY(launch_rho_normalize(drho, drho + na, dn, na, max_n, m->stream));
  }
  std::vector<SelProb> sp(na);
  for (int i = 0; i < na; i++) {
    const int a = sel[i];
    Work& w = ws[L.act[a]];
    sp[i].rho = w.rho; sp[i].n = L.ne[a]; sp[i].perm = w.perm;
    sp[i].lam_out = m->lam[w.q0 + L.shift[a]]; sp[i].res = w.res;
    sp[i].W_ext = L.sk[a] ? w.res + 8 : nullptr;
    sp[i].rank_cap = L.mm[a];
    if (L.ne[a] > 4096) return fail(CTEBD_ERR_ARG, "split wider than 4096");
  }
  const SelProb* dsp;
  TRY(m->stage.push(sp.data(), na, &dsp));
  {
    ProfScope pss(m->prof, m->stream, KK_SELECT, 0, 0);
    // FP32 pass 1 leaves couplings of up to ~8 eps W: weights within 16 eps W
    // of the cut may still cross it, and kept weights below 1024 eps W are not
    // resolved relative to their own size -- their second-order error
    // (8 eps W)^2 / gap reaches 1e-3 of the weight on spectra whose neighbours
    // are a few per cent apart (refinement pass classes)
    const double eps32 = 1.1920928955078125e-07;
    const double band = f64 ? 0.0 : 16.0 * eps32, resolved = f64 ? 0.0 : 1024.0 * eps32;
    CUDA_TRY(launch_select(dsp, na, m->cfg.chi_max, m->cfg.cutoff, band, resolved, floor_rel * floor_rel,
                           m->stream));
  }
  // results land at the level-local index a (h_res[16 a .. 16 a + 15])
  if (L.act.size() > m->h_res_cap) return fail(CTEBD_ERR_ARG, "too many clusters");
  for (int a : sel)
    CUDA_TRY(cudaMemcpyAsync(m->h_res + 16 * a, ws[L.act[a]].res, 16 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  m->stage.reset();
  return CTEBD_OK;
}

// CholeskyQR passes on the columns of X (rows x l, ld l) -> orthonormal Q in
// out; shifted first pass (shifted CholeskyQR3) so the Cholesky never breaks
// down on rank-deficient or ill-conditioned sketches.
static int level_cholqr(ctebd_mps* m, std::vector<Work>& ws, const Level& L, const std::vector<int>& sel,
                        const std::vector<int>& rows, const std::vector<int>& lcols,
                        std::vector<void*>& X, std::vector<void*>& tmp) {
  const int na = (int)sel.size();
  for (int pass = 0; pass < 3; pass++) {
    std::vector<GemmProb> gram, mul;
    std::vector<CholProb> cp(na);
    for (int i = 0; i < na; i++) {
      Work& w = ws[L.act[sel[i]]];
      const int l = lcols[i];
      CUDA_TRY(cudaMemsetAsync(w.G, 0, (size_t)l * l * m->esz, m->stream));
      GemmProb g{};
      g.M = l; g.N = l; g.K = rows[i]; g.batch = 1;
      g.A = X[i]; g.lda = l; g.opA = 1; g.B = X[i]; g.ldb = l; g.opB = 0;
      g.C = w.G; g.ldc = l; g.alpha = 1.0;
      gram.push_back(g);
      cp[i].G = w.G; cp[i].ldg = l; cp[i].l = l;
      cp[i].shift_rel = pass == 0 ? 1e-5 : 0.0;
      cp[i].dead_rel = pass == 0 ? 0.0 : 2e-6;
      cp[i].dead = w.perm;   // perm is free until the select
      cp[i].X = w.X; cp[i].ldx = l;
      cp[i].work = (double2*)w.CW;
      cp[i].status = (int*)(w.res + 12);
      GemmProb q{};
      q.M = rows[i]; q.N = l; q.K = l; q.batch = 1;
      q.A = X[i]; q.lda = l; q.opA = 0; q.B = w.X; q.ldb = l; q.opB = 0;
      q.C = tmp[i]; q.ldc = l; q.alpha = 1.0;
      mul.push_back(q);
    }
    TRY(run_gemms(m, gram, KK_GEMM_GRAM));
    const CholProb* dcp;
    TRY(m->stage.push(cp.data(), cp.size(), &dcp));
    {
      ProfScope ps(m->prof, m->stream, KK_CHOL, 0, 0);
      CUDA_TRY(launch_chol_inv(dcp, na, m->stream));
    }
    TRY(run_gemms(m, mul, KK_GEMM_PROJ));
    std::swap(X, tmp);
  }
  std::vector<int> st(na);
  for (int i = 0; i < na; i++)
    CUDA_TRY(cudaMemcpyAsync(&st[i], ws[L.act[sel[i]]].res + 12, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  m->stage.reset();
  for (int i = 0; i < na; i++)
    if (st[i] != 0) return fail(CTEBD_ERR_NUMERIC, "CholeskyQR: non-finite sketch");
  return CTEBD_OK;
}

// Sketched basis (spec range finder): Y = M Omega (power iterations
// Y <- M M^H Y), Q = CholQR(Y), B^H = M^H Q, Q_B = CholQR(B^H); then
// Z = Mbar Q_B (bufB) for the Rayleigh-Ritz Gram.  M = diag(lambda_L) Mbar.
static int level_sketch(ctebd_mps* m, std::vector<Work>& ws, const Level& L, const std::vector<int>& sel,
                        uint64_t step_key) {
  const int na = (int)sel.size();
  if (na == 0) return CTEBD_OK;
  auto rowscale = [&](const std::vector<void*>& Xs, const std::vector<int>& rows) -> int {
    std::vector<RowScaleProb> rp(na);
    long long mx = 0;
    for (int i = 0; i < na; i++) {
      const int a = sel[i];
      rp[i].X = Xs[i]; rp[i].rows = rows[i]; rp[i].cols = L.ne[a]; rp[i].ld = L.ne[a];
      rp[i].lam = m->lam[ws[L.act[a]].q0]; rp[i].shift = L.shift[a];
      mx = std::max(mx, (long long)rows[i] * L.ne[a]);
    }
    const RowScaleProb* drp;
    TRY(m->stage.push(rp.data(), rp.size(), &drp));
    CUDA_TRY(launch_rowscale(drp, na, mx, m->stream));
    return CTEBD_OK;
  };
  std::vector<int> mrows(na), nrows(na), ls(na);
  std::vector<void*> Y(na), Qv(na), Bv(na), QBv(na);
  for (int i = 0; i < na; i++) {
    const int a = sel[i];
    Work& w = ws[L.act[a]];
    mrows[i] = L.mm[a]; nrows[i] = L.nn[a]; ls[i] = L.ne[a];
    Y[i] = w.Ys; Qv[i] = w.Qs; Bv[i] = w.Bs; QBv[i] = w.QB;
    // Omega (n x l) in QB, counter-based: key = seed, stream = (step, cluster, bond)
    const uint64_t stream = (step_key << 24) ^ ((uint64_t)w.q0 << 8) ^ (uint64_t)L.shift[a];
    CUDA_TRY(launch_gauss(w.QB, (long long)L.nn[a] * L.ne[a], m->cfg.seed, stream, m->stream));
  }
  auto gemm_MY = [&](const std::vector<void*>& B, const std::vector<void*>& C) -> int {  // C = Mbar B
    std::vector<GemmProb> pr;
    for (int i = 0; i < na; i++) {
      const int a = sel[i];
      GemmProb p{};
      p.M = L.mm[a]; p.N = L.ne[a]; p.K = L.nn[a]; p.batch = 1;
      p.A = ws[L.act[a]].bufA; p.lda = L.nn[a]; p.opA = 0;
      p.B = B[i]; p.ldb = L.ne[a]; p.opB = 0; p.C = C[i]; p.ldc = L.ne[a]; p.alpha = 1.0;
      pr.push_back(p);
    }
    return run_gemms(m, pr, KK_GEMM_SKETCH);
  };
  auto gemm_MhY = [&](const std::vector<void*>& B, const std::vector<void*>& C) -> int {  // C = Mbar^H D B
    std::vector<GemmProb> pr;
    for (int i = 0; i < na; i++) {
      const int a = sel[i];
      Work& w = ws[L.act[a]];
      GemmProb p{};
      p.M = L.nn[a]; p.N = L.ne[a]; p.K = L.mm[a]; p.batch = 1;
      p.A = w.bufA; p.lda = L.nn[a]; p.opA = 1;
      p.B = B[i]; p.ldb = L.ne[a]; p.opB = 0; p.C = C[i]; p.ldc = L.ne[a]; p.alpha = 1.0;
      p.kw = m->lam[w.q0]; p.kw_shift = L.shift[a]; p.kw_pow = 1;
      pr.push_back(p);
    }
    return run_gemms(m, pr, KK_GEMM_SKETCH);
  };
  TRY(gemm_MY(QBv, Y));                // Y = Mbar Omega
  TRY(rowscale(Y, mrows));             // Y = M Omega
  for (int q = 0; q < m->cfg.power_iters; q++) {
    TRY(gemm_MhY(Y, Bv));              // Z = M^H Y
    TRY(gemm_MY(Bv, Y));
    TRY(rowscale(Y, mrows));           // Y = M Z
  }
  // level_cholqr leaves the orthonormal factor in the buffers its first vector
  // names on return (three ping-pong passes): Q ends in Qs, Q_B in QB
  TRY(level_cholqr(m, ws, L, sel, mrows, ls, Y, Qv));
  TRY(gemm_MhY(Y, Bv));                // B^H = M^H Q   (n x l)
  std::vector<void*> Bx = Bv, Btmp = QBv;
  TRY(level_cholqr(m, ws, L, sel, nrows, ls, Bx, Btmp));
  for (int i = 0; i < na; i++)
    if (Bx[i] != ws[L.act[sel[i]]].QB || Y[i] != ws[L.act[sel[i]]].Qs)
      return fail(CTEBD_ERR_STATE, "internal: CholeskyQR buffer hand-off");
  std::vector<void*> Zb(na);
  for (int i = 0; i < na; i++) Zb[i] = ws[L.act[sel[i]]].bufB;
  TRY(gemm_MY(Bx, Zb));                // Z = Mbar Q_B
  // ||M||_F^2 (FP64) for the tail check and the total weight of the select
  std::vector<WNormProb> wp(na);
  long long mx = 0;
  for (int i = 0; i < na; i++) {
    const int a = sel[i];
    Work& w = ws[L.act[a]];
    CUDA_TRY(cudaMemsetAsync(w.res + 8, 0, sizeof(double), m->stream));
    wp[i].X = w.bufA; wp[i].rows = L.mm[a]; wp[i].cols = L.nn[a]; wp[i].ld = L.nn[a];
    wp[i].lam = m->lam[w.q0]; wp[i].shift = L.shift[a]; wp[i].out = w.res + 8;
    mx = std::max(mx, (long long)L.mm[a] * L.nn[a]);
  }
  const WNormProb* dwp;
  TRY(m->stage.push(wp.data(), wp.size(), &dwp));
  CUDA_TRY(launch_wnorm(dwp, na, mx, m->stream));
  return CTEBD_OK;
}

// pass 1 (+ FP32 pass 2) for a selection: Gram of Z, eigen-solve, V, weights, select
static int level_solve(ctebd_mps* m, std::vector<Work>& ws, Level& L, const std::vector<int>& sel) {
  if (sel.empty()) return CTEBD_OK;
  const bool f64 = m->fp64;
  std::vector<const void*> Z;
  std::vector<void*> accV;
  for (int a : sel) {
    Work& w = ws[L.act[a]];
    Z.push_back(L.sk[a] ? w.bufB : w.bufA);
    accV.push_back(L.sk[a] ? w.W : w.V);
  }
  TRY(level_gram(m, ws, L, sel, Z));
  TRY(level_eig(m, ws, L, sel, accV, 1.0, 4.0, L.sw1));
  // sketched problems: V = Q_B W (n x l, ld nepad) into V
  {
    std::vector<GemmProb> probs;
    for (int a : sel) {
      if (!L.sk[a]) continue;
      Work& w = ws[L.act[a]];
      GemmProb p{};
      p.M = L.nn[a]; p.N = L.ne[a]; p.K = L.ne[a]; p.batch = 1;
      p.A = w.QB; p.lda = L.ne[a]; p.opA = 0;
      p.B = w.W; p.ldb = L.nepad[a]; p.opB = 0;
      p.C = w.V; p.ldc = L.vld[a]; p.alpha = 1.0;
      probs.push_back(p);
    }
    TRY(run_gemms(m, probs, KK_GEMM_PROJ));
  }
  TRY(level_project_select(m, ws, L, sel));
  if (f64) return CTEBD_OK;
  // pass 2 (FP32).  Pass 1 resolves the spectrum of G only to an absolute
  // level of about eps * trace(G): a kept direction p of weight rho_p can keep
  // couplings of that size to discarded ones and so lose up to
  // ~ n (eps trace)^2 / rho_p of its weight -- summed over the kept set this
  // exceeds 1e-5 of the total for n ~ 2048 with a flat spectrum, whether the
  // cutoff or chi_max decides the rank.  Re-diagonalise the freshly computed
  // Gram of the rotated columns Z = M V (whose rounding is relative to each
  // column's own weight) with relative thresholds only, and rotate V and Z by
  // the result.  Rotations below 32 eps sqrt(a d) are skipped: the weight they
  // could move is below n (32 eps)^2 of the total.  A rotation keeps the
  // sweeps going only if it moves more than 1e-13 of the total weight: among
  // directions whose weights sit at the rounding level the relative test
  // alone never settles, and what such rotations leave unmoved is below
  // n^2 / 2 * 1e-13 of the total.  The pass also ends after a sweep whose
  // significant rotations moved at most min(1e-10, cutoff / 100) of the total
  // in all; a problem whose moved weight stalls rotates every pair from then
  // on (the skipped classes below otherwise keep renewing couplings across
  // the cut); see level_eig for the sweep cap.
  //
  // The kept weight is a sum over the kept set and the tail a sum over the
  // discarded set, so rotations within either set change neither.  With the
  // columns sorted by their pass-1 weight, pairs of surely discarded
  // directions are skipped, and so are pairs of kept directions whose weights
  // pass 1 already resolved (>= 1024 eps W: their Rayleigh quotients are
  // accurate to second order); block pairs entirely in one such class are
  // skipped outright.
  // Refine where something is discarded, and where a cutoff is set and pass 1
  // left directions below its resolution (weights under 1024 eps W, or within
  // the band of the smallest kept one): their pass-1 weights are mixtures of
  // everything below ~eps W, so a cutoff smaller than that would otherwise
  // keep every direction.  Nothing to refine where every direction is kept
  // and resolved, or where no cutoff applies.
  std::vector<int> ref;
  for (int a : sel) {
    const double* res = m->h_res + 16 * a;
    const bool discarded = (int)res[0] < L.ne[a];
    const bool unresolved = m->cfg.cutoff > 0 && (int)res[6] < L.ne[a];
    if (discarded || unresolved) ref.push_back(a);
  }
  if (ref.empty()) return CTEBD_OK;
  std::vector<const void*> Z2;
  for (int a : ref) Z2.push_back(ws[L.act[a]].bufB);
  TRY(level_gram(m, ws, L, ref, Z2));
  {
    // Gram rows / columns and V columns into descending pass-1 order
    std::vector<PermProb> pg, pv;
    long long mg = 0, mv = 0;
    for (int a : ref) {
      Work& w = ws[L.act[a]];
      PermProb g{};
      g.src = w.G; g.dst = w.W; g.perm = w.perm; g.rows = L.nepad[a]; g.cols = L.ne[a];
      g.lds = L.nepad[a]; g.ldd = L.nepad[a]; g.mode = 1;
      pg.push_back(g);
      mg = std::max(mg, (long long)L.nepad[a] * L.nepad[a]);
      PermProb v{};
      v.src = w.V; v.dst = w.G; v.perm = w.perm; v.rows = L.nn[a]; v.cols = L.ne[a];
      v.lds = L.vld[a]; v.ldd = L.vld[a]; v.mode = 0;
      pv.push_back(v);
      mv = std::max(mv, (long long)L.nn[a] * L.ne[a]);
    }
    const PermProb *dpg, *dpv;
    TRY(m->stage.push(pg.data(), pg.size(), &dpg));
    TRY(m->stage.push(pv.data(), pv.size(), &dpv));
    ProfScope ps(m->prof, m->stream, KK_GATHER, 0, 0);
    // sorted Gram -> W; the raw Gram (G) is then free for the sorted V
    CUDA_TRY(f64 ? launch_permute<double>(dpg, (int)pg.size(), mg, m->stream)
                 : launch_permute<float>(dpg, (int)pg.size(), mg, m->stream));
    CUDA_TRY(f64 ? launch_permute<double>(dpv, (int)pv.size(), mv, m->stream)
                 : launch_permute<float>(dpv, (int)pv.size(), mv, m->stream));
    for (int a : ref) {
      Work& w = ws[L.act[a]];
      void* gram = w.W;   // sorted Gram
      w.W = w.V;          // old V: free, the pass-2 accumulator
      w.V = w.G;          // sorted V
      w.G = gram;
    }
  }
  std::vector<void*> accW;
  for (int a : ref) accW.push_back(ws[L.act[a]].W);
  TRY(level_eig(m, ws, L, ref, accW, 1e-12, 32.0, L.sw2, true));
  std::vector<GemmProb> probs;
  for (int a : ref) {
    Work& w = ws[L.act[a]];
    GemmProb p{};
    p.M = L.nn[a]; p.N = L.ne[a]; p.K = L.ne[a]; p.batch = 1;
    p.A = w.V; p.lda = L.vld[a]; p.opA = 0;
    p.B = w.W; p.ldb = L.nepad[a]; p.opB = 0;
    p.C = w.G; p.ldc = L.vld[a]; p.alpha = 1.0;
    probs.push_back(p);
  }
  TRY(run_gemms(m, probs, KK_GEMM_PROJ));
  for (int a : ref) std::swap(ws[L.act[a]].V, ws[L.act[a]].G);
  return level_project_select(m, ws, L, ref);
}

// k-1 splits, right to left (Fig. 2 with the truncation of Fig. 3)
static int split_levels(ctebd_mps* m, std::vector<Work>& ws, std::vector<std::vector<double>>& fs,
                        uint64_t step_key) {
  const bool f64 = m->fp64;
  const int JB = eig_block(f64);
  const int p_over = m->cfg.sketch_oversample;
  fs.assign(ws.size(), {});
  int kmax = 0;
  for (auto& w : ws) kmax = std::max(kmax, w.k);
  for (int lev = 1; lev < kmax; lev++) {
    Level L;
    for (size_t i = 0; i < ws.size(); i++) if (ws[i].k - 1 >= lev) L.act.push_back((int)i);
    if (L.act.empty()) break;
    const int na = (int)L.act.size();
    for (auto* v : {&L.mm, &L.nn, &L.npad, &L.shift, &L.ne, &L.nepad, &L.nbv, &L.vld}) v->resize(na);
    L.sk.assign(na, 0);
    L.sw1.assign(na, 0);
    L.sw2.assign(na, 0);
    std::vector<int> sk_sel, full_sel;
    for (int a = 0; a < na; a++) {
      Work& w = ws[L.act[a]];
      const int j = w.k - lev;  // bond q0 + j is split off
      L.mm[a] = w.chiL << j;
      L.nn[a] = 2 * w.rdim;
      L.shift[a] = j;
      L.npad[a] = (int)round_up(L.nn[a], 2 * JB);
      if ((size_t)L.npad[a] * L.npad[a] > w.eigElems) return fail(CTEBD_ERR_ARG, "internal: eig buffer");
      level_set_full(L, a, JB);
      // sketched split when a rank hint makes the sketch at most half the width
      const int h = w.hint[j - 1];
      if (!f64 && p_over > 0 && h > 0) {
        const int l = h + p_over;
        if (2 * l <= L.nn[a] && (size_t)L.mm[a] * l <= w.bufElems / 2) {
          L.sk[a] = 1;
          L.ne[a] = l;
          L.nepad[a] = (int)round_up(l, 2 * JB);
          L.nbv[a] = L.nepad[a] / JB;
          L.vld[a] = L.nepad[a];
          sk_sel.push_back(a);
          continue;
        }
      }
      full_sel.push_back(a);
    }
    // sketched splits: tail check on the weight outside the sketch (must be
    // below max(cutoff, 1e-6) W); a rejected sketch is retried once with twice
    // the columns when that still fits in half the width, then falls back to
    // the full eigen-solve
    for (int round = 0; round < 2 && !sk_sel.empty(); round++) {
      TRY(level_sketch(m, ws, L, sk_sel, step_key * 2 + round));
      TRY(level_solve(m, ws, L, sk_sel));
      const double tol = std::max(m->cfg.cutoff, 1e-6);
      std::vector<int> retry;
      for (int a : sk_sel) {
        const double* res = m->h_res + 16 * a;
        const double Wt = res[2], inside = res[5];
        m->sk_stats[0] += 1;
        if (Wt - inside <= tol * Wt) continue;
        Work& w = ws[L.act[a]];
        const int l2 = 2 * L.ne[a];
        if (round == 0 && 2 * l2 <= L.nn[a] && (size_t)L.mm[a] * l2 <= w.bufElems / 2) {
          L.ne[a] = l2;
          L.nepad[a] = (int)round_up(l2, 2 * JB);
          L.nbv[a] = L.nepad[a] / JB;
          L.vld[a] = L.nepad[a];
          retry.push_back(a);
          continue;
        }
        m->sk_stats[1] += 1;
        level_set_full(L, a, JB);
        full_sel.push_back(a);
      }
      sk_sel.swap(retry);
    }
    TRY(level_solve(m, ws, L, full_sel));
    // write back: new right sites, unweighted remainders
    std::vector<GatherProb> gp;
    long long maxe = 0;
    for (int a = 0; a < na; a++) {
      Work& w = ws[L.act[a]];
      const int j = w.k - lev;
      const double* res = m->h_res + 16 * a;   // level-local index, as written by the select
      const int r = (int)res[0];
      const double f = res[1], W = res[2], kept = res[3];
      if (!(kept > 0) || !std::isfinite(W)) return fail(CTEBD_ERR_NUMERIC, "split: non-finite or zero weight");
      if (r < 1 || r > L.ne[a] || r > m->cfg.chi_max)
        return fail(CTEBD_ERR_NUMERIC, "split: rank out of range (" + std::to_string(r) + ")");
      const int bnd = w.q0 + j;
      TRY(ensure_site(m, bnd, (size_t)r * L.nn[a]));
      GatherProb g0{};
      g0.src = w.V; g0.dst = m->site[bnd]; g0.perm = w.perm; g0.rows = L.nn[a]; g0.r = r; g0.ld = L.vld[a]; g0.mode = 0;
      g0.cs = w.rho + w.nmax;
      gp.push_back(g0);
      GatherProb g1{};
      g1.src = w.bufB; g1.dst = w.bufA; g1.perm = w.perm; g1.rows = L.mm[a]; g1.r = r; g1.ld = L.ne[a]; g1.mode = 1;
      g1.scale = 1.0 / std::sqrt(kept);
      g1.cs = w.rho + w.nmax;
      gp.push_back(g1);
      maxe = std::max(maxe, std::max((long long)r * L.nn[a], (long long)r * L.mm[a]));
      m->chi[bnd] = r;
      w.rdim = r;
      m->logF += std::log(f);
      fs[L.act[a]].push_back(f);
      const double row[8] = {(double)w.q0, (double)w.k, (double)bnd, (double)L.mm[a], (double)L.nn[a], (double)r, f, W};
      m->splitlog.insert(m->splitlog.end(), row, row + 8);
      const double extra[6] = {(double)L.sk[a], (double)L.ne[a], res[4], (double)w.hint[j - 1],
                               (double)L.sw1[a], (double)L.sw2[a]};
      m->splitlog2.insert(m->splitlog2.end(), extra, extra + 6);
    }
    const GatherProb* dgp;
    TRY(m->stage.push(gp.data(), gp.size(), &dgp));
    double gby = 0;
    for (auto& g : gp) gby += 2.0 * g.rows * g.r * m->esz;
    ProfScope psg(m->prof, m->stream, KK_GATHER, 0, gby);
    CUDA_TRY(f64 ? launch_gather<double>(dgp, (int)gp.size(), maxe, m->stream)
                 : launch_gather<float>(dgp, (int)gp.size(), maxe, m->stream));
  }
  // leftmost site of every cluster: the remainder (chiL*2 x r1)
  for (auto& w : ws) {
    const size_t elems = (size_t)w.chiL * 2 * w.rdim;
    TRY(ensure_site(m, w.q0, elems));
    CUDA_TRY(cudaMemcpyAsync(m->site[w.q0], w.bufA, elems * m->esz, cudaMemcpyDeviceToDevice, m->stream));
  }
  return CTEBD_OK;
}

static int make_work(ctebd_mps* m, const ctebd_cluster* c, Work& w) {
  if (!c || c->k < 2 || c->q0 < 0 || c->q0 + c->k > m->n) return fail(CTEBD_ERR_ARG, "cluster out of range (k >= 2 required)");
  if (c->k > 12) return fail(CTEBD_ERR_ARG, "cluster too large");
  w.q0 = c->q0; w.k = c->k; w.chiL = m->chi[c->q0]; w.chiR = m->chi[c->q0 + c->k];
  for (int j = 0; j < 12; j++) w.hint[j] = (j < c->k - 1 && j < 11) ? c->rank_hint[j] : 0;
  const long long D = 1LL << c->k;
  const long long theta = (long long)w.chiL * D * w.chiR;
  if (theta > (1LL << 31)) return fail(CTEBD_ERR_ARG, "cluster tensor too large");
  return CTEBD_OK;
}

// a tensor-core completion wait that ran out sets the flag; report and clear it
static int check_tc_flag(ctebd_mps* m) {
  if (!m->tc_err) return CTEBD_OK;
  int h = 0;
  CUDA_TRY(cudaMemcpy(&h, m->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (!h) return CTEBD_OK;
  CUDA_TRY(cudaMemset(m->tc_err, 0, sizeof(int)));
  return fail(CTEBD_ERR_TIMEOUT, "a tensor-core completion wait timed out");
}

extern "C" int step(ctebd_mps* m, const ctebd_cluster* c, int n, const double* const* U, double* f_out) {
  if (!m || n < 0 || (n > 0 && (!c || !U))) return fail(CTEBD_ERR_ARG, "step: bad args");
  if (n == 0) return CTEBD_OK;
  std::vector<Work> ws(n);
  std::vector<char> used(m->n, 0);
  for (int i = 0; i < n; i++) {
    TRY(make_work(m, &c[i], ws[i]));
    for (int t = 0; t < c[i].k; t++) {
      if (used[c[i].q0 + t]) return fail(CTEBD_ERR_ARG, "step: clusters overlap");
      used[c[i].q0 + t] = 1;
    }
    if (m->pending.count(c[i].q0)) return fail(CTEBD_ERR_STATE, "step: cluster pending from apply_cluster");
  }
  m->splitlog.clear();
  m->splitlog2.clear();
  m->stage.reset();
  TRY(carve_work(m, ws));
  std::vector<const double*> Us(U, U + n);
  TRY(merge_apply(m, ws, Us));
  std::vector<std::vector<double>> fs;
  TRY(split_levels(m, ws, fs, ++m->nstep));
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  TRY(check_tc_flag(m));
  if (f_out) {
    size_t o = 0;
    for (int i = 0; i < n; i++) for (double f : fs[i]) f_out[o++] = f;
  }
  return CTEBD_OK;
}

extern "C" int apply_cluster(ctebd_mps* m, const ctebd_cluster* c, const double* U) {
  if (!m || !U) return fail(CTEBD_ERR_ARG, "apply_cluster: null argument");
  Work w;
  TRY(make_work(m, c, w));
  if (m->pending.count(c->q0)) return fail(CTEBD_ERR_STATE, "apply_cluster: cluster already pending");
  m->stage.reset();
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  TRY(alloc_owned(m, w));
  std::vector<Work> ws{w};
  std::vector<const double*> Us{U};
  int rc = merge_apply(m, ws, Us);
  if (rc) { free_owned(m, ws[0]); return rc; }
  m->pending[c->q0] = ws[0];
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  return CTEBD_OK;
}

extern "C" int truncate_split(ctebd_mps* m, const ctebd_cluster* c, double* f_out) {
  if (!m || !c) return fail(CTEBD_ERR_ARG, "truncate_split: null argument");
  auto it = m->pending.find(c->q0);
  if (it == m->pending.end() || it->second.k != c->k) return fail(CTEBD_ERR_STATE, "truncate_split: no pending apply_cluster for this cluster");
  std::vector<Work> ws{it->second};
  m->pending.erase(it);
  m->splitlog.clear();
  m->stage.reset();
  std::vector<std::vector<double>> fs;
  m->splitlog2.clear();
  int rc = split_levels(m, ws, fs, ++m->nstep);
  free_owned(m, ws[0]);
  if (rc) return rc;
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  if (f_out) for (size_t i = 0; i < fs[0].size(); i++) f_out[i] = fs[0][i];
  return CTEBD_OK;
}

extern "C" int apply_1q(ctebd_mps* m, int q, const double* u) {
  if (!m || !u || q < 0 || q >= m->n) return fail(CTEBD_ERR_ARG, "apply_1q: bad args");
  m->stage.reset();
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  void* s = m->site[q];
  const int cl = m->chi[q], cr = m->chi[q + 1];
  void* const* ds; const int *dcl, *dcr; const double* du;
  TRY(m->stage.push(&s, 1, (void* const**)&ds));
  TRY(m->stage.push(&cl, 1, &dcl));
  TRY(m->stage.push(&cr, 1, &dcr));
  TRY(m->stage.push(u, 8, &du));
  {
    ProfScope ps(m->prof, m->stream, KK_ONEQ, 28.0 * cl * cr, 4.0 * cl * cr * m->esz);
    CUDA_TRY(m->fp64 ? launch_apply_1q<double>(ds, dcl, dcr, du, 1, (long long)cl * cr, m->stream)
                     : launch_apply_1q<float>(ds, dcl, dcr, du, 1, (long long)cl * cr, m->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  return CTEBD_OK;
}

extern "C" int apply_singletons(ctebd_mps* m, const ctebd_gate* gates, int n_gates,
                                const ctebd_cluster* cl, int ncl, int lo, int hi) {
  if (!m || n_gates < 0 || (n_gates && !gates) || ncl < 0 || (ncl && !cl))
    return fail(CTEBD_ERR_ARG, "apply_singletons: bad args");
  std::vector<char> inc(m->n, 0);
  for (int c = 0; c < ncl; c++)
    for (int t = 0; t < cl[c].k; t++) {
      const int q = cl[c].q0 + t;
      if (q < 0 || q >= m->n) return fail(CTEBD_ERR_ARG, "apply_singletons: cluster out of range");
      inc[q] = 1;
    }
  std::vector<int> order;
  for (int i = 0; i < n_gates; i++)
    if (gates[i].layer > lo && gates[i].layer <= hi && gates[i].n_q == 1 && !inc[gates[i].q[0]]) order.push_back(i);
  if (order.empty()) return CTEBD_OK;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return gates[a].layer < gates[b].layer; });
  std::map<int, std::vector<cd>> prod;
  for (int gi : order) {
    const ctebd_gate& g = gates[gi];
    if (g.q[0] < 0 || g.q[0] >= m->n) return fail(CTEBD_ERR_ARG, "apply_singletons: qubit out of range");
    cd u[16];
    if (gate_dim(g.kind, g.param, u) != 2) return fail(CTEBD_ERR_ARG, "apply_singletons: not a one-qubit gate");
    auto it = prod.find(g.q[0]);
    if (it == prod.end()) { prod[g.q[0]] = std::vector<cd>(u, u + 4); continue; }
    std::vector<cd>& p = it->second;
    const cd r0 = u[0] * p[0] + u[1] * p[2], r1 = u[0] * p[1] + u[1] * p[3];
    const cd r2 = u[2] * p[0] + u[3] * p[2], r3 = u[2] * p[1] + u[3] * p[3];
    p = {r0, r1, r2, r3};
  }
  std::vector<void*> sites;
  std::vector<int> cls, crs;
  std::vector<double> us;
  long long maxe = 0;
  for (auto& kv : prod) {
    const int q = kv.first;
    sites.push_back(m->site[q]);
    cls.push_back(m->chi[q]);
    crs.push_back(m->chi[q + 1]);
    for (const cd& z : kv.second) { us.push_back(z.real()); us.push_back(z.imag()); }
    maxe = std::max(maxe, (long long)m->chi[q] * m->chi[q + 1]);
  }
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  m->stage.reset();
  void* const* ds; const int *dcl, *dcr; const double* du;
  TRY(m->stage.push(sites.data(), sites.size(), (void* const**)&ds));
  TRY(m->stage.push(cls.data(), cls.size(), &dcl));
  TRY(m->stage.push(crs.data(), crs.size(), &dcr));
  TRY(m->stage.push(us.data(), us.size(), &du));
  double e1 = 0;
  for (size_t i = 0; i < sites.size(); i++) e1 += (double)cls[i] * crs[i];
  {
    ProfScope ps(m->prof, m->stream, KK_ONEQ, 28.0 * e1, 4.0 * e1 * m->esz);
    CUDA_TRY(m->fp64 ? launch_apply_1q<double>(ds, dcl, dcr, du, (int)sites.size(), maxe, m->stream)
                     : launch_apply_1q<float>(ds, dcl, dcr, du, (int)sites.size(), maxe, m->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  return CTEBD_OK;
}

extern "C" int fidelity(const ctebd_mps* m, double* F) {
  if (!m || !F) return fail(CTEBD_ERR_ARG, "fidelity: null argument");
  *F = std::exp(m->logF);
  return CTEBD_OK;
}

extern "C" int amplitude(const ctebd_mps* mc, const uint8_t* bits, double* re, double* im) {
  ctebd_mps* m = const_cast<ctebd_mps*>(mc);
  if (!m || !bits || !re || !im) return fail(CTEBD_ERR_ARG, "amplitude: null argument");
  int cmax = 1;
  for (int c : m->chi) cmax = std::max(cmax, c);
  double2 *va = nullptr, *vb = nullptr;
  CUDA_TRY(cudaMallocAsync(&va, sizeof(double2) * cmax, m->stream));
  CUDA_TRY(cudaMallocAsync(&vb, sizeof(double2) * cmax, m->stream));
  const double one[2] = {1.0, 0.0};
  CUDA_TRY(cudaMemcpyAsync(va, one, sizeof(one), cudaMemcpyHostToDevice, m->stream));
  for (int q = 0; q < m->n; q++) {
    if (bits[q] > 1) return fail(CTEBD_ERR_ARG, "amplitude: bits must be 0/1");
    ProfScope ps(m->prof, m->stream, KK_AMP, 8.0 * m->chi[q] * m->chi[q + 1], (double)m->chi[q] * m->chi[q + 1] * m->esz);
    CUDA_TRY(m->fp64 ? launch_amp_step<double>(va, vb, m->site[q], m->chi[q], m->chi[q + 1], bits[q], m->stream)
                     : launch_amp_step<float>(va, vb, m->site[q], m->chi[q], m->chi[q + 1], bits[q], m->stream));
    std::swap(va, vb);
  }
  double out[2];
  CUDA_TRY(cudaMemcpyAsync(out, va, sizeof(out), cudaMemcpyDeviceToHost, m->stream));
  CUDA_TRY(cudaFreeAsync(va, m->stream));
  CUDA_TRY(cudaFreeAsync(vb, m->stream));
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  *re = out[0];
  *im = out[1];
  return CTEBD_OK;
}

extern "C" int mps_bond_dims(const ctebd_mps* m, int* chi) {
  if (!m || !chi) return fail(CTEBD_ERR_ARG, "mps_bond_dims: null argument");
  std::memcpy(chi, m->chi.data(), sizeof(int) * m->chi.size());
  return CTEBD_OK;
}

extern "C" int mps_to_host(const ctebd_mps* mc, int q, double* buf, size_t cap) {
  ctebd_mps* m = const_cast<ctebd_mps*>(mc);
  if (!m || !buf || q < 0 || q >= m->n) return fail(CTEBD_ERR_ARG, "mps_to_host: bad args");
  const long long n = (long long)m->chi[q] * 2 * m->chi[q + 1];
  if ((size_t)(2 * n) > cap) return fail(CTEBD_ERR_ARG, "mps_to_host: buffer too small");
  double* d = nullptr;
  CUDA_TRY(cudaMallocAsync(&d, sizeof(double) * 2 * n, m->stream));
  CUDA_TRY(m->fp64 ? launch_convert_to_c128<double>(m->site[q], d, n, m->stream)
                   : launch_convert_to_c128<float>(m->site[q], d, n, m->stream));
  CUDA_TRY(cudaMemcpyAsync(buf, d, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, m->stream));
  CUDA_TRY(cudaFreeAsync(d, m->stream));
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  return CTEBD_OK;
}

extern "C" int mps_lambda_to_host(const ctebd_mps* mc, int b, double* buf, size_t cap) {
  ctebd_mps* m = const_cast<ctebd_mps*>(mc);
  if (!m || !buf || b < 0 || b > m->n) return fail(CTEBD_ERR_ARG, "mps_lambda_to_host: bad args");
  if ((size_t)m->chi[b] > cap) return fail(CTEBD_ERR_ARG, "mps_lambda_to_host: buffer too small");
  CUDA_TRY(cudaMemcpyAsync(buf, m->lam[b], sizeof(double) * m->chi[b], cudaMemcpyDeviceToHost, m->stream));
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  return CTEBD_OK;
}

static int check_chi(const ctebd_mps* m, const int* chi) {
  if (chi[0] != 1 || chi[m->n] != 1) return fail(CTEBD_ERR_ARG, "mps_load: boundary bonds must be 1");
  for (int b = 0; b <= m->n; b++)
    if (chi[b] < 1 || chi[b] > m->lam_cap) return fail(CTEBD_ERR_ARG, "mps_load: chi out of range");
  return CTEBD_OK;
}

extern "C" int mps_load(ctebd_mps* m, const int* chi, const double* const* sites, const double* const* lams) {
  if (!m || !chi || !sites || !lams) return fail(CTEBD_ERR_ARG, "mps_load: null argument");
  TRY(check_chi(m, chi));
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  for (int q = 0; q < m->n; q++) {
    const long long n = (long long)chi[q] * 2 * chi[q + 1];
    TRY(ensure_site(m, q, (size_t)n));
    double* d = nullptr;
    CUDA_TRY(cudaMallocAsync(&d, sizeof(double) * 2 * n, m->stream));
    CUDA_TRY(cudaMemcpyAsync(d, sites[q], sizeof(double) * 2 * n, cudaMemcpyHostToDevice, m->stream));
    CUDA_TRY(m->fp64 ? launch_convert_from_c128<double>(d, m->site[q], n, m->stream)
                     : launch_convert_from_c128<float>(d, m->site[q], n, m->stream));
    CUDA_TRY(cudaFreeAsync(d, m->stream));
    CUDA_TRY(cudaStreamSynchronize(m->stream));
  }
  for (int b = 0; b <= m->n; b++)
    CUDA_TRY(cudaMemcpyAsync(m->lam[b], lams[b], sizeof(double) * chi[b], cudaMemcpyHostToDevice, m->stream));
  m->chi.assign(chi, chi + m->n + 1);
  m->logF = 0;
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  return CTEBD_OK;
}

extern "C" int mps_load_device(ctebd_mps* m, const int* chi, const void* const* sites, const double* const* lams) {
  if (!m || !chi || !sites || !lams) return fail(CTEBD_ERR_ARG, "mps_load_device: null argument");
  TRY(check_chi(m, chi));
  for (int q = 0; q < m->n; q++) {
    const size_t n = (size_t)chi[q] * 2 * chi[q + 1];
    TRY(ensure_site(m, q, n));
    CUDA_TRY(cudaMemcpyAsync(m->site[q], sites[q], n * m->esz, cudaMemcpyDeviceToDevice, m->stream));
  }
  for (int b = 0; b <= m->n; b++)
    CUDA_TRY(cudaMemcpyAsync(m->lam[b], lams[b], sizeof(double) * chi[b], cudaMemcpyDefault, m->stream));
  m->chi.assign(chi, chi + m->n + 1);
  m->logF = 0;
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  return CTEBD_OK;
}

extern "C" int mps_split_log(const ctebd_mps* m, double* rows, int cap, int* n_rows) {
  if (!m || !n_rows) return fail(CTEBD_ERR_ARG, "mps_split_log: null argument");
  const int nr = (int)(m->splitlog.size() / 8);
  *n_rows = nr;
  if (rows)
    for (int i = 0; i < std::min(nr, cap); i++) {
      std::memcpy(rows + 14 * i, m->splitlog.data() + 8 * i, sizeof(double) * 8);
      std::memcpy(rows + 14 * i + 8, m->splitlog2.data() + 6 * i, sizeof(double) * 6);
    }
  return CTEBD_OK;
}

extern "C" int mps_solver_stats(const ctebd_mps* m, double* out) {
  if (!m || !out) return fail(CTEBD_ERR_ARG, "mps_solver_stats: null argument");
  out[0] = m->solve_stats[0];
  out[1] = m->solve_stats[1];
  return CTEBD_OK;
}

extern "C" int mps_sketch_stats(const ctebd_mps* m, double* out) {
  if (!m || !out) return fail(CTEBD_ERR_ARG, "mps_sketch_stats: null argument");
  out[0] = m->sk_stats[0];
  out[1] = m->sk_stats[1];
  return CTEBD_OK;
}

// operator-Schmidt rank of a gate across a cut between its qubits
// ---------------------------------------------------------------------------
// Sec. III.B, Eqs. 9-11: the virtual MPS of a circuit section and the
// adaptive grouping of its sites by recursive min-cut bipartitioning.
// ---------------------------------------------------------------------------
extern "C" int virtual_mps_bonds(const ctebd_gate* gates, int n_gates, int n_qubits, int layer_start, int l_max,
                                 const int* chi, int chi_max, int* out, int* entangling) {
  if (!gates && n_gates > 0) return fail(CTEBD_ERR_ARG, "virtual_mps_bonds: null gates");
  if (n_qubits < 1 || !chi || !out || chi_max < 1 || layer_start < 0)
    return fail(CTEBD_ERR_ARG, "virtual_mps_bonds: bad arguments");
  std::vector<long long> E(n_qubits + 1, 0);
  const long long hi = l_max > 0 ? (long long)layer_start + l_max : (long long)1 << 60;
  for (int i = 0; i < n_gates; i++) {
    const ctebd_gate& g = gates[i];
    if (g.layer <= layer_start || g.layer > hi || g.n_q < 2) continue;
    int lo = g.q[0];
    for (int j = 1; j < g.n_q; j++) lo = std::min(lo, g.q[j]);
    if (lo < 0 || lo + g.n_q > n_qubits) return fail(CTEBD_ERR_ARG, "virtual_mps_bonds: gate out of range");
    for (int b = lo + 1; b < lo + g.n_q; b++) E[b] += 1;   // bonds the gate spans
  }
  for (int b = 0; b <= n_qubits; b++) {
    if (chi[b] < 1) return fail(CTEBD_ERR_ARG, "virtual_mps_bonds: chi < 1");
    // min(2^E chi_b, chi_max, 2^min(b, N-b)), saturating
    const int edge = std::min(b, n_qubits - b);
    long long v = chi_max;
    if (edge < 31) v = std::min<long long>(v, 1LL << edge);
    long long grown = chi[b];
    for (long long e = 0; e < E[b] && grown < v; e++) grown *= 2;
    out[b] = (int)std::min(v, grown);
    if (entangling) entangling[b] = (int)std::min<long long>(E[b], 1 << 30);
  }
  return CTEBD_OK;
}

// 2^size * chi_l * chi_r <= 2^q_max, exactly (Eq. 10 / Eq. 11 in log form)
static bool group_fits(int size, long long chi_l, long long chi_r, int q_max) {
  const int room = q_max - size;
  if (room < 0) return false;
  if (room >= 62) return true;
  return chi_l * chi_r <= (1LL << room);
}

extern "C" int adaptive_grouping(const int* chi_v, int n_qubits, int q_max, double imbalance, int* group_start,
                                 int cap, int* n_groups) {
  if (!chi_v || n_qubits < 1 || !group_start || !n_groups || cap < 1 || !(imbalance >= 0.0))
    return fail(CTEBD_ERR_ARG, "adaptive_grouping: bad arguments");
  for (int b = 0; b <= n_qubits; b++)
    if (chi_v[b] < 1) return fail(CTEBD_ERR_ARG, "adaptive_grouping: bond dimension < 1");
  // segments [lo, hi) of qubits, bounded by bonds lo and hi (the chain ends count as 1)
  auto bond = [&](int b) -> long long { return (b == 0 || b == n_qubits) ? 1 : chi_v[b]; };
  std::vector<std::pair<int, int>> stack = {{0, n_qubits}};
  int count = 0;
  while (!stack.empty()) {
    const auto [lo, hi] = stack.back();
    stack.pop_back();
    const int size = hi - lo;
    if (group_fits(size, bond(lo), bond(hi), q_max)) {
      if (count >= cap) return fail(CTEBD_ERR_ARG, "adaptive_grouping: cap too small");
      group_start[count++] = lo;
      continue;
    }
    if (size == 1)
      return fail(CTEBD_ERR_STATE, "adaptive_grouping: site " + std::to_string(lo) +
                                       " does not fit Q_max with its bonds");
    // balanced min-cut: parts no larger than (1 + imbalance) * ceil(size / 2)
    const long long cap_part = (long long)std::floor((1.0 + imbalance) * ((size + 1) / 2) + 1e-9);
    int best = -1;
    for (int k = lo + 1; k < hi; k++) {
      if (k - lo > cap_part || hi - k > cap_part) continue;
      if (best < 0) { best = k; continue; }
      const long long a = bond(k), b = bond(best);
      const int dk = std::abs(2 * k - (lo + hi)), db = std::abs(2 * best - (lo + hi));
      if (a < b || (a == b && dk < db)) best = k;
    }
    stack.push_back({best, hi});   // right part after the left one
    stack.push_back({lo, best});
  }
  *n_groups = count;
  return CTEBD_OK;
}

static int gate_osr(int kind, int n_q) {
  if (n_q >= 3) return 4;
  if (kind == CTEBD_SWAP || kind == CTEBD_SQSWAP) return 4;
  return 2;
}

extern "C" int cluster_rank_bounds(const ctebd_gate* gates, int n_gates, const ctebd_cluster* c,
                                   const int* chi, int* out) {
  if (!c || !chi || !out || c->k < 2 || c->k > 12 || n_gates < 0 || (n_gates && !gates))
    return fail(CTEBD_ERR_ARG, "cluster_rank_bounds: bad args");
  const int k = c->k, q0 = c->q0;
  const long long cap = 1LL << 30;
  std::vector<long long> prod(k, 1);
  for (int j = 1; j < k; j++) prod[j] = chi[q0 + j];
  for (int i = 0; i < n_gates; i++) {
    const ctebd_gate& g = gates[i];
    if (g.layer <= c->layer_lo || g.layer > c->layer_hi || g.n_q < 2) continue;
    int lo = g.q[0], hi = g.q[0];
    for (int t = 1; t < g.n_q; t++) { lo = std::min(lo, g.q[t]); hi = std::max(hi, g.q[t]); }
    if (lo < q0 || hi >= q0 + k) continue;
    for (int b = lo + 1; b <= hi; b++) prod[b - q0] = std::min(cap, prod[b - q0] * gate_osr(g.kind, g.n_q));
  }
  for (int j = 1; j < k; j++) {
    long long r = prod[j];
    r = std::min(r, std::min(cap, (long long)chi[q0] << j));
    r = std::min(r, std::min(cap, ((long long)1 << (k - j)) * chi[q0 + k]));
    out[j - 1] = (int)r;
  }
  return CTEBD_OK;
}

extern "C" int ctebd_profile(ctebd_mps* m, int mode) {
  if (!m) return fail(CTEBD_ERR_ARG, "ctebd_profile: null");
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  m->prof.drain();
  m->prof.reset();
  m->prof.on = mode != 0;
  return CTEBD_OK;
}

extern "C" int ctebd_profile_read(ctebd_mps* m, double* rows, int cap, int* n_kinds) {
  if (!m || !n_kinds) return fail(CTEBD_ERR_ARG, "ctebd_profile_read: null");
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  m->prof.drain();
  *n_kinds = KK_COUNT;
  for (int k = 0; k < KK_COUNT && k < cap && rows; k++) {
    rows[5 * k + 0] = m->prof.launches[k];
    rows[5 * k + 1] = m->prof.ms[k];
    rows[5 * k + 2] = m->prof.flops[k];
    rows[5 * k + 3] = m->prof.bytes[k];
    rows[5 * k + 4] = m->prof.tc[k];
  }
  return CTEBD_OK;
}

extern "C" int ctebd_measure_fma(int repeats, double* tflops_best, double* tflops_mean, int* n_sm) {
  if (repeats < 1 || !tflops_best || !tflops_mean || !n_sm) return fail(CTEBD_ERR_ARG, "ctebd_measure_fma: bad args");
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  float* out = nullptr;
  int rc = CTEBD_OK;
  const int blocks = 4 * sms, iters = 1 << 19;
  double best = 0, sum = 0;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
      cudaEventCreate(&b) != cudaSuccess || cudaMalloc(&out, sizeof(float) * blocks * 256) != cudaSuccess) {
    rc = fail(CTEBD_ERR_CUDA, "ctebd_measure_fma: setup");
  }
  for (int r = -1; r < repeats && rc == CTEBD_OK; r++) {   // r = -1: warm-up
    cudaEventRecord(a, s);
    if (launch_fma_peak(out, blocks, iters, s) != cudaSuccess) { rc = fail(CTEBD_ERR_CUDA, "fma probe launch"); break; }
    cudaEventRecord(b, s);
    if (cudaEventSynchronize(b) != cudaSuccess) { rc = fail(CTEBD_ERR_CUDA, "fma probe"); break; }
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    const double tf = 2.0 * 8.0 * iters * (double)blocks * 256 / (ms * 1e-3) / 1e12;
    if (r >= 0) { best = std::max(best, tf); sum += tf; }
  }
  if (out) cudaFree(out);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (s) cudaStreamDestroy(s);
  if (rc != CTEBD_OK) return rc;
  *tflops_best = best;
  *tflops_mean = sum / repeats;
  *n_sm = sms;
  return CTEBD_OK;
}

extern "C" int ctebd_kernel_name(int kind, char* buf, size_t n) {
  if (kind < 0 || kind >= KK_COUNT || !buf || !n) return fail(CTEBD_ERR_ARG, "ctebd_kernel_name: bad kind");
  std::snprintf(buf, n, "%s", kKindNames[kind]);
  return CTEBD_OK;
}

// ---------------------------------------------------------------------------
// Learned rank predictor (sizes the sketched split; not in the paper)
// ---------------------------------------------------------------------------
static bool is_nonclifford(int kind) {
  return kind == CTEBD_T || kind == CTEBD_P || kind == CTEBD_X14 || kind == CTEBD_SQW || kind == CTEBD_CH ||
         kind == CTEBD_CS || kind == CTEBD_CT || kind == CTEBD_SQSWAP || kind == CTEBD_CP;
}

extern "C" int rank_features(const ctebd_gate* gates, int n_gates, const ctebd_cluster* c, const int* chi,
                             const double* entropy, const ctebd_config* cfg, float* out) {
  if (!c || !chi || !entropy || !cfg || !out || c->k < 2 || c->k > 12 || n_gates < 0 || (n_gates && !gates))
    return fail(CTEBD_ERR_ARG, "rank_features: bad args");
  const int k = c->k, q0 = c->q0;
  std::vector<int> bound(k - 1);
  TRY(cluster_rank_bounds(gates, n_gates, c, chi, bound.data()));
  std::vector<int> cross(k, 0);
  int n2 = 0, nc1 = 0, nc2 = 0;
  for (int i = 0; i < n_gates; i++) {
    const ctebd_gate& g = gates[i];
    if (g.layer <= c->layer_lo || g.layer > c->layer_hi) continue;
    int lo = g.q[0], hi = g.q[0];
    for (int t = 1; t < g.n_q; t++) { lo = std::min(lo, g.q[t]); hi = std::max(hi, g.q[t]); }
    if (lo < q0 || hi >= q0 + k) continue;
    if (g.n_q >= 2) {
      n2++;
      if (is_nonclifford(g.kind)) nc2++;
      for (int b = lo + 1; b <= hi; b++) cross[b - q0]++;
    } else if (is_nonclifford(g.kind)) {
      nc1++;
    }
  }
  auto lg = [](double x) { return (float)std::log2(std::max(x, 1.0)); };
  for (int j = 1; j < k; j++) {
    float* f = out + (size_t)(j - 1) * MLP_F;
    f[0] = (float)k / 10.f;
    f[1] = (float)j / (float)k;
    f[2] = lg(chi[q0]) / 10.f;
    f[3] = lg(chi[q0 + k]) / 10.f;
    f[4] = lg(chi[q0 + j]) / 10.f;
    f[5] = lg((double)chi[q0] * (1 << j)) / 10.f;
    f[6] = lg((double)chi[q0 + k] * (1 << (k - j))) / 10.f;
    f[7] = lg(bound[j - 1]) / 10.f;
    f[8] = (float)cross[j] / 10.f;
    f[9] = (float)n2 / 10.f;
    f[10] = (float)nc1 / 10.f;
    f[11] = (float)nc2 / 10.f;
    f[12] = (float)(c->layer_hi - c->layer_lo) / 10.f;
    f[13] = (float)entropy[q0 + j] / 10.f;
    f[14] = (float)entropy[q0] / 10.f;
    f[15] = cfg->cutoff > 0 ? (float)(-std::log10(cfg->cutoff) / 10.0) : 0.f;
  }
  return CTEBD_OK;
}

extern "C" int mps_bond_entropies(ctebd_mps* m, double* out) {
  if (!m || !out) return fail(CTEBD_ERR_ARG, "mps_bond_entropies: null argument");
  const int nb = m->n + 1;
  double* d = nullptr;
  CUDA_TRY(cudaMallocAsync(&d, sizeof(double) * nb, m->stream));
  const double* const* dl; const int* dc;
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  m->stage.reset();
  std::vector<const double*> lp(m->lam.begin(), m->lam.end());
  TRY(m->stage.push(lp.data(), lp.size(), (const double* const**)&dl));
  TRY(m->stage.push(m->chi.data(), nb, &dc));
  CUDA_TRY(launch_entropy(dl, dc, nb, d, m->stream));
  CUDA_TRY(cudaMemcpyAsync(out, d, sizeof(double) * nb, cudaMemcpyDeviceToHost, m->stream));
  CUDA_TRY(cudaFreeAsync(d, m->stream));
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  return CTEBD_OK;
}

extern "C" int rank_model_load(ctebd_mps* m, const float* weights, size_t n) {
  if (!m || !weights) return fail(CTEBD_ERR_ARG, "rank_model_load: null argument");
  if (n != (size_t)mlp_nparams())
    return fail(CTEBD_ERR_ARG, "rank_model_load: expected " + std::to_string(mlp_nparams()) + " parameters");
  if (!m->mlp) CUDA_TRY(cudaMalloc(&m->mlp, sizeof(float) * n));
  CUDA_TRY(cudaMemcpyAsync(m->mlp, weights, sizeof(float) * n, cudaMemcpyHostToDevice, m->stream));
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  return CTEBD_OK;
}

// hints_out[i] = ceil(bounds[i] * 2^(-b/2)) for the predicted bucket b (the
// upper edge of the bucket: ratio r / bound in (2^-(b+1)/2, 2^-b/2])
extern "C" int rank_model_predict(ctebd_mps* m, const float* features, int B, const int* bounds, int* hints_out) {
  if (!m || B < 0 || (B && (!features || !bounds || !hints_out))) return fail(CTEBD_ERR_ARG, "rank_model_predict: bad args");
  if (!m->mlp) return fail(CTEBD_ERR_STATE, "rank_model_predict: no model loaded");
  if (B == 0) return CTEBD_OK;
  float *dX = nullptr, *dL = nullptr;
  CUDA_TRY(cudaMallocAsync(&dX, sizeof(float) * B * MLP_F, m->stream));
  CUDA_TRY(cudaMallocAsync(&dL, sizeof(float) * B * MLP_NB, m->stream));
  CUDA_TRY(cudaMemcpyAsync(dX, features, sizeof(float) * B * MLP_F, cudaMemcpyHostToDevice, m->stream));
  {
    ProfScope ps(m->prof, m->stream, KK_MLP, 2.0 * B * (MLP_F * MLP_H1 + MLP_H1 * MLP_H2 + MLP_H2 * MLP_NB), 0);
    CUDA_TRY(launch_mlp_forward(m->mlp, dX, B, dL, m->stream));
  }
  std::vector<float> lo((size_t)B * MLP_NB);
  CUDA_TRY(cudaMemcpyAsync(lo.data(), dL, sizeof(float) * lo.size(), cudaMemcpyDeviceToHost, m->stream));
  CUDA_TRY(cudaFreeAsync(dX, m->stream));
  CUDA_TRY(cudaFreeAsync(dL, m->stream));
  CUDA_TRY(cudaStreamSynchronize(m->stream));
  for (int i = 0; i < B; i++) {
    int best = 0;
    for (int b = 1; b < MLP_NB; b++) if (lo[(size_t)i * MLP_NB + b] > lo[(size_t)i * MLP_NB + best]) best = b;
    hints_out[i] = std::max(1, (int)std::ceil(bounds[i] * std::pow(2.0, -0.5 * best)));
  }
  return CTEBD_OK;
}

// training entry points on caller-owned device buffers (FP32)
extern "C" int mlp_nparams_abi(void) { return mlp_nparams(); }

extern "C" int mlp_forward(const float* params, const float* X, int B, float* logits, void* stream) {
  if (!params || !X || !logits || B < 0) return fail(CTEBD_ERR_ARG, "mlp_forward: bad args");
  CUDA_TRY(launch_mlp_forward(params, X, B, logits, (cudaStream_t)stream));
  return CTEBD_OK;
}

extern "C" int mlp_loss_grad(const float* params, const float* X, const int* y, int B, float* grad, float* loss,
                             void* stream) {
  if (!params || !X || !y || !grad || !loss || B < 0) return fail(CTEBD_ERR_ARG, "mlp_loss_grad: bad args");
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaMemsetAsync(grad, 0, sizeof(float) * mlp_nparams(), s));
  CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), s));
  CUDA_TRY(launch_mlp_loss_grad(params, X, y, B, grad, loss, s));
  return CTEBD_OK;
}

extern "C" int mlp_adam(float* params, const float* grad, float* m1, float* m2, int n, float lr, int t, void* stream) {
  if (!params || !grad || !m1 || !m2 || n != mlp_nparams() || t < 1) return fail(CTEBD_ERR_ARG, "mlp_adam: bad args");
  CUDA_TRY(launch_adam(params, grad, m1, m2, n, lr, t, (cudaStream_t)stream));
  return CTEBD_OK;
}

// C (M x N) = A (M x K) B (K x N), complex64 row-major device buffers, on the
// tensor cores (3xTF32, packed operands), any sizes.  Used to validate the
// tile engine against a reference product.
extern "C" int tc_cgemm(const void* A, const void* B, void* C, int M, int K, int N, void* stream) {
  if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0) return fail(CTEBD_ERR_ARG, "tc_cgemm: bad args");
  cudaStream_t s = (cudaStream_t)stream;
  PackedProb q{};
  GemmProb& g = q.g;
  g.M = M; g.N = N; g.K = K; g.batch = 1;
  g.A = A; g.lda = K; g.B = B; g.ldb = N; g.C = C; g.ldc = N; g.alpha = 1.0;
  tc_packed_shape(g, q.tilesM, q.tilesN, q.chunks);
  const size_t pbytes = tc_packed_bytes(g);
  const long long off[4] = {0, tc_packed_pack_blocks(g), 0, tc_packed_tiles(g)};
  unsigned char* buf = nullptr;
  const size_t head = 1024;   // err flag, descriptor, offsets
  CUDA_TRY(cudaMallocAsync((void**)&buf, head + pbytes, s));
  q.pa = reinterpret_cast<float*>(buf + head);
  q.pb = reinterpret_cast<float*>(buf + head + tc_packed_a_bytes(g));
  int* err = reinterpret_cast<int*>(buf);
  static_assert(sizeof(PackedProb) <= 512, "tc_cgemm: descriptor slot");
  PackedProb* dq = reinterpret_cast<PackedProb*>(buf + 256);
  long long* doff = reinterpret_cast<long long*>(buf + 768);
  CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  CUDA_TRY(cudaMemcpyAsync(dq, &q, sizeof(q), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(doff, off, sizeof(off), cudaMemcpyHostToDevice, s));
  CUDA_TRY(launch_tc_packed(dq, doff, doff + 2, 1, off[1], off[3], err, s));
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaFreeAsync(buf, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (h) return fail(CTEBD_ERR_TIMEOUT, "tc_cgemm: tensor-core completion wait timed out");
  return CTEBD_OK;
}
