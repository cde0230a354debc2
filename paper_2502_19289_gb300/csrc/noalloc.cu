// noalloc.cu -- split2_noalloc: the two-site truncated split without any
// device allocation.
//
// Some callers cannot allocate device memory while they run: a host that owns
// every byte of device memory through its own pool, a plugin loaded into a
// process that forbids cudaMalloc/cudaFree on its hot path (both can
// synchronise the device and stall other streams), or a caller that has
// already handed all free memory to another component.  This entry point does
// the same work as apply_cluster + truncate_split for k = 2 but uses only the
// caller's input/output buffers plus one fixed scratch area that lives in this
// library's file-scope device array.  It never calls cudaMalloc, cudaFree,
// cudaMallocAsync or any allocating library routine.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ctebd.h"
#include "internal.h"

namespace ctebd {

// Limits of the static variant: both outer bonds <= 128, so the split matrix
// is at most 256 x 256 (complex64).
constexpr int NA_CHI = 128;
constexpr int NA_M = 2 * NA_CHI;          // rows of the split matrix
constexpr int NA_N = 2 * NA_CHI;          // columns of the split matrix
constexpr int NA_JB = 32;                 // FP32 Jacobi block (must match kernels.cu)
constexpr size_t NA_CPLX = 8;             // complex64
constexpr size_t al256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t NA_OFF_MBAR = 0;
constexpr size_t NA_OFF_RFULL = NA_OFF_MBAR + al256((size_t)NA_M * NA_N * NA_CPLX);
constexpr size_t NA_OFF_G = NA_OFF_RFULL + al256((size_t)NA_M * NA_N * NA_CPLX);
constexpr size_t NA_OFF_V = NA_OFF_G + al256((size_t)NA_N * NA_N * NA_CPLX);
constexpr size_t NA_OFF_W = NA_OFF_V + al256((size_t)NA_N * NA_N * NA_CPLX);
constexpr size_t NA_OFF_J = NA_OFF_W + al256((size_t)NA_N * NA_N * NA_CPLX);
constexpr size_t NA_OFF_RHO = NA_OFF_J + al256((size_t)NA_N * 2 * NA_JB * NA_CPLX);
constexpr size_t NA_OFF_PERM = NA_OFF_RHO + al256(2 * NA_N * sizeof(double));   // rho, then |v_i|^2
constexpr size_t NA_OFF_RES = NA_OFF_PERM + al256(NA_N * sizeof(int));
constexpr size_t NA_OFF_CNT = NA_OFF_RES + al256(8 * sizeof(double));
constexpr int NA_SLOTS = NA_N / (2 * NA_JB);   // pair slots of the largest eigenproblem
constexpr size_t NA_OFF_DESC = NA_OFF_CNT + al256((8 + NA_SLOTS) * sizeof(double));
constexpr size_t NA_DESC_BYTES = 4096;
constexpr size_t NA_BYTES = NA_OFF_DESC + NA_DESC_BYTES;   // ~2.4 MiB

// The scratch area: every GPU that loads this library holds it until exit.
static __device__ __align__(256) unsigned char g_na_scratch[NA_BYTES];

static std::mutex g_na_mu;
static void* g_na_ptr[64] = {nullptr};

static int na_fail(int code, const std::string& m) {
  set_last_error(m);   // shared with ctebd_last_error()
  return code;
}

// Device address of the scratch array for the current device (resolved once
// per device, with that device current).
static int na_scratch(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return na_fail(CTEBD_ERR_CUDA, "split2_noalloc: no current CUDA device");
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    if (e != cudaSuccess || !p)
      return na_fail(CTEBD_ERR_CUDA, std::string("split2_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_na_ptr[dev] = p;
  }
  *out = (unsigned char*)g_na_ptr[dev];
  return CTEBD_OK;
}

#define NA_CUDA(call)                                                                         \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return na_fail(CTEBD_ERR_CUDA, std::string("split2_noalloc: ") + #call + ": " + cudaGetErrorString(e_)); \
  } while (0)

// host -> scratch descriptor copy from pageable memory (staged by the driver)
struct NaDesc {
  unsigned char* base;
  size_t off = 0;
  cudaStream_t s;
  template <typename T>
  int put(const T* src, size_t count, const T** dst) {
    const size_t bytes = sizeof(T) * count, need = al256(bytes);
    if (off + need > NA_DESC_BYTES) return na_fail(CTEBD_ERR_ARG, "split2_noalloc: descriptor area full");
    NA_CUDA(cudaMemcpyAsync(base + off, src, bytes, cudaMemcpyHostToDevice, s));
    *dst = reinterpret_cast<const T*>(base + off);
    off += need;
    return CTEBD_OK;
  }
};

static int na_gemm(NaDesc& d, const GemmProb& p) {
  const GemmProb* dp;
  const long long off[2] = {0, gemm_tiles(p, false)};
  const long long* doff;
  int rc = d.put(&p, 1, &dp);
  if (!rc) rc = d.put(off, 2, &doff);
  if (rc) return rc;
  NA_CUDA(launch_gemm<float>(dp, doff, 1, off[1], d.s));
  return CTEBD_OK;
}

// Block-Jacobi on G (npad x npad) accumulating into acc; same kernels and
// stopping rule as the handle path.
static int na_eig(NaDesc& d, unsigned char* S, void* acc, int npad, double floor_factor,
                  double rel_skip, double move_rel, double move_tol) {
  // [0] significant rotations, [1] all rotations, [2] applied flops (the
  // kernels' third counter, unused without pair flags), [4] trace of G,
  // [8 ..) the weight moved by each pair slot's significant rotations
  double* cnt = (double*)(S + NA_OFF_CNT);
  EigProb e{};
  e.G = S + NA_OFF_G; e.V = acc; e.J = S + NA_OFF_J;
  e.npad = npad; e.nb = npad / NA_JB; e.active = 1;
  e.off = cnt; e.scale = cnt + 4; e.floor_factor = floor_factor;
  e.rel_skip = rel_skip;   // no pair flags: every tile is updated
  e.move_rel = move_rel;
  e.move_tol = move_tol;
  e.mv = move_tol > 0 ? cnt + 8 : nullptr;
  const EigProb* de;
  const size_t mark = d.off;
  if (int rc = d.put(&e, 1, &de)) return rc;
  NA_CUDA(launch_eig_init<float>(de, 1, npad, d.s));
  NA_CUDA(launch_eig_trace<float>(de, 1, d.s));
  const int max_sweeps = max_jacobi_sweeps();
  bool converged = false;
  for (int sweep = 0; sweep < max_sweeps && !converged; sweep++) {
    NA_CUDA(cudaMemsetAsync(cnt, 0, 4 * sizeof(double), d.s));
    NA_CUDA(cudaMemsetAsync(cnt + 8, 0, NA_SLOTS * sizeof(double), d.s));
    for (int t = 0; t < e.nb - 1; t++) {
      NA_CUDA(launch_eig_inner<float>(de, 1, e.nb, t, d.s));
      NA_CUDA(launch_eig_apply<float>(de, 1, e.nb, t, d.s));
    }
    double h[8 + NA_SLOTS] = {};
    NA_CUDA(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, d.s));
    NA_CUDA(cudaStreamSynchronize(d.s));
    for (int k = 0; k < e.nb / 2; k++) h[3] += h[8 + k];   // moved weight, in slot order
    converged = h[0] == 0.0 || (move_tol > 0 && h[3] <= move_tol * h[4]);
    // a refinement pass still moving at most 1e-8 of the trace at the cap is
    // accepted, as on the handle path
    if (!converged && move_tol > 0 && sweep == max_sweeps - 1 && h[3] <= 1e-8 * h[4]) converged = true;
  }
  d.off = mark;
  if (!converged)
    return na_fail(CTEBD_ERR_NUMERIC, "split2_noalloc: Jacobi eigen-solve still rotating after " +
                                          std::to_string(max_sweeps) + " sweeps");
  return CTEBD_OK;
}

// Rfull = Mbar V and its weighted column norms rho (the select follows)
static int na_project(NaDesc& d, unsigned char* S, const void* V, int m, int n, int npad,
                      const double* lamL) {
  GemmProb p{};
  p.M = m; p.N = n; p.K = n; p.batch = 1;
  p.A = S + NA_OFF_MBAR; p.lda = n; p.opA = 0;
  p.B = V; p.ldb = npad; p.opB = 0;
  p.C = S + NA_OFF_RFULL; p.ldc = n; p.alpha = 1.0;
  if (int rc = na_gemm(d, p)) return rc;
  // rho (weighted column norms of Rfull) and |v_i|^2 (column norms of V),
  // then rho_i / |v_i|^2 as the handle path does
  double* rho = (double*)(S + NA_OFF_RHO);
  NA_CUDA(cudaMemsetAsync(rho, 0, sizeof(double) * 2 * NA_N, d.s));
  const void* R[2] = {S + NA_OFF_RFULL, V};
  const int ms[2] = {m, n}, ns[2] = {n, n}, shs[2] = {1, 0}, lds[2] = {n, npad};
  const double* lams[2] = {lamL, nullptr};
  double* rhos[2] = {rho, rho + NA_N};
  const void* const* dR; const int *dm, *dn, *dsh, *dld; const double* const* dL; double* const* drho;
  if (int rc = d.put(R, 2, (const void* const**)&dR)) return rc;
  if (int rc = d.put(ms, 2, &dm)) return rc;
  if (int rc = d.put(ns, 2, &dn)) return rc;
  if (int rc = d.put(shs, 2, &dsh)) return rc;
  if (int rc = d.put(lds, 2, &dld)) return rc;
  if (int rc = d.put(lams, 2, (const double* const**)&dL)) return rc;
  if (int rc = d.put(rhos, 2, (double* const**)&drho)) return rc;
  NA_CUDA(launch_colnorm_batch<float>(dR, dm, dn, dld, dL, dsh, drho, 2, n, std::max(m, n), d.s));
  NA_CUDA(launch_rho_normalize(drho, drho + 1, dn, 1, n, d.s));
  return CTEBD_OK;
}

}  // namespace ctebd

using namespace ctebd;

extern "C" int split2_noalloc(const void* theta, const double* lam_l, int chi_l, int chi_r, int chi_max,
                              double cutoff, void* site_l_out, void* site_r_out, double* lam_out,
                              int* r_out, double* f_out, void* cuda_stream) {
  if (!theta || !lam_l || !site_l_out || !site_r_out || !lam_out || !r_out || !f_out)
    return na_fail(CTEBD_ERR_ARG, "split2_noalloc: null argument");
  if (chi_l < 1 || chi_r < 1 || chi_l > NA_CHI || chi_r > NA_CHI)
    return na_fail(CTEBD_ERR_ARG, "split2_noalloc: chi_l and chi_r must be in [1, " +
                                      std::to_string(NA_CHI) + "] (static scratch limit)");
  if (chi_max < 1 || !(cutoff >= 0.0) || cutoff >= 1.0)
    return na_fail(CTEBD_ERR_ARG, "split2_noalloc: chi_max >= 1 and 0 <= cutoff < 1 required");
  unsigned char* S = nullptr;
  if (int rc = na_scratch(&S)) return rc;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int m = 2 * chi_l, n = 2 * chi_r;
  const int npad = (n + 2 * NA_JB - 1) / (2 * NA_JB) * (2 * NA_JB);
  NaDesc d{S + NA_OFF_DESC, 0, s};
  // Mbar: copy of theta viewed (chi_l * 2) x (2 * chi_r)
  NA_CUDA(cudaMemcpyAsync(S + NA_OFF_MBAR, theta, (size_t)m * n * NA_CPLX, cudaMemcpyDeviceToDevice, s));
  // pass 1: Gram of Mbar weighted by lambda_l^2 (row a of theta carries lambda_l[a])
  NA_CUDA(cudaMemsetAsync(S + NA_OFF_G, 0, (size_t)npad * npad * NA_CPLX, s));
  {
    GemmProb p{};
    p.M = n; p.N = n; p.K = m; p.batch = 1;
    p.A = S + NA_OFF_MBAR; p.lda = n; p.opA = 1;
    p.B = S + NA_OFF_MBAR; p.ldb = n; p.opB = 0;
    p.C = S + NA_OFF_G; p.ldc = npad;
    p.kw = lam_l; p.kw_shift = 1; p.alpha = 1.0;
    if (int rc = na_gemm(d, p)) return rc;
  }
  void* V = S + NA_OFF_V;
  if (int rc = na_eig(d, S, V, npad, 1.0, 4.0, 0.0, 0.0)) return rc;
  double res[8];
  auto select = [&](const void* Vc) -> int {
    if (int rc = na_project(d, S, Vc, m, n, npad, lam_l)) return rc;
    SelProb sp{};
    sp.rho = (double*)(S + NA_OFF_RHO); sp.n = n; sp.perm = (int*)(S + NA_OFF_PERM);
    sp.lam_out = lam_out; sp.res = (double*)(S + NA_OFF_RES);
    sp.rank_cap = std::min(m, n);   // lam_out and site_l_out hold at most min(chi_max, m, n)
    const SelProb* dsp;
    if (int rc = d.put(&sp, 1, &dsp)) return rc;
    // same truncation parameters as the handle path's FP32 split
    const double eps32 = 1.1920928955078125e-07;
    NA_CUDA(launch_select(dsp, 1, chi_max, cutoff, 16.0 * eps32, 1024.0 * eps32, 1e-12, s));
    NA_CUDA(cudaMemcpyAsync(res, S + NA_OFF_RES, sizeof(res), cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    d.off = 0;
    return CTEBD_OK;
  };
  if (int rc = select(V)) return rc;
  // pass 2 wherever something is discarded, or a cutoff is set and pass 1 left
  // unresolved directions (relative thresholds and the moved-weight stopping
  // rule of the handle path)
  if ((int)res[0] < n || (cutoff > 0 && (int)res[6] < n)) {
    NA_CUDA(cudaMemsetAsync(S + NA_OFF_G, 0, (size_t)npad * npad * NA_CPLX, s));
    GemmProb p{};
    p.M = n; p.N = n; p.K = m; p.batch = 1;
    p.A = S + NA_OFF_RFULL; p.lda = n; p.opA = 1;
    p.B = S + NA_OFF_RFULL; p.ldb = n; p.opB = 0;
    p.C = S + NA_OFF_G; p.ldc = npad;
    p.kw = lam_l; p.kw_shift = 1; p.alpha = 1.0;
    if (int rc = na_gemm(d, p)) return rc;
    const double move_tol = cutoff > 0 ? std::min(1e-10, 1e-2 * cutoff) : 1e-10;
    if (int rc = na_eig(d, S, S + NA_OFF_W, npad, 1e-12, 32.0, 1e-13, move_tol)) return rc;
    GemmProb q{};
    q.M = n; q.N = n; q.K = n; q.batch = 1;
    q.A = V; q.lda = npad; q.opA = 0;
    q.B = S + NA_OFF_W; q.ldb = npad; q.opB = 0;
    q.C = S + NA_OFF_G; q.ldc = npad; q.alpha = 1.0;
    if (int rc = na_gemm(d, q)) return rc;
    V = S + NA_OFF_G;
    if (int rc = select(V)) return rc;
  }
  const int r = (int)res[0];
  const double kept = res[3];
  if (!(kept > 0) || r < 1 || r > n || r > m || r > chi_max)
    return na_fail(CTEBD_ERR_NUMERIC, "split2_noalloc: zero weight or rank out of range");
  GatherProb g[2] = {};
  g[0].src = V; g[0].dst = site_r_out; g[0].perm = (int*)(S + NA_OFF_PERM);
  g[0].rows = n; g[0].r = r; g[0].ld = npad; g[0].mode = 0;
  g[0].cs = (const double*)(S + NA_OFF_RHO) + NA_N;
  g[1].src = S + NA_OFF_RFULL; g[1].dst = site_l_out; g[1].perm = (int*)(S + NA_OFF_PERM);
  g[1].rows = m; g[1].r = r; g[1].ld = n; g[1].mode = 1; g[1].scale = 1.0 / std::sqrt(kept);
  g[1].cs = g[0].cs;
  const GatherProb* dg;
  if (int rc = d.put(g, 2, &dg)) return rc;
  NA_CUDA(launch_gather<float>(dg, 2, (long long)std::max(m, n) * r, s));
  NA_CUDA(cudaStreamSynchronize(s));
  *r_out = r;
  *f_out = res[1];
  return CTEBD_OK;
}
