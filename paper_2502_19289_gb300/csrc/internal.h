// internal.h -- declarations shared by the host orchestration (host.cpp) and
// the CUDA kernels (kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>

namespace ctebd {

// One complex GEMM of a grouped launch, interleaved complex of real type R:
//   C[b] (M x N) = alpha * op(A[b]) (M x K) * op(B[b]) (K x N)
// op = 0: X[r][c] = X[r*ld + c];  op = 1: X[r][c] = conj(X[c*ld + r]).
// kw (optional): real weights; column k of op(A) is multiplied by
// kw[k >> kw_shift]^2 (the Schmidt-weighted Gram matrix M^H diag(lambda^2) M).
struct GemmProb {
  int M, N, K, batch;
  long long sA, sB, sC;  // batch strides in complex elements
  const void* A;
  const void* B;
  void* C;
  int lda, ldb, ldc;
  int opA, opB;
  const double* kw;
  int kw_shift;
  double alpha;
  int kw_pow;   // 1: multiply by kw; otherwise by kw^2
};

// One Hermitian eigenproblem of the batched block-Jacobi solver.  G and V are
// row-major npad x npad (npad = nb * JB), G Hermitian (zero padded), V
// accumulates the rotations (starts as identity).  J holds nb/2 unitary
// blocks of (2 JB)^2 for the current round.
struct EigProb {
  void* G;
  void* V;
  void* J;
  int npad;
  int nb;       // number of JB-blocks, even
  int active;   // 0: converged, skip
  double* off;         // [0] significant rotations this sweep, [1] all rotations,
                       // [2] flops of the tile updates actually applied (when jflag set)
  const double* scale; // trace of G (noise floor of the rotations)
  double floor_factor; // absolute rotation floor = eps * trace * floor_factor
  int* jflag;          // per pair slot: 1 when its J_p is not the identity; null: always apply
  double rel_skip;     // relative rotation floor in units of eps (0: 4)
  double move_rel;     // > 0: a rotation keeps the sweeps going only if it moves more
                       // than move_rel * trace of weight between its two directions
  int cut_lo, cut_hi;  // cut_hi > 0: columns sorted by weight, [0, cut_lo) kept and
                       // [cut_hi, npad) discarded for sure; rotations inside either
                       // set are skipped (they move no weight across the cut)
  void* T;             // npad x npad scratch of the tensor-core round update (FP32)
  double move_tol;     // > 0: the solve also ends after a sweep whose significant
                       // rotations moved at most move_tol * trace of weight in all
  double* mv;          // move_tol > 0: per pair slot, the weight its significant
                       // rotations moved this sweep (sum |t g|); summed in slot order
  int nact;            // > 0: the eigen-dimension (rows / columns past it are zero); a
                       // problem of one block pair then pairs only its first nact
                       // (rounded up to even) indices; 0: all 2 JB
};

// Per-problem truncation inputs/outputs of one split level.
struct SelProb {
  const double* rho;   // n weighted column norms
  int n;
  int* perm;           // out: kept column indices, descending rho
  double* lam_out;     // out: renormalised kept spectrum (fp64)
  double* res;         // out: [0] r, [1] f, [2] W, [3] kept, [4] rank before chi_max cap,
                       // [5] weight inside the n directions, [6] first index whose weight
                       // is within band * W of the smallest kept weight or below
                       // resolved * W, [7] first index below that band; perm receives
                       // the full descending order
  const double* W_ext; // optional total weight ||M||_F^2 (sketched split): the
                       // weight outside the n directions counts as discarded
  int rank_cap;        // > 0: the rank of the split matrix is at most rank_cap (its
                       // row count): no more directions than that are kept
};

// theta'[a, s', b] = sum_s U[s', s] theta[a, s, b] for every (a, b) column,
// theta row-major (chiL, D, chiR), U row-major D x D in the run precision.
struct ApplyUProb {
  const void* U;
  const void* src;
  void* dst;
  int chiL, chiR, D;   // D <= 16
};

// Column permutation (mode 0: dst[r][c] = src[r][perm[c]], r < rows, c < cols)
// or symmetric permutation of a padded square matrix (mode 1: dst[i][j] =
// src[perm[i]][perm[j]] for i, j < cols, zero elsewhere up to rows = npad).
struct PermProb {
  const void* src;
  void* dst;
  const int* perm;
  int rows, cols, lds, ldd, mode;
};

struct RowScaleProb {   // X[r][c] *= lam[r >> shift]
  void* X;
  int rows, cols, ld;
  const double* lam;
  int shift;
};

struct CholProb {       // X = (chol(G + s I))^{-H}, s = shift_rel * trace(G)
  const void* G;
  int ldg, l;
  double shift_rel;
  void* X;
  int ldx;
  double2* work;        // 2 l^2 complex128
  int* status;
  double dead_rel;      // pivots below dead_rel * trace drop their column (0: never)
  int* dead;            // l flags (scratch)
};

struct WNormProb {      // out += sum lam[r >> shift]^2 |X[r][c]|^2
  const void* X;
  int rows, cols, ld;
  const double* lam;
  int shift;
  double* out;
};

cudaError_t launch_gauss(void* out, long long count, uint64_t seed, uint64_t stream, cudaStream_t s);
cudaError_t launch_rowscale(const RowScaleProb* d_probs, int n, long long max_elems, cudaStream_t s);
cudaError_t launch_chol_inv(const CholProb* d_probs, int n, cudaStream_t s);
cudaError_t launch_wnorm(const WNormProb* d_probs, int n, long long max_elems, cudaStream_t s);

struct GatherProb {
  const void* src;     // V (ld) or Rfull (ld)
  void* dst;
  const int* perm;
  int rows, r, ld;
  int mode;            // 0: site = conj(V[c][perm[mu]]) -> dst[mu][c] (rows = n)
                       // 1: rem  = Rfull[row][perm[mu]] * scale -> dst[row][mu]
  double scale;
  const double* cs;    // per source column scale (1 / |v_j|), or null
};

// Launchers (R = float or double).  Descriptor arrays are device pointers.
template <typename R>
cudaError_t launch_gemm(const GemmProb* d_probs, const long long* d_tile_off, int n_probs,
                        long long total_tiles, cudaStream_t s);
// tile bookkeeping helper (host): tiles of a problem in the GEMM grid
long long gemm_tiles(const GemmProb& p, bool fp64);

template <typename R>
cudaError_t launch_eig_init(const EigProb* d_probs, int n_probs, int max_npad, cudaStream_t s);
// kernel launches of one launch_eig_inner call (round `round` of a batch of width max_nb)
int eig_inner_launches(int max_nb, int round);
template <typename R>
cudaError_t launch_eig_inner(const EigProb* d_probs, int n_probs, int max_nb, int round,
                             cudaStream_t s);
template <typename R>
cudaError_t launch_eig_apply(const EigProb* d_probs, int n_probs, int max_nb, int round,
                             cudaStream_t s);
int eig_block(bool fp64);  // JB
// FP32 round update on the tensor cores (two launches: V and the upper G tiles
// into T, then the G tiles from T); same contract as launch_eig_apply<float>,
// plus the scratch EigProb::T; a bounded completion wait that expires sets *err.
cudaError_t launch_eig_apply_tc(const EigProb* d_probs, int n_probs, int max_nb, int max_npad, int round, int* err,
                                cudaStream_t s);
cudaError_t eig_apply_tc_prepare();
// Set the kernels' shared-memory attributes (idempotent); call before any
// stream capture of the eigen-solve launches.
cudaError_t eig_prepare(bool fp64);
// End of one device-side sweep over n problems (descriptors in device memory,
// modified in place): add the sweep's counters to cum (4 per problem:
// rotations, applied flops, sweeps, and the weight the last sweep moved
// relative to the trace), deactivate converged problems, zero the counters,
// and let the sweep loop continue while any problem is active and fewer than
// max_sweeps sweeps ran (count in *n_sweeps).
// With compact != null, the problems still active are also copied to
// compact[0 .. compact_cap) when they fit, and *mode = 1 (else 0).
cudaError_t launch_sweep_end(EigProb* d_probs, int n, double* cum, double* n_sweeps, int max_sweeps,
                             cudaGraphConditionalHandle h, EigProb* compact, int compact_cap, int* mode,
                             cudaStream_t s);
// Sets the two conditional handles of a sweep body from *mode: h_compact =
// mode, h_full = !mode.
cudaError_t launch_sweep_begin(const int* mode, cudaGraphConditionalHandle h_compact,
                               cudaGraphConditionalHandle h_full, cudaStream_t s);
template <typename R>
cudaError_t launch_eig_trace(const EigProb* d_probs, int n_probs, cudaStream_t s);

template <typename R>
cudaError_t launch_colnorm_batch(const void* const* d_R, const int* d_m, const int* d_n, const int* d_ld,
                                 const double* const* d_lam, const int* d_shift,
                                 double* const* d_rho, int n_probs, int max_n, int max_m,
                                 cudaStream_t s);
cudaError_t launch_rho_normalize(double* const* d_rho, double* const* d_vn, const int* d_n, int n_probs,
                                 int max_n, cudaStream_t s);
template <typename R>
cudaError_t launch_apply_u(const ApplyUProb* d_probs, int n_probs, long long max_cols, cudaStream_t s);
template <typename R>
cudaError_t launch_permute(const PermProb* d_probs, int n_probs, long long max_elems, cudaStream_t s);
cudaError_t launch_select(const SelProb* d_probs, int n_probs, int chi_max, double cutoff, double band,
                          double resolved, double floor2, cudaStream_t s);
template <typename R>
cudaError_t launch_gather(const GatherProb* d_probs, int n_probs, long long max_elems,
                          cudaStream_t s);
template <typename R>
cudaError_t launch_apply_1q(void* const* d_sites, const int* d_cl, const int* d_cr,
                            const double* d_u, int n_sites, long long max_elems, cudaStream_t s);
template <typename R>
cudaError_t launch_amp_step(const void* v_in, void* v_out, const void* site, int cl, int cr,
                            int bit, cudaStream_t s);
template <typename R>
cudaError_t launch_convert_from_c128(const double* src, void* dst, long long n, cudaStream_t s);
template <typename R>
cudaError_t launch_convert_to_c128(const void* src, double* dst, long long n, cudaStream_t s);

// rank predictor network (features -> hidden -> hidden -> rank buckets)
constexpr int MLP_F = 16, MLP_H1 = 64, MLP_H2 = 64, MLP_NB = 16;
int mlp_nparams();
cudaError_t launch_mlp_forward(const float* params, const float* X, int B, float* logits, cudaStream_t s);
cudaError_t launch_mlp_loss_grad(const float* params, const float* X, const int* y, int B, float* grad,
                                 float* loss, cudaStream_t s);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, int t, cudaStream_t s);
cudaError_t launch_entropy(const double* const* d_lams, const int* d_chi, int nb, double* d_out, cudaStream_t s);


// tensor-core complex GEMM on operands packed once per launch (tc_packed.cu):
// op(A) as 32 KB blocks per (batch, 128-row tile, 16-complex K chunk), op(B)
// as 16 KB blocks per (batch, 64-column tile, chunk), each block four TF32
// planes (Re hi / lo, Im hi / lo); pa and pb point into a scratch buffer of
// tc_packed_bytes(g) (A blocks first, tc_packed_a_bytes(g) of them)
struct PackedProb {
  GemmProb g;
  float* pa;
  float* pb;
  int tilesM, tilesN, chunks;
};
void tc_packed_shape(const GemmProb& g, int& tilesM, int& tilesN, int& chunks);
size_t tc_packed_bytes(const GemmProb& g);
size_t tc_packed_a_bytes(const GemmProb& g);
long long tc_packed_pack_blocks(const GemmProb& g);
long long tc_packed_tiles(const GemmProb& g);
// pack (one block per operand block, prefix offsets d_pack_off) then product
// (one CTA per output tile, prefix offsets d_tile_off)
cudaError_t launch_tc_packed(const PackedProb* d_probs, const long long* d_pack_off, const long long* d_tile_off,
                             int n_probs, long long pack_blocks, long long tiles, int* err, cudaStream_t s);

// message returned by ctebd_last_error() in the calling thread
void set_last_error(const std::string& msg);

// FP32 FMA throughput probe: blocks x 256 threads x 8 chains x iters FMAs
cudaError_t launch_fma_peak(float* out, int blocks, int iters, cudaStream_t s);

// sweep cap of the Jacobi eigen-solves (ctebd_set_max_sweeps; default 30)
int max_jacobi_sweeps();

}  // namespace ctebd
