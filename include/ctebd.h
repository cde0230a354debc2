/*
 * ctebd.h -- C ABI of the GB300 cluster-TEBD cluster-update library.
 *
 * Method: arXiv 2502.19289, Sec. III.A (cluster-TEBD).  One iteration takes the
 * circuit's gate list, partitions it into entanglement clusters up to a stop
 * layer L* (Eqs. 6-8), contracts every cluster exactly -- the k MPS sites are
 * merged into theta (chi_L, 2^k, chi_R) and the cluster's gates act as one
 * 2^k x 2^k unitary -- and decomposes theta back into k sites by successive
 * truncated SVDs (Fig. 2, Fig. 3), accumulating the fidelity product of
 * Eqs. 4-5.
 *
 * Conventions
 *   - Qubits 0..n-1, big-endian basis (qubit 0 is the most significant bit of
 *     a basis-state index; |x> = |x_0> (x) |x_1> ..., Sec. IV.A).
 *   - Bond b in 0..n sits left of qubit b; chi[0] = chi[n] = 1.
 *   - Site q is a row-major complex tensor (chi[q], 2, chi[q+1]).  Complex
 *     numbers are interleaved (re, im) pairs.  Host copies are complex128.
 *   - The MPS is held in right-canonical (Vidal) form: right isometries B_q
 *     plus the Schmidt spectrum lambda_b of every bond.  A cluster's theta is
 *     diag(lambda_L) * B_q ... B_{q+k-1}, so every disjoint cluster of an
 *     iteration is truncated against its own Schmidt weights independently.
 *   - Gate matrices: App. A (plus S = P(pi/2)); the first listed qubit of a
 *     two-qubit gate is the most significant bit of its 4x4 matrix.
 *
 * Ownership and errors
 *   - Every call returns int status: CTEBD_OK (0) or a negative CTEBD_ERR_*.
 *     ctebd_last_error() returns the message of the last failure in the
 *     calling thread.
 *   - The library owns all device memory of an mps handle.  The caller owns
 *     every host array it passes and may pass a cudaStream_t (NULL: the
 *     library creates its own stream).  Host results are returned only after
 *     the work producing them has completed on that stream.
 *   - No call falls back to a CPU implementation: a missing or failing GPU
 *     returns CTEBD_ERR_CUDA.
 */
#ifndef CTEBD_ABI_H_
#define CTEBD_ABI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  CTEBD_OK = 0,
  CTEBD_ERR_ARG = -1,     /* invalid argument or precondition */
  CTEBD_ERR_OOM = -2,     /* device or host allocation failed */
  CTEBD_ERR_CUDA = -3,    /* CUDA runtime error (message has details) */
  CTEBD_ERR_TIMEOUT = -4, /* a bounded device-side wait expired */
  CTEBD_ERR_NUMERIC = -5, /* non-finite data or a factorisation that failed */
  CTEBD_ERR_STATE = -6    /* call out of order (e.g. truncate_split without apply_cluster) */
};

/* Arithmetic of the contractions.  FP64: complex128 everywhere.  FP32:
   complex64 sites and contractions, FP64 spectra, weights and fidelities. */
enum { CTEBD_FP64 = 0, CTEBD_FP32 = 1 };

/* Gate codes of the input format (App. A, plus S = P(pi/2) and C-P(phi)). */
enum {
  CTEBD_H = 1, CTEBD_X, CTEBD_Y, CTEBD_Z, CTEBD_S, CTEBD_T, CTEBD_P, CTEBD_X14, CTEBD_SQW,
  CTEBD_CNOT = 10, CTEBD_CY, CTEBD_CZ, CTEBD_SWAP, CTEBD_CH, CTEBD_CS, CTEBD_CT,
  CTEBD_SQSWAP, CTEBD_CP
};

/* Simulation parameters (Sec. II.B truncation, Eqs. 7-8 partition limits). */
typedef struct {
  int n_qubits;
  int chi_max;        /* maximum bond dimension (Sec. II.B) */
  double cutoff;      /* eta: discarded-weight cutoff, relative (0 = keep all) */
  int q_max;          /* Eq. 7: log2 of the largest cluster tensor */
  int l_max;          /* Eq. 8: max layers per iteration (<= 0: unbounded) */
  int k_max;          /* max qubits per cluster (<= 0: only Eq. 7 limits) */
  int precision;      /* CTEBD_FP64 | CTEBD_FP32 */
  int sketch_oversample; /* p of the randomized range finder (0: default 16) */
  int power_iters;    /* q of the randomized range finder */
  int use_rank_model; /* 1: size sketches with the loaded rank predictor */
  uint64_t seed;      /* counter-based RNG key of the sketch matrices */
} ctebd_config;

/* One gate.  layer is 1-based (Sec. II.A); assign_layers() fills it. */
typedef struct {
  int layer;
  int n_q;            /* 1, 2 or 3 qubits, contiguous for n_q > 1 */
  int q[3];
  int kind;
  double param;
} ctebd_gate;

/* One entanglement cluster: qubits q0..q0+k-1 (Sec. III.A).  rank_hint[j-1]
   (j = 1..k-1) is an estimate of the rank of theta across the internal bond
   q0+j; when sketching is enabled (FP32, sketch_oversample > 0) a positive
   hint h with 2 (h + p) <= n sizes a randomized range finder with l = h + p
   columns for that split, otherwise (<= 0) the split is the full eigen-solve.
   cluster_partition sets the hints to 0. */
typedef struct {
  int q0;
  int k;
  int layer_lo;       /* gates with layer_lo < layer <= layer_hi belong to it */
  int layer_hi;
  int rank_hint[11];
} ctebd_cluster;

typedef struct ctebd_mps ctebd_mps;

/* Create the product state |0...0> (all chi = 1, Sec. IV.A) on the current
   CUDA device.  cuda_stream: a cudaStream_t or NULL.  Validates the Eq. 7/8
   preconditions: k_max >= 2 (or <= 0), and q_max >= 2 + 2 log2(chi_max) so a
   single layer of two-qubit gates always fits.  *out is owned by the caller
   and released with mps_destroy.  Errors: ARG, OOM, CUDA. */
int mps_create(const ctebd_config* cfg, void* cuda_stream, ctebd_mps** out);
int mps_destroy(ctebd_mps* mps);

/* Sec. II.A: assign every gate the earliest layer after the last gate on any
   of its qubits (1-based).  Returns the number of layers in *n_layers.
   Pure host function.  Errors: ARG (qubit out of range). */
int assign_layers(ctebd_gate* gates, int n_gates, int n_qubits, int* n_layers);

/* Sec. III.A, Eqs. 6-8: the clusters of one iteration starting after layer
   layer_start.  chi: n_qubits+1 current bond dimensions.  The bond array is
   grown layer by layer; the iteration stops at the last layer L* for which
   every run of entangled bonds (cluster of k = run length + 1 qubits,
   bounded by chi[q0] and chi[q0+k]) satisfies 2^k chi_L chi_R <= 2^q_max,
   k <= k_max, and L* - layer_start <= l_max.  Writes up to cap clusters
   (q0 ascending, layer_lo = layer_start, layer_hi = L*), *n_out and
   *layer_stop = L*.  Pure host function, deterministic.
   Errors: ARG (non-contiguous multi-qubit gate, cap too small),
   STATE (no layer fits: preconditions violated). */
int cluster_partition(const ctebd_gate* gates, int n_gates, int layer_start,
                      const int* chi, const ctebd_config* cfg,
                      ctebd_cluster* out, int cap, int* n_out, int* layer_stop);

/* The exactly contracted cluster as one unitary: the ordered product of the
   gates with layer_lo < layer <= layer_hi acting inside [q0, q0+k).  U is
   written row-major 2^k x 2^k complex128 (q0 is the MSB).  Host function.
   Errors: ARG (a gate straddles the window). */
int cluster_unitary(const ctebd_gate* gates, int n_gates, const ctebd_cluster* c, double* U);

/* Eq. 9 (virtual-MPS bond estimate) as a rank bound for the splits of
   cluster c: out[j-1] = min(chi[q0+j] * prod osr(g), chi[q0] 2^j,
   2^(k-j) chi[q0+k]) where the product runs over the cluster's gates whose
   qubits straddle bond q0+j and osr is the gate's operator-Schmidt rank
   across the cut (2 for controlled gates, 4 for SWAP, sqrt(SWAP) and
   three-qubit gates).  chi: current bond dimensions (n+1).  Host function.
   Errors: ARG. */
int cluster_rank_bounds(const ctebd_gate* gates, int n_gates, const ctebd_cluster* c,
                        const int* chi, int* out);

/* Sec. III.B, Eq. 9: bond dimensions of the virtual MPS of the circuit section
   of layers (layer_start, layer_start + l_max] (l_max <= 0: every later
   layer): out[b] = min(2^E(b) chi[b], chi_max, 2^min(b, N - b)) for b = 0..N,
   where E(b) counts the multi-qubit gates of the section spanning bond b
   (a gate on qubits q..q+w-1 spans bonds q+1..q+w-1) and chi holds the current
   bond dimensions (N+1).  entangling (N+1, may be NULL) receives E(b).  Gates
   must carry layers (assign_layers).  Pure host function.  Errors: ARG. */
int virtual_mps_bonds(const ctebd_gate* gates, int n_gates, int n_qubits, int layer_start, int l_max,
                      const int* chi, int chi_max, int* out, int* entangling);

/* Sec. III.B, Eqs. 10-11: grouping of the N sites of a virtual MPS (chi_v,
   N+1 bond dimensions, e.g. from virtual_mps_bonds) by recursive
   bipartitioning.  A segment of sites lo..hi-1 is a group when
   (hi - lo) + log2 chi_v[lo] + log2 chi_v[hi] <= q_max (the chain's end bonds
   count as 1, which is Eq. 10 for the end segments); otherwise it is cut at
   the bond of smallest chi_v among the cuts that leave neither part larger
   than (1 + imbalance) * ceil((hi - lo) / 2) sites (ties: the most central),
   and both parts recur.  Writes the first site of every group in ascending
   order (up to cap) and *n_groups.  Pure host function.
   Errors: ARG (bad arguments, cap too small), STATE (a single site with its
   bonds exceeds q_max). */
int adaptive_grouping(const int* chi_v, int n_qubits, int q_max, double imbalance, int* group_start,
                      int cap, int* n_groups);

/* One-qubit gate on a qubit outside every cluster (applied to its site's
   physical index; the paper is silent on such qubits).  u: 2x2 complex128
   row-major host array.  Errors: ARG, CUDA. */
int apply_1q(ctebd_mps* mps, int q, const double* u);

/* All one-qubit gates of layers (layer_lo, layer_hi] on qubits outside the
   n_clusters clusters, applied in layer order as one 2x2 product per qubit
   (one batched launch).  Errors: ARG, CUDA. */
int apply_singletons(ctebd_mps* mps, const ctebd_gate* gates, int n_gates,
                     const ctebd_cluster* clusters, int n_clusters, int layer_lo, int layer_hi);

/* Sec. III.A contraction of one cluster: theta = diag(lambda_L) B_q...B_{q+k-1}
   with U (2^k x 2^k complex128, row-major, host) applied to its physical
   multi-index.  theta stays on the device, pending truncate_split on the same
   cluster.  Errors: ARG, CUDA, STATE (cluster already pending). */
int apply_cluster(ctebd_mps* mps, const ctebd_cluster* c, const double* U);

/* Fig. 2 / Fig. 3: split the pending theta of cluster c back into k sites by
   k-1 truncated SVDs (right to left), truncation rule of Sec. II.B (chi_max
   and the relative discarded-weight cutoff eta), per-split fidelity f_j of
   Eq. 4 written to f_out[k-1] (may be NULL), product accumulated (Eq. 5).
   Errors: STATE (nothing pending), CUDA, NUMERIC. */
int truncate_split(ctebd_mps* mps, const ctebd_cluster* c, double* f_out);

/* All clusters of one iteration, batched: every phase is one launch over all
   n clusters.  U[i]: host pointer to cluster i's unitary.  f_out: per-split
   fidelities, cluster by cluster (sum of k_i - 1 entries), may be NULL.
   Clusters must be disjoint.  Errors: ARG, CUDA, NUMERIC. */
int step(ctebd_mps* mps, const ctebd_cluster* c, int n, const double* const* U, double* f_out);

/* Eq. 5: product of all per-split fidelities so far (FP64). */
int fidelity(const ctebd_mps* mps, double* F);

/* <bits|psi>: bits has n_qubits entries in {0,1}, qubit 0 first. */
int amplitude(const ctebd_mps* mps, const uint8_t* bits, double* re, double* im);

/* Current bond dimensions, n_qubits+1 entries. */
int mps_bond_dims(const ctebd_mps* mps, int* chi);

/* Copy site q to host as complex128 (chi[q]*2*chi[q+1] complex = 2x doubles);
   cap is the capacity of buf in doubles.  Errors: ARG (cap too small). */
int mps_to_host(const ctebd_mps* mps, int site, double* buf, size_t cap);

/* Copy bond b's spectrum (chi[b] doubles). */
int mps_lambda_to_host(const ctebd_mps* mps, int bond, double* buf, size_t cap);

/* Replace the state: chi (n+1), sites[q] complex128 host arrays of
   chi[q]*2*chi[q+1] complex, lambdas[b] host arrays of chi[b] doubles.
   Sites must be right isometries (not checked). Errors: ARG, OOM, CUDA. */
int mps_load(ctebd_mps* mps, const int* chi, const double* const* sites,
             const double* const* lambdas);

/* Same, from device buffers already in the run precision (complex64 for
   FP32, complex128 for FP64), row-major; copies device-to-device. */
int mps_load_device(ctebd_mps* mps, const int* chi, const void* const* sites,
                    const double* const* lambdas);

/* Per-split log of the last step() / truncate_split: rows of 12 doubles
   (q0, k, bond, m, n, r, f, W, sketched, eigen-dimension, rank before the
   chi_max cap, rank hint, Jacobi sweeps of the first pass, Jacobi sweeps of
   the FP32 refinement pass) -- 14 doubles per row.  *n_rows receives the row count; up to cap rows
   are written. */
int mps_split_log(const ctebd_mps* mps, double* rows, int cap, int* n_rows);

/* Sketched splits attempted and fallen back to the full split (the tail
   check failed) since mps_create: out[0], out[1]. */
int mps_sketch_stats(const ctebd_mps* mps, double* out);

/* Eigen-solver record since mps_create (not in the paper; the solver of this
   implementation): out[0] = FP32 refinement passes accepted at the sweep cap
   (ctebd_set_max_sweeps) because their last sweep moved at most 1e-8 of the
   trace in weight, out[1] = the largest such last-sweep weight relative to
   the trace.  A pass left rotating with more than that makes the update fail
   with CTEBD_ERR_NUMERIC instead.  Errors: ARG. */
int mps_solver_stats(const ctebd_mps* mps, double* out);

/* ---- Learned rank predictor (sizes the sketched split; not in the paper) ----
   A network F=16 -> 64 -> 64 -> 16 (ReLU, FP32) maps cheap per-split
   features to a bucket b of the ratio rank / Eq.-9 bound, ratio in
   (2^-(b+1)/2, 2^-b/2]; the hint is bound * 2^-b/2.  Parameters are packed
   W1 (64x16), b1, W2 (64x64), b2, W3 (16x64), b3, row-major. */

/* Features of every split of cluster c (k-1 rows of 16 floats, bond q0+1
   first), each divided by 10 except j/k: k, j/k, log2 chi_L, log2 chi_R,
   log2 chi_b, log2 rows, log2 cols, log2 Eq.-9 bound, two-qubit gates
   crossing the bond, two-qubit gates in the cluster, non-Clifford one-qubit
   gates, non-Clifford two-qubit gates, layers in the window, entropy of bond
   b, entropy of the left bond (bits), -log10(cutoff).  entropy: n+1 bond entropies (mps_bond_entropies).
   Host function.  Errors: ARG. */
int rank_features(const ctebd_gate* gates, int n_gates, const ctebd_cluster* c, const int* chi,
                  const double* entropy, const ctebd_config* cfg, float* out);

/* Von Neumann entropy (bits) of every bond spectrum, n+1 doubles. */
int mps_bond_entropies(ctebd_mps* mps, double* out);

/* Copy n = 6288 parameters (host FP32) to the handle's device model. */
int rank_model_load(ctebd_mps* mps, const float* weights, size_t n);

/* Forward pass for B feature rows (host); hints_out[i] = ceil(bounds[i] *
   2^-b/2) for the arg-max bucket b.  Errors: STATE (no model loaded). */
int rank_model_predict(ctebd_mps* mps, const float* features, int B, const int* bounds, int* hints_out);

/* Training kernels on caller-owned device buffers (FP32), stream may be NULL:
   logits (B x 16) = net(X (B x 16)); grad (6288) and the scalar loss receive
   the mean softmax cross-entropy against labels y (B ints) and its gradient
   (both overwritten); one Adam step (lr, 1-based step t) on params with
   moment buffers m1, m2 (n = 6288). */
int mlp_nparams_abi(void);
int mlp_forward(const float* params, const float* X, int B, float* logits, void* stream);
int mlp_loss_grad(const float* params, const float* X, const int* y, int B, float* grad, float* loss,
                  void* stream);
int mlp_adam(float* params, const float* grad, float* m1, float* m2, int n, float lr, int t, void* stream);

/* C (M x N) = A (M x K) B (K x N) on the tensor cores (tcgen05, 3xTF32 for
   FP32 accuracy); complex64 row-major device buffers, M % 128 == 0,
   N % 64 == 0, K % 16 == 0.  Building block of the tensor-core paths, exposed
   for validation.  Errors: ARG, CUDA, TIMEOUT (bounded completion wait). */
int tc_cgemm(const void* A, const void* B, void* C, int M, int K, int N, void* stream);

/* Tensor-core policy for the FP32 complex products, process-wide: 0 never;
   1 (default) the GEMMs (merge, U on clusters with 2^k > 16, Gram,
   projections, sketches) of batches above 2 GFLOP of work, whose problems
   with fewer than 64 rows run on the CUDA cores; 2 always, including the
   Jacobi round updates of the eigen-solve (3xTF32 tile products on tcgen05).
   FP64 products always use the CUDA cores; U on clusters with 2^k <= 16 is a
   streaming kernel in every mode. */
int ctebd_set_tensor_cores(int mode);

/* Eigen-solve sweep loop on the device (not in the paper): with per-launch
   profiling off, a batched eigen-solve runs as one CUDA graph whose WHILE
   node repeats a sweep until every problem has converged (or the sweep cap), with
   no host round trip per sweep.  mode = 1 (default) uses it for batches at
   least 16 Jacobi blocks wide (512 columns in FP32, 256 in FP64) and launches
   the sweeps of narrower batches from the host; 2 uses it for every batch, 0
   for none.  Process-wide; results are the same either way.
   Returns CTEBD_ERR_ARG for other values. */
int ctebd_set_sweep_graphs(int mode);

/* Sweep cap of the Jacobi eigen-solves of the split (not in the paper; the
   solver of this implementation), process-wide, 1..1000 (default 60: the
   first pass takes about 10 sweeps at width 2048, the refinement pass up to
   about 20 on steep spectra).  A solve whose problems still make significant
   rotations after n sweeps makes step / truncate_split / split2_noalloc return
   CTEBD_ERR_NUMERIC (the state's sites of that iteration are then
   undefined).  Errors: ARG. */
int ctebd_set_max_sweeps(int n);

/* The current sweep cap. */
int ctebd_max_sweeps(void);

/* Per-kernel-class accounting.  ctebd_profile(mps, 1) clears the counters
   and starts CUDA-event timing of every launch on the handle's stream (0
   stops timing; launch counts and algorithmic flop/byte counts are always
   kept).  ctebd_profile_read writes one row per kernel class k < cap and the
   number of classes in *n_kinds; ctebd_kernel_name names class k.
   Rows are (launches, total ms, algorithmic flops, algorithmic bytes,
   launches that ran on the tensor cores) at rows[5k].
   Not part of the paper: instrumentation of this implementation. */
int ctebd_profile(ctebd_mps* mps, int mode);
int ctebd_profile_read(ctebd_mps* mps, double* rows, int cap, int* n_kinds);
int ctebd_kernel_name(int kind, char* buf, size_t n);

/* FP32 CUDA-core throughput of the current device, measured (not in the
   paper: the roofline denominator of this implementation's FP32 kernels):
   repeats timed launches of an FMA loop (4 CTAs of 256 threads per SM, 8
   independent chains per thread, 2 flops per FMA), after one warm-up launch.
   Writes the best and mean TFLOP/s and the SM count.  Allocates a small
   buffer.  Errors: ARG, CUDA. */
int ctebd_measure_fma(int repeats, double* tflops_best, double* tflops_mean, int* n_sm);

/* split2_noalloc: the two-site split (apply_cluster + truncate_split for a
   k = 2 cluster) for callers that cannot allocate device memory while they
   run -- e.g. a host that owns all device memory through its own pool, or a
   plugin in a process that forbids cudaMalloc/cudaFree on its hot path
   (both can synchronise the device and stall other streams).  The paper has
   no counterpart: this is an integration variant of this library.

   Inputs (device, complex64 / fp64, row-major): theta is the cluster tensor
   with the gate already applied and WITHOUT the left Schmidt weights,
   (chi_l, 4, chi_r); lam_l holds the chi_l Schmidt values of the left bond.
   Outputs (device, caller-allocated): site_l_out (chi_l, 2, r) -- the
   unweighted left site; site_r_out (r, 2, chi_r) -- the right isometry;
   lam_out (r doubles) -- the renormalised spectrum of the new bond; host
   r_out and f_out (Eq. 4).  Capacities: r <= min(chi_max, 2 chi_l, 2 chi_r).
   Same truncation rule and FP32 arithmetic as the handle path.

   It allocates nothing: its scratch is one file-scope device array of about
   2.4 MiB inside this library, which every GPU that loads the library holds
   until the process exits.  chi_l and chi_r are limited to 128 (larger
   values return CTEBD_ERR_ARG).  The first call on a device resolves the
   array's device address (cudaGetSymbolAddress) with that device current.
   Every call copies descriptors from pageable host memory, reads results
   back and synchronises cuda_stream (NULL: the legacy default stream) before
   returning, so it cannot be called while that stream is being captured.
   Every call shares the array and leaves the previous call's data in it;
   calls that overlap on the GPU (other streams or threads) race on it.
   Errors: ARG, CUDA, NUMERIC. */
int split2_noalloc(const void* theta, const double* lam_l, int chi_l, int chi_r, int chi_max,
                   double cutoff, void* site_l_out, void* site_r_out, double* lam_out,
                   int* r_out, double* f_out, void* cuda_stream);

/* Message of the last error in this thread (NUL-terminated, truncated to n). */
int ctebd_last_error(char* buf, size_t n);

#ifdef __cplusplus
}
#endif
#endif /* CTEBD_ABI_H_ */
