// tc_packed.cu -- grouped complex64 GEMM on the 5th-generation tensor cores
// (tcgen05, sm_103a) with FP32-equivalent accuracy (3xTF32), on operands
// packed once per launch.
//
// Packing.  A pack kernel writes every operand in the order the MMAs read it:
// for each 128-row tile of op(A) and each K chunk of 16 complex, one 32 KB
// block of four planes -- Re_hi, Re_lo, Im_hi, Im_lo, each 128 rows x 16 k
// of TF32 values (x_hi = tf32(x), x_lo = tf32(x - x_hi)) -- and for each
// 64-column tile of op(B), one 16 KB block of the same four planes, 64 rows
// (the columns of B) x 16 k.  Each plane is in the no-swizzle K-major
// core-matrix layout: 8 rows x 4 k (16 bytes) per core matrix, core
// matrices 128 bytes apart along k and 512 bytes apart along the rows.  The
// pack applies op (transpose, conjugate), the per-k weights of A and the zero
// fill of ragged edges, so the product kernel sees only full tiles.
//
// Product.  C = A B is four real products on the planes, Re C = Re A Re B -
// Im A Im B and Im C = Re A Im B + Im A Re B, each as hi.hi + hi.lo + lo.hi
// (the minus through the instruction's negate-A bit).  One CTA computes a
// 128 x 64 complex tile; per K chunk one bulk copy brings the A block and one
// the B block into a 4-stage ring (mbarrier transaction counts), one thread
// issues 24 MMAs (M = 128, N = 64, K = 8) into a fresh pair of TMEM
// accumulators (Re, Im; two pairs alternate), and warps 0-3 drain the
// finished pair with tcgen05.ld into round-to-nearest FP32 registers -- the
// per-chunk drain keeps the product at FP32 accuracy at any K.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "tcgen05.h"

namespace ctebd {
namespace {

constexpr int PM = 128, PN = 64, PKC = 16;                  // tile rows, complex columns, complex k per chunk
constexpr int PLANE_A = PM * PKC * 4, PLANE_B = PN * PKC * 4; // bytes per plane: 8 KB, 4 KB
constexpr int BLOCK_A = 4 * PLANE_A, BLOCK_B = 4 * PLANE_B;   // 32 KB, 16 KB
constexpr int STAGES = 4, STAGE_BYTES = BLOCK_A + BLOCK_B;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr int NT = 192;                                     // warps 0-3 drain, 4 copies, 5 issues MMAs
constexpr uint32_t TMEM_COLS = 256;                         // two (Re, Im) accumulator pairs of 64 + 64
constexpr uint32_t IDESC = t5::idesc_tf32(128, 64);
constexpr uint32_t IDESC_NEGA = IDESC | (1u << 13);        // D -= A B
constexpr uint32_t WAIT_LIMIT = 1u << 26;

__device__ __forceinline__ void split_store(float* plane_hi, float* plane_lo, int o, float x) {
  const float h = t5::tf32_rna(x);
  plane_hi[o] = h;
  plane_lo[o] = t5::tf32_rna(x - h);
}

__device__ __forceinline__ int find_prob(const long long* off, int n, long long v) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= v) lo = mid; else hi = mid;
  }
  return lo;
}

// One block per (problem, operand, batch, tile, chunk): the A blocks of a
// problem first, then its B blocks.  256 threads: coalesced loads of the
// 128 x 16 (A) or 16 x 64 (B) complex sub-block into shared memory, then the
// four planes written out in core-matrix order, 128 contiguous bytes per warp
// and plane.
__global__ void __launch_bounds__(256) k_tc_pack(const PackedProb* __restrict__ probs,
                                                 const long long* __restrict__ off, int n_probs) {
  __shared__ float2 T[PM][PKC + 1];
  const long long bid = blockIdx.x;
  const int pi = find_prob(off, n_probs, bid);
  const PackedProb& Q = probs[pi];
  const GemmProb& g = Q.g;
  long long r = bid - off[pi];
  const int aBat = g.sA ? g.batch : 1;
  const long long nA = (long long)aBat * Q.tilesM * Q.chunks;
  const int t = threadIdx.x;
  if (r < nA) {
    const int c = (int)(r % Q.chunks);
    const long long rt = r / Q.chunks;
    const int tm = (int)(rt % Q.tilesM), b = (int)(rt / Q.tilesM);
    const float2* A = (const float2*)g.A + (long long)b * g.sA;
    const int m0 = tm * PM, k0 = c * PKC;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      int row, k;
      if (g.opA == 0) { k = t & 15; row = (t >> 4) + 16 * j; }
      else { row = t & 127; k = (t >> 7) + 2 * j; }
      const int m = m0 + row, kk = k0 + k;
      float2 v = make_float2(0.f, 0.f);
      if (m < g.M && kk < g.K) {
        if (g.opA == 0) v = A[(long long)m * g.lda + kk];
        else { v = A[(long long)kk * g.lda + m]; v.y = -v.y; }
        if (g.kw) {
          const float w = (float)g.kw[kk >> g.kw_shift];   // FP32 like the operands
          const float f = g.kw_pow == 1 ? w : w * w;
          v.x *= f; v.y *= f;
        }
      }
      T[row][k] = v;
    }
    __syncthreads();
    float* dst = Q.pa + (r * BLOCK_A) / 4;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      // float index o in each plane: core matrix cm = (row / 8) * 4 + k / 4,
      // then (row mod 8) * 4 + k mod 4 inside it
      const int o = t + 256 * j;
      const int cm = o >> 5, w = o & 31;
      const int row = (cm >> 2) * 8 + (w >> 2), k = (cm & 3) * 4 + (w & 3);
      const float2 v = T[row][k];
      split_store(dst, dst + PLANE_A / 4, o, v.x);
      split_store(dst + 2 * PLANE_A / 4, dst + 3 * PLANE_A / 4, o, v.y);
    }
    return;
  }
  r -= nA;
  const int c = (int)(r % Q.chunks);
  const long long rt = r / Q.chunks;
  const int tn = (int)(rt % Q.tilesN), b = (int)(rt / Q.tilesN);
  const float2* B = (const float2*)g.B + (long long)b * g.sB;
  const int n0 = tn * PN, k0 = c * PKC;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    int n, k;
    if (g.opB == 0) { n = t & 63; k = (t >> 6) + 4 * j; }
    else { k = t & 15; n = (t >> 4) + 16 * j; }
    const int nn = n0 + n, kk = k0 + k;
    float2 v = make_float2(0.f, 0.f);
    if (nn < g.N && kk < g.K) {
      if (g.opB == 0) v = B[(long long)kk * g.ldb + nn];
      else { v = B[(long long)nn * g.ldb + kk]; v.y = -v.y; }
    }
    T[n][k] = v;
  }
  __syncthreads();
  float* dst = Q.pb + (r * BLOCK_B) / 4;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const int o = t + 256 * j;
    const int cm = o >> 5, w = o & 31;
    const int n = (cm >> 2) * 8 + (w >> 2), k = (cm & 3) * 4 + (w & 3);
    const float2 v = T[n][k];
    split_store(dst, dst + PLANE_B / 4, o, v.x);
    split_store(dst + 2 * PLANE_B / 4, dst + 3 * PLANE_B / 4, o, v.y);
  }
}

// One CTA per 128 x 64 complex output tile, consecutive CTAs along the
// tile's row (they share the A blocks in L2).
__global__ void __launch_bounds__(NT, 1) k_tc_packed(const PackedProb* __restrict__ probs,
                                                     const long long* __restrict__ off, int n_probs, int* err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ uint64_t full[STAGES], empty[STAGES], accf[2], acce[2];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  unsigned char* ring = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const long long bid = blockIdx.x;
  const int pi = find_prob(off, n_probs, bid);
  const PackedProb& Q = probs[pi];
  const long long rr = bid - off[pi];
  const int tn = (int)(rr % Q.tilesN);
  const long long r2 = rr / Q.tilesN;
  const int tm = (int)(r2 % Q.tilesM), b = (int)(r2 / Q.tilesM);
  const int nch = Q.chunks;
  const int ab = Q.g.sA ? b : 0, bb = Q.g.sB ? b : 0;
  const unsigned char* srcA = (const unsigned char*)Q.pa + ((long long)ab * Q.tilesM + tm) * nch * (long long)BLOCK_A;
  const unsigned char* srcB = (const unsigned char*)Q.pb + ((long long)bb * Q.tilesN + tn) * nch * (long long)BLOCK_B;

  if (warp == 0) t5::tmem_alloc(&tmem_base, TMEM_COLS);
  if (t == 0) {
    for (int s = 0; s < STAGES; s++) { t5::mbar_init(&full[s], 1); t5::mbar_init(&empty[s], 1); }
    for (int i = 0; i < 2; i++) { t5::mbar_init(&accf[i], 1); t5::mbar_init(&acce[i], 128); }
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  t5::fence_before();
  __syncthreads();
  t5::fence_after();
  const uint32_t tmem = tmem_base;
  auto wait_bar = [&](uint64_t* bar, long long n) {   // completion number n of bar
    if (!t5::mbar_wait(bar, (uint32_t)(n & 1), WAIT_LIMIT)) failed = 1;
  };

  if (warp == 4) {                                        // producer: one bulk copy per operand block
    if (lane == 0) {
      int c = 0;
      for (; c < nch; c++) {
        const int s = c % STAGES;
        if (c >= STAGES) wait_bar(&empty[s], c / STAGES - 1);
        if (failed) break;
        unsigned char* st = ring + s * STAGE_BYTES;
        t5::mbar_expect_tx(&full[s], STAGE_BYTES);
        t5::bulk_g2s(st, srcA + (long long)c * BLOCK_A, BLOCK_A, &full[s]);
        t5::bulk_g2s(st + BLOCK_A, srcB + (long long)c * BLOCK_B, BLOCK_B, &full[s]);
      }
      // no copy may still be landing when the CTA exits
      for (int u = std::max(0, c - STAGES); u < c; u++) t5::mbar_wait(&full[u % STAGES], (uint32_t)((u / STAGES) & 1), WAIT_LIMIT);
    }
  } else if (warp == 5) {                                 // MMA issuer
    if (lane == 0) {
      int c = 0;
      for (; c < nch; c++) {
        const int s = c % STAGES, set = c & 1;
        wait_bar(&full[s], c / STAGES);
        if (c >= 2) wait_bar(&acce[set], c / 2 - 1);
        if (failed) break;
        t5::fence_after();
        const uint32_t a0 = t5::smem_u32(ring + s * STAGE_BYTES), b0 = a0 + BLOCK_A;
        const uint32_t cre = tmem + (uint32_t)set * 128, cim = cre + 64;
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {                  // K = 8 per MMA: two core matrices
          const uint32_t ko = (uint32_t)ks * 256;
          const uint64_t are_h = t5::desc_noswizzle(a0 + ko, 128, 512);
          const uint64_t are_l = t5::desc_noswizzle(a0 + PLANE_A + ko, 128, 512);
          const uint64_t aim_h = t5::desc_noswizzle(a0 + 2 * PLANE_A + ko, 128, 512);
          const uint64_t aim_l = t5::desc_noswizzle(a0 + 3 * PLANE_A + ko, 128, 512);
          const uint64_t bre_h = t5::desc_noswizzle(b0 + ko, 128, 512);
          const uint64_t bre_l = t5::desc_noswizzle(b0 + PLANE_B + ko, 128, 512);
          const uint64_t bim_h = t5::desc_noswizzle(b0 + 2 * PLANE_B + ko, 128, 512);
          const uint64_t bim_l = t5::desc_noswizzle(b0 + 3 * PLANE_B + ko, 128, 512);
          const uint32_t acc = ks > 0 ? 1u : 0u;
          // small terms first
          t5::mma_tf32<IDESC>(cre, are_l, bre_h, acc);
          t5::mma_tf32<IDESC>(cre, are_h, bre_l, 1u);
          t5::mma_tf32<IDESC>(cre, are_h, bre_h, 1u);
          t5::mma_tf32<IDESC_NEGA>(cre, aim_l, bim_h, 1u);
          t5::mma_tf32<IDESC_NEGA>(cre, aim_h, bim_l, 1u);
          t5::mma_tf32<IDESC_NEGA>(cre, aim_h, bim_h, 1u);
          t5::mma_tf32<IDESC>(cim, are_l, bim_h, acc);
          t5::mma_tf32<IDESC>(cim, are_h, bim_l, 1u);
          t5::mma_tf32<IDESC>(cim, are_h, bim_h, 1u);
          t5::mma_tf32<IDESC>(cim, aim_l, bre_h, 1u);
          t5::mma_tf32<IDESC>(cim, aim_h, bre_l, 1u);
          t5::mma_tf32<IDESC>(cim, aim_h, bre_h, 1u);
        }
        t5::mma_commit(&empty[s]);
        t5::mma_commit(&accf[set]);
      }
      // after a timeout: the MMAs already issued finish before TMEM is freed
      if (failed && c > 0) t5::mbar_wait(&accf[(c - 1) & 1], (uint32_t)(((c - 1) / 2) & 1), WAIT_LIMIT);
    }
  } else {                                                // warps 0-3: lanes 32 warp .. 32 warp + 31 = rows
    float acc[128];                                       // Re 0..63, Im 64..127
#pragma unroll
    for (int i = 0; i < 128; i++) acc[i] = 0.f;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c = 0; c < nch; c++) {
      const int set = c & 1;
      wait_bar(&accf[set], c / 2);
      if (failed) break;
      t5::fence_after();
#pragma unroll
      for (int q = 0; q < 4; q++) {
        float v[32];
        t5::tmem_ld32(lane_base + (uint32_t)set * 128 + (uint32_t)q * 32, v);
#pragma unroll
        for (int i = 0; i < 32; i++) acc[q * 32 + i] = __fadd_rn(acc[q * 32 + i], v[i]);
      }
      t5::fence_before();
      t5::mbar_arrive(&acce[set]);
    }
    if (!failed) {
      const GemmProb& g = Q.g;
      const int m = tm * PM + warp * 32 + lane;
      const float alpha = (float)g.alpha;
      if (m < g.M) {
        float2* Crow = (float2*)g.C + (long long)b * g.sC + (long long)m * g.ldc;
        const int nmax = min(PN, g.N - tn * PN);
#pragma unroll
        for (int j = 0; j < PN; j++)
          if (j < nmax) Crow[tn * PN + j] = make_float2(alpha * acc[j], alpha * acc[64 + j]);
      }
    }
  }
  t5::fence_before();
  __syncthreads();
  t5::fence_after();
  if (warp == 0) t5::tmem_dealloc(tmem, TMEM_COLS);
  if (failed && t == 0) atomicExch(err, 1);
}

}  // namespace

void tc_packed_shape(const GemmProb& g, int& tilesM, int& tilesN, int& chunks) {
  tilesM = (g.M + PM - 1) / PM;
  tilesN = (g.N + PN - 1) / PN;
  chunks = (g.K + PKC - 1) / PKC;
}

size_t tc_packed_bytes(const GemmProb& g) {
  int tM, tN, ch;
  tc_packed_shape(g, tM, tN, ch);
  const size_t aBat = g.sA ? g.batch : 1, bBat = g.sB ? g.batch : 1;
  return aBat * tM * ch * (size_t)BLOCK_A + bBat * tN * ch * (size_t)BLOCK_B;
}

size_t tc_packed_a_bytes(const GemmProb& g) {
  int tM, tN, ch;
  tc_packed_shape(g, tM, tN, ch);
  return (size_t)(g.sA ? g.batch : 1) * tM * ch * (size_t)BLOCK_A;
}

long long tc_packed_pack_blocks(const GemmProb& g) {
  int tM, tN, ch;
  tc_packed_shape(g, tM, tN, ch);
  return (long long)(g.sA ? g.batch : 1) * tM * ch + (long long)(g.sB ? g.batch : 1) * tN * ch;
}

long long tc_packed_tiles(const GemmProb& g) {
  int tM, tN, ch;
  tc_packed_shape(g, tM, tN, ch);
  return (long long)tM * tN * g.batch;
}

cudaError_t launch_tc_packed(const PackedProb* d_probs, const long long* d_pack_off, const long long* d_tile_off,
                             int n_probs, long long pack_blocks, long long tiles, int* err, cudaStream_t s) {
  if (tiles <= 0) return cudaSuccess;
  if (pack_blocks > 0x7fffffffLL || tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_packed, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_tc_pack<<<(unsigned)pack_blocks, 256, 0, s>>>(d_probs, d_pack_off, n_probs);
  k_tc_packed<<<(unsigned)tiles, NT, SMEM_BYTES, s>>>(d_probs, d_tile_off, n_probs, err);
  return cudaGetLastError();
}

}  // namespace ctebd
