// tc_gemm.cu -- complex64 tile products on the 5th-generation tensor cores
// (tcgen05, sm_103a) with FP32-equivalent accuracy (3xTF32).
//
// A complex product C = A B is computed as one real product through the
// interleaved embedding: the raw memory of a complex row [re, im, re, im, ...]
// is the real row of A', and B' (2K x 2N) holds [[re, im], [-im, re]] blocks,
// so C' = A' B' is the raw memory of C.  Each operand x is split into
// x_hi = tf32(x) and x_lo = tf32(x - x_hi); D = A_hi B_hi + A_hi B_lo + A_lo B_hi
// accumulates in FP32 in tensor memory.
//
// One CTA computes a 128 x 64 complex tile (M = 128, N = 128 real) over K in
// chunks of 16 complex (32 real): operands are staged by 256 threads in the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes; padded strides),
// one thread issues 12 MMAs (3 products x 4 K-steps of 8) per chunk and
// commits them to the chunk's mbarrier; two stages let the staging of the next
// chunk overlap the tensor cores.  Each chunk accumulates into a fresh TMEM
// accumulator (two alternate); warps 0-3 (lanes 32w..32w+31 = rows) drain the
// finished one with tcgen05.ld into FP32 registers and finally hand each
// element to the caller's store functor.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace ctebd {
namespace tc {

constexpr int TM = 128;        // rows per tile
constexpr int TNC = 64;        // complex columns per tile (128 real)
constexpr int TKC = 16;        // complex K per chunk (32 real)
constexpr int NTHREADS = 256;
// operand copy: 16 row groups x 8 K-core-matrices; core matrices 144 B apart
// along K and row groups 1168 B apart (padding spreads the stores over the
// shared-memory banks; both offsets are multiples of 16 B)
constexpr uint32_t LBO = 144, SBO = 8 * 144 + 16;
constexpr int OP_BYTES = 16 * SBO;                 // 18688 B
constexpr int STAGE_BYTES = 4 * OP_BYTES;          // A_hi, A_lo, B_hi, B_lo
// raw FP32 operand chunks in their source memory order (A: 128 x 16 or 16 x 128
// complex; B: 16 x 64 or 64 x 16), two buffers, filled by cp.async one chunk ahead
constexpr int RAW_A = TM * TKC, RAW_B = TKC * TNC;   // complex elements
constexpr int RAW_BYTES = (RAW_A + RAW_B) * 8;       // 24576 B
constexpr int SMEM_BYTES = 2 * STAGE_BYTES + 2 * RAW_BYTES + 1024;
constexpr uint32_t TMEM_COLS = 128;
// kind::tf32, D = F32, A = B = TF32, both K-major, N = 128, M = 128
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t WAIT_LIMIT = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// 16-byte asynchronous copy global -> shared; bytes < 16 are zero-filled
__device__ __forceinline__ void cp16_zfill(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// shared-memory matrix descriptor (tcgen05), no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((LBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((SBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < WAIT_LIMIT; it++) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it > 64) __nanosleep(32);
  }
  return false;
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// byte offset of real element (row, k) of a 128 x 32 K-major operand copy
__device__ __forceinline__ uint32_t op_off(int row, int k) {
  return (uint32_t)((row >> 3) * SBO + (k >> 2) * LBO + ((row & 7) << 4) + ((k & 3) << 2));
}

// two consecutive real K elements (k even) as hi/lo tf32 pairs
__device__ __forceinline__ void put2(unsigned char* hi, unsigned char* lo, uint32_t off, float x, float y) {
  const float hx = tf32_round(x), hy = tf32_round(y);
  *reinterpret_cast<float2*>(hi + off) = make_float2(hx, hy);
  *reinterpret_cast<float2*>(lo + off) = make_float2(tf32_round(x - hx), tf32_round(y - hy));
}

// a_rows_fast / b_k_fast choose which index consecutive threads walk, so
// that global loads are coalesced for both memory orders of each operand
template <class LoadA, class LoadB>
__device__ __forceinline__ void stage_chunk(unsigned char* st, int kc0, LoadA& loadA, LoadB& loadB,
                                            bool a_rows_fast, bool b_k_fast) {
  unsigned char *ah = st, *al = st + OP_BYTES, *bh = st + 2 * OP_BYTES, *bl = st + 3 * OP_BYTES;
  const int t = threadIdx.x;
  // A': 128 rows x 16 complex
  #pragma unroll 4
  for (int e = t; e < TM * TKC; e += NTHREADS) {
    const int r = a_rows_fast ? e % TM : e / TKC, c = a_rows_fast ? e / TM : e % TKC;
    const float2 v = loadA(r, kc0 + c);
    put2(ah, al, op_off(r, 2 * c), v.x, v.y);
  }
  // B'^T: row 2d = (re, -im), row 2d+1 = (im, re) at K = 2c, 2c+1
  #pragma unroll 4
  for (int e = t; e < TKC * TNC; e += NTHREADS) {
    const int c = b_k_fast ? e % TKC : e / TNC, d = b_k_fast ? e / TKC : e % TNC;
    const float2 b = loadB(kc0 + c, d);
    put2(bh, bl, op_off(2 * d, 2 * c), b.x, -b.y);
    put2(bh, bl, op_off(2 * d + 1, 2 * c), b.y, b.x);
  }
}

// read the 128 accumulator columns of this warp's 32 lanes (rows) and add
// them to acc (round-to-nearest FP32 adds)
__device__ __forceinline__ void drain_add(uint32_t taddr_row, float (&acc)[128]) {
  #pragma unroll
  for (int cb = 0; cb < 4; cb++) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr_row + (uint32_t)(cb * 32)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    #pragma unroll
    for (int i = 0; i < 32; i++) acc[cb * 32 + i] = __fadd_rn(acc[cb * 32 + i], __uint_as_float(r[i]));
  }
}

// C tile = A B over complex K.  Two shared-memory stages and two TMEM
// accumulators: while the tensor cores work on chunk i (into accumulator
// i % 2, started fresh), the other threads stage chunk i+1 and warps 0-3
// drain the finished accumulator of chunk i-1 into round-to-nearest FP32
// registers.  (Accumulating all of K inside the tensor core loses about one
// bit per chunk to its internal accumulation; per-chunk draining keeps the
// product at FP32 accuracy.)  Returns false (and sets *err) when a bounded
// completion wait timed out.
template <class LoadA, class LoadB, class Store>
__device__ bool tile_product(int kc_total, LoadA loadA, LoadB loadB, Store store, int* err,
                             bool a_rows_fast = false, bool b_k_fast = false) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_smem + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(2 * TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])));
    failed = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t d_tmem = tmem_base;
  const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
  float acc[128];
  #pragma unroll
  for (int i = 0; i < 128; i++) acc[i] = 0.f;
  const int nchunks = (kc_total + TKC - 1) / TKC;
  uint32_t phase[2] = {0u, 0u};
  for (int i = 0; i < nchunks; i++) {
    const int sidx = i & 1;
    unsigned char* st = base + sidx * STAGE_BYTES;
    if (i >= 2) {   // chunk i-2 used this stage and this accumulator
      if (!mbar_wait(&bar[sidx], phase[sidx])) failed = 1;
      phase[sidx] ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (warp < 4 && !failed) drain_add(d_tmem + lane_off + sidx * TMEM_COLS, acc);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    stage_chunk(st, i * TKC, loadA, loadB, a_rows_fast, b_k_fast);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (failed) break;
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = smem_u32(st), al = ah + OP_BYTES, bh = ah + 2 * OP_BYTES, bl = ah + 3 * OP_BYTES;
      const uint32_t dt = d_tmem + sidx * TMEM_COLS;
      #pragma unroll
      for (int s = 0; s < 4; s++) {   // K = 8 real per instruction: two core matrices
        const uint32_t o = 2u * LBO * s;
        mma_tf32(dt, make_desc(al + o), make_desc(bh + o), s > 0 ? 1u : 0u);
        mma_tf32(dt, make_desc(ah + o), make_desc(bl + o), 1u);
        mma_tf32(dt, make_desc(ah + o), make_desc(bh + o), 1u);
      }
      mma_commit(&bar[sidx]);
    }
  }
  // drain the last (up to) two chunks; after a timeout, one more bounded wait
  // per stage so no MMA still runs when TMEM is freed
  if (!failed) {
    for (int i = (nchunks >= 2 ? nchunks - 2 : 0); i < nchunks; i++) {
      const int sidx = i & 1;
      if (!mbar_wait(&bar[sidx], phase[sidx])) { failed = 1; break; }
      phase[sidx] ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (warp < 4) drain_add(d_tmem + lane_off + sidx * TMEM_COLS, acc);
    }
  } else {
    mbar_wait(&bar[0], phase[0]);
    mbar_wait(&bar[1], phase[1]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (!failed && warp < 4) {
    const int row = warp * 32 + lane;
    #pragma unroll
    for (int i = 0; i < 64; i++) store(row, i, make_float2(acc[2 * i], acc[2 * i + 1]));
  }
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(d_tmem), "r"(2 * TMEM_COLS));
  if (failed && threadIdx.x == 0) atomicExch(err, 1);
  return !failed;
}

// tile_product with the operand loads taken off the critical path: fetch(raw,
// kc0) issues the cp.async copies of chunk kc0 into a raw buffer one chunk
// ahead, and convA / convB (raw buffer, row or k index, local k, global k)
// read the element from it while the chunk is staged.  Same tensor-core
// schedule, drains and error handling as tile_product.
template <class Fetch, class ConvA, class ConvB, class Store>
__device__ bool tile_product_async(int kc_total, Fetch fetch, ConvA convA, ConvB convB, Store store, int* err,
                                   bool a_rows_fast, bool b_k_fast) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  unsigned char* base = (unsigned char*)(((uintptr_t)tc_smem + 1023) & ~(uintptr_t)1023);
  unsigned char* raw0 = base + 2 * STAGE_BYTES;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = (kc_total + TKC - 1) / TKC;
  fetch(raw0, 0);
  cp_commit();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(2 * TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])));
    failed = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t d_tmem = tmem_base;
  const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
  float acc[128];
  #pragma unroll
  for (int i = 0; i < 128; i++) acc[i] = 0.f;
  uint32_t phase[2] = {0u, 0u};
  const float2* rawA = nullptr;
  const float2* rawB = nullptr;
  int kc0 = 0;
  auto la = [&](int r, int k) { return convA(rawA, r, k - kc0, k); };
  auto lb = [&](int k, int d) { return convB(rawB, k - kc0, d, k); };
  for (int i = 0; i < nchunks; i++) {
    const int sidx = i & 1;
    unsigned char* st = base + sidx * STAGE_BYTES;
    // the raw buffer of chunk i + 1 was last read while staging chunk i - 1
    if (i + 1 < nchunks) fetch(raw0 + ((i + 1) & 1) * RAW_BYTES, (i + 1) * TKC);
    cp_commit();
    if (i >= 2) {   // chunk i-2 used this stage and this accumulator
      if (!mbar_wait(&bar[sidx], phase[sidx])) failed = 1;
      phase[sidx] ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (warp < 4 && !failed) drain_add(d_tmem + lane_off + sidx * TMEM_COLS, acc);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    cp_wait_prev();   // this thread's copies of chunk i have landed
    __syncthreads();  // and everybody's
    rawA = reinterpret_cast<const float2*>(raw0 + sidx * RAW_BYTES);
    rawB = rawA + RAW_A;
    kc0 = i * TKC;
    stage_chunk(st, kc0, la, lb, a_rows_fast, b_k_fast);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (failed) break;
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = smem_u32(st), al = ah + OP_BYTES, bh = ah + 2 * OP_BYTES, bl = ah + 3 * OP_BYTES;
      const uint32_t dt = d_tmem + sidx * TMEM_COLS;
      #pragma unroll
      for (int s = 0; s < 4; s++) {   // K = 8 real per instruction: two core matrices
        const uint32_t o = 2u * LBO * s;
        mma_tf32(dt, make_desc(al + o), make_desc(bh + o), s > 0 ? 1u : 0u);
        mma_tf32(dt, make_desc(ah + o), make_desc(bl + o), 1u);
        mma_tf32(dt, make_desc(ah + o), make_desc(bh + o), 1u);
      }
      mma_commit(&bar[sidx]);
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");   // no copy in flight past this point
  if (!failed) {
    for (int i = (nchunks >= 2 ? nchunks - 2 : 0); i < nchunks; i++) {
      const int sidx = i & 1;
      if (!mbar_wait(&bar[sidx], phase[sidx])) { failed = 1; break; }
      phase[sidx] ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (warp < 4) drain_add(d_tmem + lane_off + sidx * TMEM_COLS, acc);
    }
  } else {
    mbar_wait(&bar[0], phase[0]);
    mbar_wait(&bar[1], phase[1]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (!failed && warp < 4) {
    const int row = warp * 32 + lane;
    #pragma unroll
    for (int i = 0; i < 64; i++) store(row, i, make_float2(acc[2 * i], acc[2 * i + 1]));
  }
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(d_tmem), "r"(2 * TMEM_COLS));
  if (failed && threadIdx.x == 0) atomicExch(err, 1);
  return !failed;
}

// ---------------------------------------------------------------------------
// Plain product: C (M x N) = A (M x K) B (K x N), complex64 row-major;
// M % 128 == 0, N % 64 == 0, K % 16 == 0.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tc_plain(const float2* __restrict__ A, const float2* __restrict__ B,
                                                  float2* __restrict__ C, int M, int K, int N, int* err) {
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TNC;
  tile_product(
      K, [&](int r, int c) { return A[(long long)(m0 + r) * K + c]; },
      [&](int c, int d) { return B[(long long)c * N + n0 + d]; },
      [&](int r, int d, float2 v) { C[(long long)(m0 + r) * N + n0 + d] = v; }, err);
}

// ---------------------------------------------------------------------------
// Grouped complex GEMM on the tensor cores: the same problem descriptors as
// the SIMT k_gemm (op(A), op(B), per-k weights, batches, alpha); tiles of 128
// rows x 64 complex columns; ragged edges read as zero and are not stored.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tc_gemm(const GemmProb* __restrict__ probs,
                                                 const long long* __restrict__ tile_off, int n_probs, int* err) {
  const long long tid_tile = blockIdx.x;
  int lo = 0, hi = n_probs;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (tile_off[mid] <= tid_tile) lo = mid; else hi = mid;
  }
  const GemmProb P = probs[lo];
  long long t = tid_tile - tile_off[lo];
  const int tilesN = (P.N + TNC - 1) / TNC, tilesM = (P.M + TM - 1) / TM;
  const int tn = (int)(t % tilesN);
  t /= tilesN;
  const int tm = (int)(t % tilesM);
  const long long bidx = t / tilesM;
  const float2* A = (const float2*)P.A + bidx * P.sA;
  const float2* B = (const float2*)P.B + bidx * P.sB;
  float2* Cm = (float2*)P.C + bidx * P.sC;
  const int m0 = tm * TM, n0 = tn * TNC;
  const float alpha = (float)P.alpha;
  auto loadA = [&](int r, int c) -> float2 {
    const int m = m0 + r;
    if (m >= P.M || c >= P.K) return make_float2(0.f, 0.f);
    float2 v;
    if (P.opA == 0) v = A[(long long)m * P.lda + c];
    else { v = A[(long long)c * P.lda + m]; v.y = -v.y; }
    if (P.kw) {
      const float w = (float)P.kw[c >> P.kw_shift];   // FP32 like the operands (FP64 is slow here)
      const float f = P.kw_pow == 1 ? w : w * w;
      v.x *= f; v.y *= f;
    }
    return v;
  };
  auto loadB = [&](int c, int d) -> float2 {
    const int n = n0 + d;
    if (n >= P.N || c >= P.K) return make_float2(0.f, 0.f);
    if (P.opB == 0) return B[(long long)c * P.ldb + n];
    float2 v = B[(long long)n * P.ldb + c];
    v.y = -v.y;
    return v;
  };
  auto store = [&](int r, int d, float2 v) {
    const int m = m0 + r, n = n0 + d;
    if (m < P.M && n < P.N) Cm[(long long)m * P.ldc + n] = make_float2(alpha * v.x, alpha * v.y);
  };
  if (!P.async_ok) {
    tile_product(P.K, loadA, loadB, store, err, P.opA == 1, P.opB == 1);
    return;
  }
  // raw chunk copies: each 16-byte granule is two complex elements of one
  // contiguous source row; out-of-range elements are zero-filled
  auto fetch = [&](unsigned char* raw, int k0) {
    float2* ra = reinterpret_cast<float2*>(raw);
    float2* rb = ra + RAW_A;
    for (int g = threadIdx.x; g < RAW_A / 2; g += NTHREADS) {
      int m, k, valid;
      long long off;
      float2* dst;
      if (P.opA == 0) {   // rows m, 16 k each
        const int o = g >> 3, c = (g & 7) * 2;
        m = m0 + o; k = k0 + c;
        valid = m < P.M ? min(2, P.K - k) : 0;
        off = (long long)m * P.lda + k;
        dst = ra + o * TKC + c;
      } else {            // rows k, 128 m each
        const int o = g >> 6, c = (g & 63) * 2;
        k = k0 + o; m = m0 + c;
        valid = k < P.K ? min(2, P.M - m) : 0;
        off = (long long)k * P.lda + m;
        dst = ra + o * TM + c;
      }
      valid = max(valid, 0);
      cp16_zfill(dst, valid > 0 ? (const void*)(A + off) : (const void*)A, 8 * valid);
    }
    for (int g = threadIdx.x; g < RAW_B / 2; g += NTHREADS) {
      int n, k, valid;
      long long off;
      float2* dst;
      if (P.opB == 0) {   // rows k, 64 n each
        const int o = g >> 5, c = (g & 31) * 2;
        k = k0 + o; n = n0 + c;
        valid = k < P.K ? min(2, P.N - n) : 0;
        off = (long long)k * P.ldb + n;
        dst = rb + o * TNC + c;
      } else {            // rows n, 16 k each
        const int o = g >> 3, c = (g & 7) * 2;
        n = n0 + o; k = k0 + c;
        valid = n < P.N ? min(2, P.K - k) : 0;
        off = (long long)n * P.ldb + k;
        dst = rb + o * TKC + c;
      }
      valid = max(valid, 0);
      cp16_zfill(dst, valid > 0 ? (const void*)(B + off) : (const void*)B, 8 * valid);
    }
  };
  auto convA = [&](const float2* ra, int r, int c, int k) -> float2 {
    float2 v = P.opA == 0 ? ra[r * TKC + c] : ra[c * TM + r];
    if (P.opA == 1) v.y = -v.y;
    if (P.kw && k < P.K) {
      const float w = (float)P.kw[k >> P.kw_shift];   // FP32 like the operands (FP64 is slow here)
      const float f = P.kw_pow == 1 ? w : w * w;
      v.x *= f; v.y *= f;
    }
    return v;
  };
  auto convB = [&](const float2* rb, int c, int d, int k) -> float2 {
    (void)k;
    float2 v = P.opB == 0 ? rb[c * TNC + d] : rb[d * TKC + c];
    if (P.opB == 1) v.y = -v.y;
    return v;
  };
  tile_product_async(P.K, fetch, convA, convB, store, err, P.opA == 1, P.opB == 1);
}

long long tc_gemm_tiles(const GemmProb& p) {
  return (long long)((p.M + TM - 1) / TM) * ((p.N + TNC - 1) / TNC) * p.batch;
}

}  // namespace tc

long long tc_gemm_tiles(const GemmProb& p) { return tc::tc_gemm_tiles(p); }

cudaError_t launch_tc_gemm(const GemmProb* d_probs, const long long* d_tile_off, int n_probs,
                           long long total_tiles, int* err, cudaStream_t s) {
  if (total_tiles <= 0) return cudaSuccess;
  if (total_tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc::k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
    attr = true;
  }
  tc::k_tc_gemm<<<(unsigned)total_tiles, tc::NTHREADS, tc::SMEM_BYTES, s>>>(d_probs, d_tile_off, n_probs, err);
  return cudaGetLastError();
}

cudaError_t launch_tc_plain(const void* A, const void* B, void* C, int M, int K, int N, int* err,
                            cudaStream_t s) {
  if (M % tc::TM || N % tc::TNC || K % tc::TKC || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc::k_tc_plain, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
    attr = true;
  }
  tc::k_tc_plain<<<dim3(M / tc::TM, N / tc::TNC), tc::NTHREADS, tc::SMEM_BYTES, s>>>(
      (const float2*)A, (const float2*)B, (float2*)C, M, K, N, err);
  return cudaGetLastError();
}

}  // namespace ctebd
