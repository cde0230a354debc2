// eig_tc.cu -- one round of the batched block-Jacobi eigensolver (FP32) on the
// 5th-generation tensor cores: G <- J^H G J and V <- V J, where J is the
// round's block-diagonal unitary (one 64 x 64 block J_p per pair of 32-wide
// column blocks, round-robin pairing).
//
// Every product is a complex 128 x 64 x 64 tile product X J_c on tcgen05
// (kind::tf32, M = 128, N = 128 real, K = 128 real, accumulator in tensor
// memory), computed in the form X + X (J_c - I):
//   - the complex product is embedded as a real one: the interleaved rows of X
//     are the real rows of A', and B' holds [[re, im], [-im, re]] blocks of
//     (J_c - I), so A' B' is the interleaved result;
//   - 3xTF32: both operands are split into hi = tf32(x) and lo = tf32(x - hi),
//     and lo*hi + hi*lo + hi*hi accumulate in FP32 in tensor memory;
//   - X itself is added in FP32 (round to nearest) in the epilogue, so the
//     tensor-pipe accumulation error scales with |J_c - I|, which vanishes as
//     the sweeps converge.
// The two-sided update runs as two launches per round:
//   phase 0: V tiles (128 rows x one column pair Q): V <- V J_Q, in place;
//            G tiles of the upper pair triangle (row pairs P <= Q, two stacked
//            per 128-row tile): T_PQ = G_PQ J_Q into the scratch T;
//   phase 1: for every column pair P and row pairs Q >= P (two stacked):
//            Y_QP = T_PQ^H J_P = J_Q^H G_QP J_P, written to G_QP and, mirrored,
//            to G_PQ (Y is Hermitian).
// A pair whose J_p is the identity (pair flag 0) is skipped: phase 0 leaves
// column Q alone (T_PQ = G_PQ, read from G), and phase 1 copies T^H where only
// the column side rotated.
//
// One CTA of 128 threads per tile; thread t owns row t of the tile in the
// operand staging and tensor-memory lane t in the epilogue.  K runs in four
// chunks of 16 complex through one shared-memory stage (64 KB: A hi/lo, B
// hi/lo); the next chunk's global loads are in registers while the tensor
// cores work on the current one, and three CTAs share an SM.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "tcgen05.h"

namespace ctebd {
namespace {

constexpr int TM = 128;                    // rows of a tile
constexpr int KC = 16;                     // complex K per chunk
constexpr int NCH = 4;                     // chunks: K = 64 complex
constexpr int NT = 128;                    // threads per CTA
constexpr uint32_t LBO = 128, SBO = 1024;  // core matrices along K / along rows
constexpr int OPB = 16 * 1024;             // one 128 x 32 real operand piece
constexpr int SMEM_BYTES = 4 * OPB + 1024; // A hi, A lo, B hi, B lo (+ 1 KB alignment slack)
constexpr uint32_t IDESC = t5::idesc_tf32(128, 128);
constexpr uint32_t TMEM_COLS = 128;
constexpr uint32_t WAIT_LIMIT = 1u << 26;

// byte offset of real element (row, k) of a 128 x 32 K-major operand piece
__device__ __forceinline__ uint32_t opoff(int row, int k) {
  return (uint32_t)((row >> 3) * SBO + (k >> 2) * LBO + ((row & 7) << 4) + ((k & 3) << 2));
}

// Round-robin (circle method) pairing of N blocks, round t, slot i -> blocks a < b.
__device__ __forceinline__ void pair_blocks(int t, int i, int N, int& a, int& b) {
  const int M = N - 1;
  if (i == 0) { a = t; b = N - 1; }
  else { a = (t + i) % M; b = (t - i + M) % M; }
  if (a > b) { const int x = a; a = b; b = x; }
}

// global index of local index l (0..63) of a pair's two 32-wide blocks
struct PairIdx {
  int a = 0, b = 0;
  __device__ __forceinline__ int operator()(int l) const { return l < 32 ? a * 32 + l : b * 32 + l - 32; }
};

__device__ __forceinline__ float4 split_hi(float4 v) {
  return make_float4(t5::tf32_rna(v.x), t5::tf32_rna(v.y), t5::tf32_rna(v.z), t5::tf32_rna(v.w));
}
__device__ __forceinline__ float4 split_lo(float4 v, float4 h) {
  return make_float4(t5::tf32_rna(v.x - h.x), t5::tf32_rna(v.y - h.y), t5::tf32_rna(v.z - h.z),
                     t5::tf32_rna(v.w - h.w));
}
__device__ __forceinline__ void put_split(unsigned char* hi, unsigned char* lo, uint32_t off, float4 v) {
  const float4 h = split_hi(v);
  *reinterpret_cast<float4*>(hi + off) = h;
  *reinterpret_cast<float4*>(lo + off) = split_lo(v, h);
}

__global__ void __launch_bounds__(NT, 3) k_eig_apply_tc(const EigProb* __restrict__ probs, int round, int phase,
                                                        int* __restrict__ err) {
  const EigProb P = probs[blockIdx.y];
  if (!P.active || round >= P.nb - 1) return;
  const int nb = P.nb, h = nb / 2;
  const long long np = P.npad;
  // ---- which tile: kind 0 = V rows, 1 = G phase 0, 2 = G phase 1 ----
  int kind, col, r0 = -1, r1 = -1;
  {
    int x = blockIdx.x;
    if (phase == 0) {
      const int nrt = (int)((np + TM - 1) / TM), nV = nrt * h;
      if (x < nV) {
        kind = 0; col = x / nrt; r0 = x % nrt;
      } else {
        x -= nV;
        int Q = 0;
        while (Q < h && x >= (Q + 2) / 2) { x -= (Q + 2) / 2; Q++; }
        if (Q >= h) return;
        kind = 1; col = Q; r0 = 2 * x; r1 = 2 * x + 1 <= Q ? 2 * x + 1 : -1;
      }
    } else {
      int Pc = 0;
      while (Pc < h && x >= (h - Pc + 1) / 2) { x -= (h - Pc + 1) / 2; Pc++; }
      if (Pc >= h) return;
      kind = 2; col = Pc; r0 = Pc + 2 * x; r1 = r0 + 1 < h ? r0 + 1 : -1;
    }
  }
  auto rotated = [&](int p) { return !P.jflag || P.jflag[p] != 0; };
  float2* G = reinterpret_cast<float2*>(P.G);
  float2* V = reinterpret_cast<float2*>(P.V);
  float2* T = reinterpret_cast<float2*>(P.T);
  const float2* Jc = reinterpret_cast<const float2*>(P.J) + (long long)col * 4096;
  PairIdx pc, pr0, pr1;
  pair_blocks(round, col, nb, pc.a, pc.b);
  if (kind >= 1) {
    pair_blocks(round, r0, nb, pr0.a, pr0.b);
    if (r1 >= 0) pair_blocks(round, r1, nb, pr1.a, pr1.b);
  }
  const int t = threadIdx.x;
  const int half = t >> 6, l = t & 63;
  bool f0 = true, f1 = true;   // phase 1: the row pairs rotated (T holds their column)
  if (kind <= 1) {
    if (!rotated(col)) return;
  } else {
    f0 = rotated(r0);
    f1 = r1 >= 0 && rotated(r1);
    if (!rotated(col)) {
      // only the row side rotated: Y_QP = T_PQ^H, no product
      const int Qx = half ? r1 : r0;
      if (Qx >= 0 && (half ? f1 : f0)) {
        const PairIdx& pq = half ? pr1 : pr0;
        const long long gq = pq(l);
        for (int p = 0; p < 64; p++) {
          const long long gp = pc(p);
          const float2 v = T[gp * np + gq];
          G[gq * np + gp] = make_float2(v.x, -v.y);
          G[gp * np + gq] = v;
        }
      }
      return;
    }
  }
  // ---- row of this thread ----
  bool valid;
  long long grow = 0;              // kinds 0/1: global row; kind 2: global index of q
  const float2* xsrc;              // source of the X element rows
  if (kind == 0) {
    grow = (long long)r0 * TM + t;
    valid = grow < np;
    xsrc = V;
  } else if (kind == 1) {
    const int rp = half ? r1 : r0;
    valid = rp >= 0;
    grow = valid ? (half ? pr1 : pr0)(l) : 0;
    xsrc = G;
  } else {
    const int Qx = half ? r1 : r0;
    valid = Qx >= 0;
    grow = valid ? (half ? pr1 : pr0)(l) : 0;
    xsrc = (half ? f1 : f0) ? T : G;
  }

  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  unsigned char* st = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  unsigned char *Ah = st, *Al = st + OPB, *Bh = st + 2 * OPB, *Bl = st + 3 * OPB;
  const int warp = t >> 5;
  if (warp == 0) t5::tmem_alloc(&tmem_base, TMEM_COLS);
  if (t == 0) {
    t5::mbar_init(&bar, 1);
    failed = 0;
  }
  t5::fence_before();
  __syncthreads();
  t5::fence_after();
  const uint32_t tmem = tmem_base;

  float2 xa[KC];   // this thread's row of the next A chunk (16 complex)
  float2 jv[8];    // 8 elements of the next (J - I) chunk
  const int jj = t & 63, kh = t >> 6;
  auto load_chunk = [&](int c) {
    const int k0 = KC * c;
    if (valid) {
      if (kind <= 1) {
        const float4* src = reinterpret_cast<const float4*>(xsrc + grow * np + pc(k0));
#pragma unroll
        for (int i = 0; i < KC / 2; i++) {
          const float4 v = src[i];
          xa[2 * i] = make_float2(v.x, v.y);
          xa[2 * i + 1] = make_float2(v.z, v.w);
        }
      } else {   // A = T_PQ^H: A[q][p] = conj(T[p][q])
#pragma unroll
        for (int i = 0; i < KC; i++) {
          const float2 v = xsrc[(long long)pc(k0 + i) * np + grow];
          xa[i] = make_float2(v.x, -v.y);
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < KC; i++) xa[i] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < 8; i++) {
      const int k = k0 + 8 * kh + i;
      float2 v = Jc[k * 64 + jj];
      if (k == jj) v.x -= 1.f;
      jv[i] = v;
    }
  };
  auto write_chunk = [&]() {
#pragma unroll
    for (int g = 0; g < KC / 2; g++)   // row t, real K 4g .. 4g+3
      put_split(Ah, Al, opoff(t, 4 * g), make_float4(xa[2 * g].x, xa[2 * g].y, xa[2 * g + 1].x, xa[2 * g + 1].y));
    // B'^T rows 2j = (re, -im), 2j+1 = (im, re) at K = 2k, 2k+1; this thread: k = 8 kh .. 8 kh + 7
#pragma unroll
    for (int g = 0; g < 4; g++) {
      const float2 d0 = jv[2 * g], d1 = jv[2 * g + 1];
      const int k = 16 * kh + 4 * g;
      put_split(Bh, Bl, opoff(2 * jj, k), make_float4(d0.x, -d0.y, d1.x, -d1.y));
      put_split(Bh, Bl, opoff(2 * jj + 1, k), make_float4(d0.y, d0.x, d1.y, d1.x));
    }
  };

  load_chunk(0);
  int issued = 0;
  for (int c = 0; c < NCH; c++) {
    if (c > 0 && !t5::mbar_wait(&bar, (uint32_t)((c - 1) & 1), WAIT_LIMIT)) failed = 1;
    write_chunk();
    t5::fence_proxy_async();
    __syncthreads();
    if (failed) break;
    if (c + 1 < NCH) load_chunk(c + 1);
    if (t == 0) {
      t5::fence_after();
      const uint32_t ah = t5::smem_u32(Ah), al = t5::smem_u32(Al), bh = t5::smem_u32(Bh), bl = t5::smem_u32(Bl);
#pragma unroll
      for (int s = 0; s < 4; s++) {   // K = 8 real per instruction: two core matrices
        const uint32_t o = 2u * LBO * s;
        t5::mma_tf32<IDESC>(tmem, t5::desc_noswizzle(al + o, LBO, SBO), t5::desc_noswizzle(bh + o, LBO, SBO),
                            (c > 0 || s > 0) ? 1u : 0u);
        t5::mma_tf32<IDESC>(tmem, t5::desc_noswizzle(ah + o, LBO, SBO), t5::desc_noswizzle(bl + o, LBO, SBO), 1u);
        t5::mma_tf32<IDESC>(tmem, t5::desc_noswizzle(ah + o, LBO, SBO), t5::desc_noswizzle(bh + o, LBO, SBO), 1u);
      }
      t5::mma_commit(&bar);
    }
    issued = c + 1;
  }
  // the last committed chunk (also after a timeout: no MMA may run past the dealloc)
  if (issued > 0 && !t5::mbar_wait(&bar, (uint32_t)((issued - 1) & 1), WAIT_LIMIT)) failed = 1;
  t5::fence_after();
  __syncthreads();
  const bool ok = !failed && issued == NCH;
  // ---- epilogue: Y = X + tensor result, 16 complex per 32-column group ----
  const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
  for (int cg = 0; cg < 4; cg++) {
    float v[32];
    t5::tmem_ld32(taddr + (uint32_t)(cg * 32), v);   // warp-collective: every lane
    if (!ok || !valid) continue;
    if (kind <= 1) {
      const long long base = grow * np + pc(16 * cg);
      const float4* xs = reinterpret_cast<const float4*>(xsrc + base);
      float4* ds = reinterpret_cast<float4*>((kind == 0 ? V : T) + base);
#pragma unroll
      for (int i = 0; i < 8; i++) {
        const float4 x = xs[i];
        ds[i] = make_float4(x.x + v[4 * i], x.y + v[4 * i + 1], x.z + v[4 * i + 2], x.w + v[4 * i + 3]);
      }
    } else {
      const bool diag = (half ? r1 : r0) == col;
      const long long pb = pc(16 * cg);    // 16 consecutive global p indices
      float2 y[16];
#pragma unroll
      for (int i = 0; i < 16; i++) {
        const float2 x = xsrc[(pb + i) * np + grow];
        y[i] = make_float2(x.x + v[2 * i], -x.y + v[2 * i + 1]);
      }
      float4* dq = reinterpret_cast<float4*>(G + grow * np + pb);
#pragma unroll
      for (int i = 0; i < 8; i++) dq[i] = make_float4(y[2 * i].x, y[2 * i].y, y[2 * i + 1].x, y[2 * i + 1].y);
      if (!diag) {
#pragma unroll
        for (int i = 0; i < 16; i++) G[(pb + i) * np + grow] = make_float2(y[i].x, -y[i].y);
      }
    }
  }
  if (ok && t == 0 && P.jflag) {
    // algorithmic work: one 64 x 64 x 64 complex product per valid 64-row half
    int halves = 0;
    if (kind == 0) halves = (int)((np - (long long)r0 * TM) >= 128 ? 2 : 1);
    else halves = 1 + (r1 >= 0 ? 1 : 0);
    atomicAdd(P.off + 2, 8.0 * 64 * 64 * 64 * halves);
  }
  t5::fence_before();
  __syncthreads();
  if (warp == 0) t5::tmem_dealloc(tmem, TMEM_COLS);
  if (failed && t == 0) atomicExch(err, 1);
}

}  // namespace

int eig_apply_tc_smem() { return SMEM_BYTES; }

cudaError_t eig_apply_tc_prepare() {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_eig_apply_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return cudaSuccess;
}

cudaError_t launch_eig_apply_tc(const EigProb* d_probs, int n_probs, int max_nb, int max_npad, int round, int* err,
                                cudaStream_t s) {
  if (n_probs <= 0) return cudaSuccess;
  const cudaError_t e = eig_apply_tc_prepare();
  if (e != cudaSuccess) return e;
  const int h = max_nb / 2, nrt = (max_npad + TM - 1) / TM;
  int nA = nrt * h, nB = 0;
  for (int q = 0; q < h; q++) nA += (q + 2) / 2;
  for (int p = 0; p < h; p++) nB += (h - p + 1) / 2;
  k_eig_apply_tc<<<dim3(nA, n_probs), NT, SMEM_BYTES, s>>>(d_probs, round, 0, err);
  k_eig_apply_tc<<<dim3(nB, n_probs), NT, SMEM_BYTES, s>>>(d_probs, round, 1, err);
  return cudaGetLastError();
}

}  // namespace ctebd
