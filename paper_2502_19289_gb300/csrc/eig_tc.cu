// eig_tc.cu -- one round of the batched block-Jacobi eigensolver (FP32) on the
// 5th-generation tensor cores: G <- J^H G J and V <- V J, where J is the
// round's block-diagonal unitary (one 64 x 64 block J_p per pair of 32-wide
// column blocks, round-robin pairing).
//
// Every product is a complex 128 x 64 x 64 tile product X J_c on tcgen05
// (kind::tf32, M = 128, N = 128 real, K = 128 real, accumulators in tensor
// memory), computed in the form X + X (J_c - I):
//   - the complex product is embedded as a real one: the interleaved rows of X
//     are the real rows of A', and B' holds [[re, im], [-im, re]] blocks of
//     (J_c - I), so A' B' is the interleaved result;
//   - 3xTF32: both operands are split into hi = tf32(x) and lo = tf32(x - hi),
//     and lo*hi + hi*lo + hi*hi accumulate in FP32 in tensor memory, the K
//     chunks spread over ETC_ACCS accumulators that the epilogue sums in FP32
//     (round to nearest);
//   - X itself is added in FP32 in the epilogue, so the tensor-pipe
//     accumulation error scales with |J_c - I|, which vanishes as the sweeps
//     converge.
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
// Persistent kernel: one CTA of 256 threads per SM walks its share of the
// tiles as a software pipeline over (tile, K chunk) units -- K = 64 complex in
// four chunks of 16:
//   - the raw A chunk of unit u + 2 is copied (cp.async, coalesced,
//     XOR-swizzled) while unit u is staged;
//   - unit u is split into hi/lo operands in one of two shared-memory stages
//     while the tensor cores work on unit u - 1 from the other;
//   - tile k accumulates in tensor-memory set k mod 2 while the epilogue of
//     tile k - 1 drains set (k - 1) mod 2, one quarter of its columns per unit
//     (tensor memory -> registers -> shared-memory transpose -> coalesced rows).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "tcgen05.h"

namespace ctebd {
namespace {

// Precision of the tensor-core products (compile time): ETC_PASSES = 3 sums
// lo*hi + hi*lo + hi*hi; 4 adds lo*lo.  ETC_ACCS accumulators per tile take
// the K chunks in turn (1 or 2).
#ifndef ETC_PASSES
#define ETC_PASSES 3
#endif
#ifndef ETC_ACCS
#define ETC_ACCS 2
#endif
// Operand layout in shared memory: 1 = K-major with 128-byte swizzle (each
// 32-wide TF32 K chunk is one 8-row x 128-byte atom per 8 rows); 0 = K-major
// core matrices without swizzle.
#ifndef ETC_SWIZZLE
#define ETC_SWIZZLE 1
#endif

constexpr int TM = 128;                    // rows of a tile
constexpr int KC = 16;                     // complex K per chunk
constexpr int NCH = 4;                     // chunks: K = 64 complex
constexpr int NT = 512;                    // threads per CTA: 8 producer + 8 epilogue warps
constexpr int GT = 256;                    // threads per group
#if !ETC_SWIZZLE
constexpr uint32_t LBO = 128, SBO = 1024;  // core matrices along K / along rows (no-swizzle layout)
#endif
constexpr int OPB = 16 * 1024;             // one 128 x 32 real operand piece
constexpr int STB = 4 * OPB;               // one operand stage: A hi, A lo, B hi, B lo
constexpr int RAWA = 16 * 1024;            // raw A chunk (128 x 16 complex)
constexpr int RAWJ = 8 * 1024;             // raw J chunk (16 x 64 complex)
constexpr int SLOT = RAWA + RAWJ;          // one raw slot of the copy ring
constexpr int EB = 128 * 128;              // epilogue transpose: 128 rows x 16 complex
constexpr int MAXP = 256;                  // problems per launch (descriptors in shared memory)
constexpr int SMEM_BYTES = 2 * STB + 2 * SLOT + EB + MAXP * 64 + 1024;   // + alignment slack
constexpr uint32_t IDESC = t5::idesc_tf32(128, 128);
constexpr uint32_t SET_COLS = 128 * ETC_ACCS;   // tensor-memory columns of one tile
constexpr uint32_t TMEM_COLS = 2 * SET_COLS;    // two tiles in flight
constexpr uint32_t WAIT_LIMIT = 1u << 26;

// byte offset of real element (row, k) of a 128 x 32 K-major operand piece
__device__ __forceinline__ uint32_t opoff(int row, int k) {
#if ETC_SWIZZLE
  return (uint32_t)((row >> 3) * 1024 + ((row & 7) << 7) + ((((k >> 2) ^ (row & 7))) << 4) + ((k & 3) << 2));
#else
  return (uint32_t)((row >> 3) * SBO + (k >> 2) * LBO + ((row & 7) << 4) + ((k & 3) << 2));
#endif
}
// operand descriptor of K step s (8 real) of the piece at shared address a
__device__ __forceinline__ uint64_t opdesc(uint32_t a, int s) {
#if ETC_SWIZZLE
  return t5::desc_sw128(a + 32u * s, 1024);
#else
  return t5::desc_noswizzle(a + 2u * LBO * s, LBO, SBO);
#endif
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

__device__ __forceinline__ void put_split(unsigned char* hi, unsigned char* lo, uint32_t off, float4 v) {
  const float4 h = make_float4(t5::tf32_rna(v.x), t5::tf32_rna(v.y), t5::tf32_rna(v.z), t5::tf32_rna(v.w));
  *reinterpret_cast<float4*>(hi + off) = h;
  *reinterpret_cast<float4*>(lo + off) =
      make_float4(t5::tf32_rna(v.x - h.x), t5::tf32_rna(v.y - h.y), t5::tf32_rna(v.z - h.z), t5::tf32_rna(v.w - h.w));
}

// One tile product in flight: 0 = V rows, 1 = G phase 0, 2 = G phase 1.
struct Tile {
  int valid = 0;
  int kind = 0, col = 0, r0 = -1, r1 = -1;
  int np = 0;   // leading dimension (npad <= 4096)
  PairIdx pc, pr0, pr1;
  bool hv0 = false, hv1 = false, f0 = true, f1 = true;
  float2 *G = nullptr, *V = nullptr, *T = nullptr;
  const float2* J = nullptr;   // J_col (64 x 64 row-major)
  double* off = nullptr;       // applied-flop counter (null: no pair flags)
  __device__ __forceinline__ const float2* xsrc(int hf) const {
    const bool f = hf ? f1 : f0;
    return kind == 0 ? V : (kind == 1 ? G : (f ? T : G));
  }
  __device__ __forceinline__ bool hvalid(int hf) const { return hf ? hv1 : hv0; }
  // global row (kinds 0/1) or global q index (kind 2) of tile row m
  __device__ __forceinline__ long long gidx(int m) const {
    if (kind == 0) return (long long)r0 * TM + m;
    return (m >> 6) ? pr1(m & 63) : pr0(m & 63);
  }
  __device__ __forceinline__ bool row_ok(int m) const {
    return hvalid(m >> 6) && (kind != 0 || (long long)r0 * TM + m < np);
  }
};

// The fields of one problem that the round update reads, with its pair flags
// as a bit mask (bit p: J_p is not the identity), cached in shared memory.
struct ProbDesc {
  int npad, nb, active, pad_;
  float2 *G, *V, *T;
  const float2* J;
  double* off;                 // applied-flop counter, null without pair flags
  unsigned long long flags;
};
static_assert(sizeof(ProbDesc) == 64, "descriptor slot");

// Decode tile index x of problem P in this phase.  Returns 1 for a tile
// product (tl filled), 0 otherwise; a copy-only tile (phase 1, the column pair
// did not rotate, a row pair did) is carried out here by all threads.
__device__ int decode(const ProbDesc& P, int x, int round, int phase, Tile& tl, bool do_copy) {
  tl.valid = 0;
  if (!P.active || round >= P.nb - 1) return 0;
  const int nb = P.nb, h = nb / 2;
  const long long np = P.npad;
  int kind, col, r0 = -1, r1 = -1;
  if (phase == 0) {
    const int nrt = (int)((np + TM - 1) / TM), nV = nrt * h;
    if (x < nV) {
      kind = 0; col = x / nrt; r0 = x % nrt;
    } else {
      x -= nV;
      int Q = 0;
      while (Q < h && x >= (Q + 2) / 2) { x -= (Q + 2) / 2; Q++; }
      if (Q >= h) return 0;
      kind = 1; col = Q; r0 = 2 * x; r1 = 2 * x + 1 <= Q ? 2 * x + 1 : -1;
    }
  } else {
    int Pc = 0;
    while (Pc < h && x >= (h - Pc + 1) / 2) { x -= (h - Pc + 1) / 2; Pc++; }
    if (Pc >= h) return 0;
    kind = 2; col = Pc; r0 = Pc + 2 * x; r1 = r0 + 1 < h ? r0 + 1 : -1;
  }
  auto rotated = [&](int p) { return ((P.flags >> p) & 1ull) != 0; };
  tl.kind = kind; tl.col = col; tl.r0 = r0; tl.r1 = r1; tl.np = (int)np;
  tl.G = P.G;
  tl.V = P.V;
  tl.T = P.T;
  tl.J = P.J + (long long)col * 4096;
  tl.off = P.off;
  pair_blocks(round, col, nb, tl.pc.a, tl.pc.b);
  if (kind >= 1) {
    pair_blocks(round, r0, nb, tl.pr0.a, tl.pr0.b);
    if (r1 >= 0) pair_blocks(round, r1, nb, tl.pr1.a, tl.pr1.b);
  }
  if (kind == 0) {
    tl.hv0 = (long long)r0 * TM < np;
    tl.hv1 = (long long)r0 * TM + 64 < np;
  } else {
    tl.hv0 = true;
    tl.hv1 = r1 >= 0;
  }
  tl.f0 = true;
  tl.f1 = true;
  if (kind <= 1) {
    if (!rotated(col)) return 0;
    tl.valid = 1;
    return 1;
  }
  tl.f0 = rotated(r0);
  tl.f1 = r1 >= 0 && rotated(r1);
  if (rotated(col)) {
    tl.valid = 1;
    return 1;
  }
  // only the row side rotated: Y_QP = T_PQ^H, no product (done by the 256
  // calling threads: thread = one q of one half, half of the p range)
  if (!do_copy) return 0;
  const int t = threadIdx.x & (GT - 1), hf = (t >> 6) & 1, q = t & 63, p0 = (t >> 7) * 32;
  if (tl.hvalid(hf) && (hf ? tl.f1 : tl.f0)) {
    const long long gq = hf ? tl.pr1(q) : tl.pr0(q);
    for (int p = p0; p < p0 + 32; p++) {
      const long long gp = tl.pc(p);
      const float2 v = tl.T[gp * np + gq];
      tl.G[gq * np + gp] = make_float2(v.x, -v.y);
      tl.G[gp * np + gq] = v;
    }
  }
  return 0;
}

__global__ void __launch_bounds__(NT, 1) k_eig_apply_tc(const EigProb* __restrict__ probs, int n_probs,
                                                        int tiles_pp, int round, int phase, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ uint64_t mma_bar[2];    // operand stage s: the MMAs that read it are done
  __shared__ uint64_t acc_full[2];   // accumulator set s: a tile's products are complete
  __shared__ uint64_t acc_empty[2];  // accumulator set s: its epilogue has read it
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  unsigned char* stg = base;                    // two operand stages
  unsigned char* ring = base + 2 * STB;         // two raw slots (A chunk + J chunk)
  unsigned char* E = ring + 2 * SLOT;           // epilogue transpose
  ProbDesc* pd = reinterpret_cast<ProbDesc*>(E + EB);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const bool producer = t < GT;
  const int pt = t & (GT - 1);   // thread index within its group
  // the launch's problem descriptors and pair flags into shared memory (one
  // problem per thread; the flag loads are independent and issued together)
  for (int i = t; i < n_probs; i += NT) {
    const EigProb& P = probs[i];
    ProbDesc d;
    d.npad = P.npad; d.nb = P.nb; d.active = P.active; d.pad_ = 0;
    d.G = reinterpret_cast<float2*>(P.G);
    d.V = reinterpret_cast<float2*>(P.V);
    d.T = reinterpret_cast<float2*>(P.T);
    d.J = reinterpret_cast<const float2*>(P.J);
    d.off = P.jflag ? P.off + 2 : nullptr;
    unsigned long long f = ~0ull;
    if (P.jflag) {
      const int h = P.nb / 2;
      f = 0;
#pragma unroll
      for (int p = 0; p < 64; p++)
        if (p < h && P.jflag[p] != 0) f |= 1ull << p;
    }
    d.flags = f;
    pd[i] = d;
  }
  __syncthreads();

  const long long total = (long long)n_probs * tiles_pp;
  long long tau = blockIdx.x;
  // the next tile product of this CTA; the producer group also carries out the
  // copy-only tiles on the way (both groups walk the same sequence)
  auto next_tile = [&](Tile& tl) {
    tl.valid = 0;
    while (tau < total) {
      const int pi = (int)(tau / tiles_pp), x = (int)(tau % tiles_pp);
      tau += gridDim.x;
      if (decode(pd[pi], x, round, phase, tl, producer)) return;
    }
  };
  Tile cur;
  next_tile(cur);
  // every thread finds a tile product or none (the copies are the producer's):
  // the exit is uniform, and one barrier orders the copies before it
  __syncthreads();
  if (!cur.valid) return;

  if (warp == 0) t5::tmem_alloc(&tmem_base, TMEM_COLS);
  if (t == 0) {
    for (int i = 0; i < 2; i++) {
      t5::mbar_init(&mma_bar[i], 1);
      t5::mbar_init(&acc_full[i], 1);
      t5::mbar_init(&acc_empty[i], GT);
    }
    failed = 0;
  }
  t5::fence_before();
  __syncthreads();
  t5::fence_after();
  const uint32_t tmem = tmem_base;
  auto wait_bar = [&](uint64_t* b, long long n) {   // completion number n of barrier b
    if (!t5::mbar_wait(b, (uint32_t)(n & 1), WAIT_LIMIT)) failed = 1;
  };

  if (producer) {
    // raw A chunk c of tile tl -> ring slot s, 16-byte granules, coalesced, XOR-swizzled:
    //  kinds 0/1: [m (128)][granule j (8) = complex 2j, 2j+1 of the chunk] at m*128 + (j ^ (m & 7))*16
    //  kind 2:    [half (2)][p (16)][granule jq (32) = q 2jq, 2jq+1] at h*8192 + p*512 + (jq ^ (p & 7))*16
    //  J rows 16c .. 16c + 15 of J_col: [k (16)][granule jg (32)] at RAWA + k*512 + (jg ^ (k & 7))*16
    auto fetch = [&](const Tile& tl, int c, int s) {
      unsigned char* slot = ring + s * SLOT;
      const int k0 = KC * c;
#pragma unroll
      for (int i = 0; i < 2; i++) {
        const int idx = i * GT + pt, kl = idx >> 5, jg = idx & 31;
        t5::cp_async16(slot + RAWA + kl * 512 + ((jg ^ (kl & 7)) << 4), tl.J + (k0 + kl) * 64 + 2 * jg, 16);
      }
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const int idx = i * GT + pt;
        unsigned char* dst;
        const float2* src;
        bool ok;
        if (tl.kind <= 1) {
          const int m = idx >> 3, j = idx & 7;
          ok = tl.row_ok(m);
          dst = slot + m * 128 + ((j ^ (m & 7)) << 4);
          src = tl.xsrc(m >> 6) + (ok ? tl.gidx(m) * tl.np + tl.pc(k0) + 2 * j : 0);
        } else {
          const int hh = idx >> 9, pi = (idx >> 5) & 15, jq = idx & 31;
          ok = tl.hvalid(hh);
          dst = slot + hh * 8192 + pi * 512 + ((jq ^ (pi & 7)) << 4);
          src = tl.xsrc(hh) + (ok ? (long long)tl.pc(k0 + pi) * tl.np + (hh ? tl.pr1(2 * jq) : tl.pr0(2 * jq)) : 0);
        }
        t5::cp_async16(dst, src, ok ? 16 : 0);
      }
    };
    const int jj = pt & 63, kq = pt >> 6;
    auto stage = [&](const Tile& tl, int c, int s) {
      const unsigned char* slot = ring + s * SLOT;
      float2 jv[4];    // (J - I)[k][jj] for k = 16c + 4kq .. + 3, from the raw slot
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const int kl = 4 * kq + i;
        float2 v = *reinterpret_cast<const float2*>(slot + RAWA + kl * 512 + (((jj >> 1) ^ (kl & 7)) << 4) +
                                                    (jj & 1) * 8);
        if (KC * c + kl == jj) v.x -= 1.f;
        jv[i] = v;
      }
      unsigned char* Ah = stg + s * STB;
      unsigned char *Al = Ah + OPB, *Bh = Ah + 2 * OPB, *Bl = Ah + 3 * OPB;
#pragma unroll
      for (int i = 0; i < 4; i++) {   // 8 rows x 4 granules per warp: conflict-free operand writes
        const int u = i * 8 + warp, m = (u >> 1) * 8 + (lane & 7), g = (u & 1) * 4 + (lane >> 3);
        float4 v;
        if (tl.kind <= 1) {
          v = *reinterpret_cast<const float4*>(slot + m * 128 + ((g ^ (m & 7)) << 4));
        } else {   // A[q][p] = conj(T[p][q]) for p = 2g, 2g + 1
          const int hh = m >> 6, q = m & 63, jq = q >> 1, o8 = (q & 1) * 8;
          const float2 a = *reinterpret_cast<const float2*>(slot + hh * 8192 + (2 * g) * 512 +
                                                            ((jq ^ ((2 * g) & 7)) << 4) + o8);
          const float2 b = *reinterpret_cast<const float2*>(slot + hh * 8192 + (2 * g + 1) * 512 +
                                                            ((jq ^ ((2 * g + 1) & 7)) << 4) + o8);
          v = make_float4(a.x, -a.y, b.x, -b.y);
        }
        put_split(Ah, Al, opoff(m, 4 * g), v);
      }
      // B'^T rows 2j = (re, -im), 2j+1 = (im, re) at K = 2k, 2k+1; this thread:
      // k = 4 kq .. 4 kq + 3 of the chunk; half of the warp writes its odd row first
      const int sw = (jj >> 2) & 1;
#pragma unroll
      for (int g = 0; g < 2; g++) {
        const float2 d0 = jv[2 * g], d1 = jv[2 * g + 1];
        const int k = 8 * kq + 4 * g;
        const float4 ev = make_float4(d0.x, -d0.y, d1.x, -d1.y), od = make_float4(d0.y, d0.x, d1.y, d1.x);
        put_split(Bh, Bl, opoff(2 * jj + sw, k), sw ? od : ev);
        put_split(Bh, Bl, opoff(2 * jj + 1 - sw, k), sw ? ev : od);
      }
    };
    auto issue = [&](int c, int s, uint32_t set) {   // thread 0
      const uint32_t ah = t5::smem_u32(stg + s * STB), al = ah + OPB, bh = ah + 2 * OPB, bl = ah + 3 * OPB;
      const int acc = c * ETC_ACCS / NCH;
      const bool fresh = c * ETC_ACCS % NCH == 0;
      const uint32_t dt = tmem + set + (uint32_t)(acc * 128);
#pragma unroll
      for (int s4 = 0; s4 < 4; s4++) {   // K = 8 real per instruction
        const uint32_t first = (fresh && s4 == 0) ? 0u : 1u;
#if ETC_PASSES == 4
        t5::mma_tf32<IDESC>(dt, opdesc(al, s4), opdesc(bl, s4), first);
        t5::mma_tf32<IDESC>(dt, opdesc(al, s4), opdesc(bh, s4), 1u);
#else
        t5::mma_tf32<IDESC>(dt, opdesc(al, s4), opdesc(bh, s4), first);
#endif
        t5::mma_tf32<IDESC>(dt, opdesc(ah, s4), opdesc(bl, s4), 1u);
        t5::mma_tf32<IDESC>(dt, opdesc(ah, s4), opdesc(bh, s4), 1u);
      }
    };
    Tile nxt;
    fetch(cur, 0, 0);
    t5::cp_commit();
    fetch(cur, 1, 1);
    t5::cp_commit();
    long long last_issued = -1;
    int ktile = 0;   // tile products started
    for (long long u = 0;; u++) {
      const int c = (int)(u & 3), s = (int)(u & 1);
      t5::cp_wait_group1();                        // this thread's copies of unit u have landed
      if (u >= 2) wait_bar(&mma_bar[s], (u - 2) >> 1);   // operand stage s is free again
      t5::named_sync(1, GT);
      if (failed) break;
      stage(cur, c, s);
      t5::fence_proxy_async();
      t5::named_sync(1, GT);
      if (pt == 0) {
        // the set of tile ktile was last read by the epilogue of tile ktile - 2
        if (c == 0 && ktile >= 2) wait_bar(&acc_empty[ktile & 1], (ktile - 2) >> 1);
        t5::fence_after();
        if (!failed) {
          issue(c, s, (uint32_t)(ktile & 1) * SET_COLS);
          t5::mma_commit(&mma_bar[s]);
          if (c == NCH - 1) t5::mma_commit(&acc_full[ktile & 1]);
        }
      }
      last_issued = u;
      // unit u + 2 into the raw slot just consumed
      if (c == 1) next_tile(nxt);
      if (c < 2) fetch(cur, c + 2, s);
      else if (nxt.valid) fetch(nxt, c - 2, s);
      t5::cp_commit();
      if (c == NCH - 1) {
        cur = nxt;
        nxt.valid = 0;
        ktile++;
        if (!cur.valid) break;
      }
    }
    t5::cp_wait_all();   // no copy in flight past this point
    // every issued MMA has completed before the accumulators are freed
    if (last_issued >= 0) wait_bar(&mma_bar[last_issued & 1], last_issued >> 1);
  } else {
    // ---- epilogue group (8 warps): tile k's set, one quarter of its columns at
    // a time: tensor memory -> registers (row m = lane row of the warp's
    // sub-partition, warp half ch = 8 of the quarter's 16 complex columns) ->
    // shared-memory transpose -> coalesced global rows.  The X values a quarter
    // needs are loaded one quarter ahead (the next tile's first quarter before
    // its products are waited for), so no quarter waits on memory. ----
    const int ew = warp - GT / 32;                     // 0..7
    const int m = (ew & 3) * 32 + lane, ch = ew >> 2;
    // X of quarter c into 4 float4: kinds 0/1 the coalesced granules of this
    // thread (row idx >> 3, granule idx & 7, idx = i * GT + pt); kind 2 the 8
    // conj-transposed elements X[p][q] of its own row m (q), two per float4
    auto xload = [&](const Tile& tl, int c, float4 (&xb)[4]) {
      if (tl.kind <= 1) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
          const int idx = i * GT + pt, mm = idx >> 3, g = idx & 7;
          xb[i] = tl.row_ok(mm) ? *reinterpret_cast<const float4*>(tl.xsrc(mm >> 6) + tl.gidx(mm) * tl.np +
                                                                    tl.pc(16 * c) + 2 * g)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      } else {
        const bool ok = tl.row_ok(m);
        const float2* X2 = tl.xsrc(m >> 6);
        const long long gm = ok ? tl.gidx(m) : 0, pb = tl.pc(16 * c + 8 * ch);
#pragma unroll
        for (int i = 0; i < 4; i++) {
          const float2 a = ok ? X2[(pb + 2 * i) * tl.np + gm] : make_float2(0.f, 0.f);
          const float2 b = ok ? X2[(pb + 2 * i + 1) * tl.np + gm] : make_float2(0.f, 0.f);
          xb[i] = make_float4(a.x, a.y, b.x, b.y);
        }
      }
    };
    // quarter c of tile tl from accumulator set `set`, with its X in xb
    auto quarter = [&](const Tile& tl, int c, uint32_t set, const float4 (&xb)[4], bool ok) {
      float v[16];
      const uint32_t taddr = tmem + ((uint32_t)((ew & 3) * 32) << 16) + set + (uint32_t)(32 * c + 16 * ch);
      t5::tmem_ld16(taddr, v);   // warp-collective
#if ETC_ACCS > 1
      {
        float w16[16];
        t5::tmem_ld16(taddr + 128, w16);
#pragma unroll
        for (int i = 0; i < 16; i++) v[i] = __fadd_rn(v[i], w16[i]);
      }
#endif
      if (tl.kind == 2 && tl.row_ok(m) && ok) {
        // Y[q][p] = conj(T[p][q]) + C[q][p]; the mirror Y[p][q]^* is written along q (coalesced)
        const long long gm = tl.gidx(m), pb = tl.pc(16 * c + 8 * ch);
        const bool diag = ((m >> 6) ? tl.r1 : tl.r0) == tl.col;
#pragma unroll
        for (int i = 0; i < 4; i++) {
          v[4 * i] += xb[i].x;
          v[4 * i + 1] += -xb[i].y;
          v[4 * i + 2] += xb[i].z;
          v[4 * i + 3] += -xb[i].w;
          if (!diag) {
            tl.G[(pb + 2 * i) * tl.np + gm] = make_float2(v[4 * i], -v[4 * i + 1]);
            tl.G[(pb + 2 * i + 1) * tl.np + gm] = make_float2(v[4 * i + 2], -v[4 * i + 3]);
          }
        }
      }
#pragma unroll
      for (int j4 = 0; j4 < 4; j4++) {
        const int g = ch * 4 + j4;
        *reinterpret_cast<float4*>(E + m * 128 + ((g ^ (m & 7)) << 4)) =
            make_float4(v[4 * j4], v[4 * j4 + 1], v[4 * j4 + 2], v[4 * j4 + 3]);
      }
      t5::named_sync(2, GT);
      if (ok) {
        // coalesced rows: 4 rows x 8 granules per warp and step
        float2* dst = tl.kind == 0 ? tl.V : (tl.kind == 1 ? tl.T : tl.G);
#pragma unroll
        for (int i = 0; i < 4; i++) {
          const int idx = i * GT + pt, mm = idx >> 3, g = idx & 7;
          if (!tl.row_ok(mm)) continue;
          const float4 y = *reinterpret_cast<const float4*>(E + mm * 128 + ((g ^ (mm & 7)) << 4));
          const float4 x = tl.kind <= 1 ? xb[i] : make_float4(0.f, 0.f, 0.f, 0.f);
          *reinterpret_cast<float4*>(dst + tl.gidx(mm) * tl.np + tl.pc(16 * c) + 2 * g) =
              make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
        }
      }
      t5::named_sync(2, GT);   // E is rewritten by the next quarter
    };
    int k = 0;
    Tile tl = cur;
    float4 xb[4], xn[4];
    xload(tl, 0, xb);
    for (; tl.valid; k++) {
      const uint32_t set = (uint32_t)(k & 1) * SET_COLS;
      wait_bar(&acc_full[k & 1], k >> 1);
      t5::fence_after();
      const bool ok = !failed;
      Tile nt;   // the next tile: its first quarter's X loads before this tile's last quarter
#pragma unroll 1
      for (int c = 0; c < NCH; c++) {
        if (c < NCH - 1) {
          xload(tl, c + 1, xn);
        } else {
          next_tile(nt);
          if (nt.valid) xload(nt, 0, xn);
        }
        quarter(tl, c, set, xb, ok);
#pragma unroll
        for (int i = 0; i < 4; i++) xb[i] = xn[i];
      }
      if (pt == 0 && tl.off && ok)   // one 64^3 complex product per valid half
        atomicAdd(tl.off, 8.0 * 64 * 64 * 64 * ((tl.hv0 ? 1 : 0) + (tl.hv1 ? 1 : 0)));
      t5::fence_before();
      t5::mbar_arrive(&acc_empty[k & 1]);   // this set may take the tile after next
      if (failed) break;
      tl = nt;
    }
  }
  t5::fence_before();
  __syncthreads();
  t5::fence_after();
  if (warp == 0) t5::tmem_dealloc(tmem, TMEM_COLS);
  if (failed && t == 0) atomicExch(err, 1);
}

}  // namespace

cudaError_t eig_apply_tc_prepare() {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_eig_apply_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_eig_apply_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return cudaSuccess;
}

cudaError_t launch_eig_apply_tc(const EigProb* d_probs, int n_probs, int max_nb, int max_npad, int round, int* err,
                                cudaStream_t s) {
  if (n_probs <= 0) return cudaSuccess;
  cudaError_t e = eig_apply_tc_prepare();
  if (e != cudaSuccess) return e;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  }
  const int h = max_nb / 2, nrt = (max_npad + TM - 1) / TM;
  int nA = nrt * h, nB = 0;
  for (int q = 0; q < h; q++) nA += (q + 2) / 2;
  for (int p = 0; p < h; p++) nB += (h - p + 1) / 2;
  // at most MAXP problems per launch (their descriptors are cached in shared memory)
  for (int p0 = 0; p0 < n_probs; p0 += MAXP) {
    const int np_ = std::min(MAXP, n_probs - p0);
    const long long totA = (long long)nA * np_;
    k_eig_apply_tc<<<(unsigned)std::min<long long>(sms, totA), NT, SMEM_BYTES, s>>>(d_probs + p0, np_, nA, round, 0,
                                                                                    err);
  }
  for (int p0 = 0; p0 < n_probs; p0 += MAXP) {
    const int np_ = std::min(MAXP, n_probs - p0);
    const long long totB = (long long)nB * np_;
    k_eig_apply_tc<<<(unsigned)std::min<long long>(sms, totB), NT, SMEM_BYTES, s>>>(d_probs + p0, np_, nB, round, 1,
                                                                                    err);
  }
  return cudaGetLastError();
}

}  // namespace ctebd
