// sketch.cu -- kernels of the randomized range finder used by the sketched
// split: counter-based Gaussian test matrices, row scaling by the Schmidt
// weights, the FP64 Cholesky + triangular inverse of CholeskyQR, and the
// FP64 weighted Frobenius norm used by the residual (tail) check.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "internal.h"

namespace ctebd {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): a 10-round counter-based generator.  Counter =
// (element pair index, stream id), key = 64-bit seed.  Two complex standard
// normals per counter by the Box-Muller transform.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t lo0 = M0 * c[0], hi0 = __umulhi(M0, c[0]);
  const uint32_t lo1 = M1 * c[2], hi1 = __umulhi(M1, c[2]);
  const uint32_t n0 = hi1 ^ c[1] ^ k[0], n1 = lo1, n2 = hi0 ^ c[3] ^ k[1], n3 = lo0;
  c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

__device__ __forceinline__ void philox10(uint32_t c[4], uint64_t seed) {
  uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int r = 0; r < 10; r++) {
    philox_round(c, k);
    k[0] += 0x9E3779B9u;
    k[1] += 0xBB67AE85u;
  }
}

__global__ void k_gauss(float2* __restrict__ out, long long count, uint64_t seed, uint64_t stream) {
  const long long pairs = (count + 1) / 2;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < pairs;
       p += (long long)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)p, (uint32_t)(p >> 32), (uint32_t)stream, (uint32_t)(stream >> 32)};
    philox10(c, seed);
    const float inv = 2.3283064365386963e-10f;  // 2^-32
    #pragma unroll
    for (int h = 0; h < 2; h++) {
      const float u1 = ((float)c[2 * h] + 0.5f) * inv, u2 = ((float)c[2 * h + 1] + 0.5f) * inv;
      const float rr = sqrtf(-2.0f * logf(u1));
      float s, co;
      sincospif(2.0f * u2, &s, &co);
      const long long e = 2 * p + h;
      if (e < count) out[e] = make_float2(rr * co, rr * s);
    }
  }
}

cudaError_t launch_gauss(void* out, long long count, uint64_t seed, uint64_t stream, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  long long g = (count / 2 + 255) / 256;
  k_gauss<<<(unsigned)(g > 4096 ? 4096 : (g < 1 ? 1 : g)), 256, 0, s>>>((float2*)out, count, seed, stream);
  return cudaGetLastError();
}

// X[r][c] *= lam[r >> shift] for r < rows, c < cols (row-major, ld)
__global__ void k_rowscale(const RowScaleProb* __restrict__ probs) {
  const RowScaleProb P = probs[blockIdx.y];
  float2* X = (float2*)P.X;
  const long long tot = (long long)P.rows * P.cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / P.cols, c = e % P.cols;
    const float w = (float)P.lam[r >> P.shift];
    float2 v = X[r * P.ld + c];
    v.x *= w; v.y *= w;
    X[r * P.ld + c] = v;
  }
}

cudaError_t launch_rowscale(const RowScaleProb* d_probs, int n, long long max_elems, cudaStream_t s) {
  if (n <= 0 || max_elems <= 0) return cudaSuccess;
  long long g = (max_elems + 255) / 256;
  k_rowscale<<<dim3((unsigned)(g > 4096 ? 4096 : g), n), 256, 0, s>>>(d_probs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CholeskyQR building block, FP64: A = G + s I (s = shift_rel * trace G),
// A = L L^H (right-looking, lower), then X = (L^{-1})^H (upper triangular,
// written as complex64) so that Q = Y X has orthonormal columns.  With
// dead_rel > 0 the factorisation is rank-revealing: a pivot below
// dead_rel * trace marks its column as numerically dependent on the previous
// ones; the column is dropped (zero column of X, so a zero column of Q).
// One CTA per problem.  status: 0 ok, 2 non-finite input.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_chol_inv(const CholProb* __restrict__ probs) {
  const CholProb P = probs[blockIdx.x];
  const int l = P.l;
  const float2* G = (const float2*)P.G;
  double2* A = P.work;                       // l x l, lower triangle
  double2* Li = P.work + (long long)l * l;   // l x l, lower triangle of L^{-1}
  __shared__ double red[32];
  __shared__ double dpiv;
  __shared__ int bad, dead_k;
  int* dead = P.dead;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nth >> 5;
  double tr = 0;
  for (int i = tid; i < l; i += nth) tr += (double)G[(long long)i * P.ldg + i].x;
  for (int o = 16; o; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  if (lane == 0) red[warp] = tr;
  if (tid == 0) bad = 0;
  __syncthreads();
  if (tid == 0) {
    double t = 0;
    for (int w = 0; w < nw; w++) t += red[w];
    red[0] = t;
  }
  __syncthreads();
  const double shift = P.shift_rel * red[0];
  const double dead_thr = P.dead_rel * red[0];
  for (long long e = tid; e < (long long)l * l; e += nth) {
    const int i = (int)(e / l), j = (int)(e % l);
    if (j > i) continue;
    const float2 g = G[(long long)i * P.ldg + j];
    A[e] = make_double2((double)g.x + (i == j ? shift : 0.0), i == j ? 0.0 : (double)g.y);
  }
  __syncthreads();
  for (int k = 0; k < l; k++) {
    if (tid == 0) {
      const double piv = A[(long long)k * l + k].x;
      if (!isfinite(piv)) bad = 2;
      dead_k = !(piv > dead_thr) || !(piv > 0.0);
      dead[k] = dead_k;
      dpiv = dead_k ? 1.0 : sqrt(piv);
      A[(long long)k * l + k] = make_double2(dpiv, 0.0);
    }
    __syncthreads();
    if (bad) break;
    const double inv = 1.0 / dpiv;
    for (int i = k + 1 + tid; i < l; i += nth) {
      double2 v = A[(long long)i * l + k];
      if (dead_k) { v.x = 0; v.y = 0; } else { v.x *= inv; v.y *= inv; }
      A[(long long)i * l + k] = v;
    }
    __syncthreads();
    for (int i = k + 1 + warp; i < l; i += nw) {
      const double2 aik = A[(long long)i * l + k];
      for (int j = k + 1 + lane; j <= i; j += 32) {
        const double2 ajk = A[(long long)j * l + k];
        double2 v = A[(long long)i * l + j];
        // v -= aik * conj(ajk)
        v.x -= aik.x * ajk.x + aik.y * ajk.y;
        v.y -= aik.y * ajk.x - aik.x * ajk.y;
        A[(long long)i * l + j] = v;
      }
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) *P.status = bad;
    return;
  }
  // L^{-1}: column j by forward substitution, one warp per column
  for (int j = warp; j < l; j += nw) {
    for (int i = j; i < l; i++) {
      double sx = 0, sy = 0;
      for (int t = j + lane; t < i; t += 32) {
        const double2 a = A[(long long)i * l + t], x = Li[(long long)t * l + j];
        sx += a.x * x.x - a.y * x.y;
        sy += a.x * x.y + a.y * x.x;
      }
      for (int o = 16; o; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
      }
      if (lane == 0) {
        const double d = A[(long long)i * l + i].x;
        const double rx = ((i == j ? 1.0 : 0.0) - sx) / d, ry = -sy / d;
        Li[(long long)i * l + j] = make_double2(rx, ry);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  float2* X = (float2*)P.X;
  for (long long e = tid; e < (long long)l * l; e += nth) {
    const int i = (int)(e / l), j = (int)(e % l);
    float2 v = make_float2(0.f, 0.f);
    if (i <= j && !dead[j] && !dead[i]) {
      const double2 li = Li[(long long)j * l + i];
      v = make_float2((float)li.x, (float)-li.y);
    }
    X[(long long)i * P.ldx + j] = v;
  }
  if (tid == 0) *P.status = 0;
}

cudaError_t launch_chol_inv(const CholProb* d_probs, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_chol_inv<<<n, 512, 0, s>>>(d_probs);
  return cudaGetLastError();
}

// Schmidt-weighted squared Frobenius norm of a row-major complex64 matrix:
// out += sum_r lam[r >> shift]^2 sum_c |X[r][c]|^2  (FP64 accumulation)
__global__ void k_wnorm(const WNormProb* __restrict__ probs) {
  const WNormProb P = probs[blockIdx.y];
  const float2* X = (const float2*)P.X;
  const long long tot = (long long)P.rows * P.cols;
  double acc = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / P.cols, c = e % P.cols;
    const float2 v = X[r * P.ld + c];
    const double w = P.lam[r >> P.shift];
    acc += w * w * ((double)v.x * v.x + (double)v.y * v.y);
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += part[w];
    atomicAdd(P.out, t);
  }
}

cudaError_t launch_wnorm(const WNormProb* d_probs, int n, long long max_elems, cudaStream_t s) {
  if (n <= 0 || max_elems <= 0) return cudaSuccess;
  long long g = (max_elems + 255) / 256;
  k_wnorm<<<dim3((unsigned)(g > 1024 ? 1024 : g), n), 256, 0, s>>>(d_probs);
  return cudaGetLastError();
}

}  // namespace ctebd
