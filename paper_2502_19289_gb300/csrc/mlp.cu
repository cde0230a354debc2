// mlp.cu -- the learned rank predictor that sizes the sketched split:
// F -> H1 -> H2 -> NB with ReLU, softmax cross-entropy over rank buckets.
// Parameters packed as W1 (H1 x F), b1, W2 (H2 x H1), b2, W3 (NB x H2), b3
// (row-major, FP32).  Forward, loss + gradient and Adam kernels; plus the
// bond-entropy kernel that provides two of the features.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace ctebd {

constexpr int MF = MLP_F, MH1 = MLP_H1, MH2 = MLP_H2, MNB = MLP_NB;
constexpr int MLP_NP = MH1 * MF + MH1 + MH2 * MH1 + MH2 + MNB * MH2 + MNB;

struct MlpView {
  const float *W1, *b1, *W2, *b2, *W3, *b3;
  __device__ explicit MlpView(const float* P) {
    W1 = P; b1 = W1 + MH1 * MF; W2 = b1 + MH1; b2 = W2 + MH2 * MH1; W3 = b2 + MH2; b3 = W3 + MNB * MH2;
  }
};

// one thread per sample; parameters staged in shared memory
__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ params,
                                                     const float* __restrict__ X, int B,
                                                     float* __restrict__ logits) {
  __shared__ float P[MLP_NP];
  for (int i = threadIdx.x; i < MLP_NP; i += blockDim.x) P[i] = params[i];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  MlpView v(P);
  float x[MF], h1[MH1], h2[MH2];
  for (int f = 0; f < MF; f++) x[f] = X[(long long)s * MF + f];
  for (int i = 0; i < MH1; i++) {
    float a = v.b1[i];
    for (int f = 0; f < MF; f++) a = fmaf(v.W1[i * MF + f], x[f], a);
    h1[i] = fmaxf(a, 0.f);
  }
  for (int i = 0; i < MH2; i++) {
    float a = v.b2[i];
    for (int j = 0; j < MH1; j++) a = fmaf(v.W2[i * MH1 + j], h1[j], a);
    h2[i] = fmaxf(a, 0.f);
  }
  for (int i = 0; i < MNB; i++) {
    float a = v.b3[i];
    for (int j = 0; j < MH2; j++) a = fmaf(v.W3[i * MH2 + j], h2[j], a);
    logits[(long long)s * MNB + i] = a;
  }
}

// mean softmax cross-entropy and its gradient w.r.t. every parameter;
// gradients are reduced in shared memory per block, then added to grad
// (which the caller zeroes) with one atomic per parameter per block.
__global__ void __launch_bounds__(128) k_mlp_loss_grad(const float* __restrict__ params,
                                                       const float* __restrict__ X,
                                                       const int* __restrict__ y, int B,
                                                       float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ float Gs[MLP_NP];
  for (int i = threadIdx.x; i < MLP_NP; i += blockDim.x) Gs[i] = 0.f;
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  MlpView v(params);
  float* gW1 = Gs; float* gb1 = gW1 + MH1 * MF; float* gW2 = gb1 + MH1; float* gb2 = gW2 + MH2 * MH1;
  float* gW3 = gb2 + MH2; float* gb3 = gW3 + MNB * MH2;
  float lsum = 0.f;
  if (s < B) {
    float x[MF], h1[MH1], h2[MH2], d3[MNB], d2[MH2];
    for (int f = 0; f < MF; f++) x[f] = X[(long long)s * MF + f];
    for (int i = 0; i < MH1; i++) {
      float a = v.b1[i];
      for (int f = 0; f < MF; f++) a = fmaf(v.W1[i * MF + f], x[f], a);
      h1[i] = fmaxf(a, 0.f);
    }
    for (int i = 0; i < MH2; i++) {
      float a = v.b2[i];
      for (int j = 0; j < MH1; j++) a = fmaf(v.W2[i * MH1 + j], h1[j], a);
      h2[i] = fmaxf(a, 0.f);
    }
    float mx = -INFINITY;
    for (int i = 0; i < MNB; i++) {
      float a = v.b3[i];
      for (int j = 0; j < MH2; j++) a = fmaf(v.W3[i * MH2 + j], h2[j], a);
      d3[i] = a;
      mx = fmaxf(mx, a);
    }
    float se = 0.f;
    for (int i = 0; i < MNB; i++) se += expf(d3[i] - mx);
    const int yi = y[s];
    lsum = logf(se) + mx - d3[yi];
    const float invB = 1.f / (float)B;
    for (int i = 0; i < MNB; i++) d3[i] = (expf(d3[i] - mx) / se - (i == yi ? 1.f : 0.f)) * invB;
    for (int i = 0; i < MNB; i++) {
      atomicAdd(&gb3[i], d3[i]);
      for (int j = 0; j < MH2; j++) atomicAdd(&gW3[i * MH2 + j], d3[i] * h2[j]);
    }
    for (int j = 0; j < MH2; j++) {
      float a = 0.f;
      for (int i = 0; i < MNB; i++) a = fmaf(v.W3[i * MH2 + j], d3[i], a);
      d2[j] = h2[j] > 0.f ? a : 0.f;
    }
    for (int i = 0; i < MH2; i++) {
      if (d2[i] == 0.f) continue;
      atomicAdd(&gb2[i], d2[i]);
      for (int j = 0; j < MH1; j++) atomicAdd(&gW2[i * MH1 + j], d2[i] * h1[j]);
    }
    for (int j = 0; j < MH1; j++) {
      float a = 0.f;
      for (int i = 0; i < MH2; i++) a = fmaf(v.W2[i * MH1 + j], d2[i], a);
      const float d1 = h1[j] > 0.f ? a : 0.f;
      if (d1 == 0.f) continue;
      atomicAdd(&gb1[j], d1);
      for (int f = 0; f < MF; f++) atomicAdd(&gW1[j * MF + f], d1 * x[f]);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < MLP_NP; i += blockDim.x)
    if (Gs[i] != 0.f) atomicAdd(&grad[i], Gs[i]);
  for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if ((threadIdx.x & 31) == 0 && lsum != 0.f) atomicAdd(loss, lsum / (float)B);
}

// Adam (Kingma & Ba 2015) with bias correction; t is the 1-based step
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, int t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.f - powf(b1, (float)t)), vh = vi / (1.f - powf(b2, (float)t));
  p[i] -= lr * mh / (sqrtf(vh) + eps);
}

cudaError_t launch_mlp_forward(const float* params, const float* X, int B, float* logits, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_mlp_forward<<<(B + 127) / 128, 128, 0, s>>>(params, X, B, logits);
  return cudaGetLastError();
}

cudaError_t launch_mlp_loss_grad(const float* params, const float* X, const int* y, int B, float* grad,
                                 float* loss, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  k_mlp_loss_grad<<<(B + 127) / 128, 128, 0, s>>>(params, X, y, B, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, int t, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_adam<<<(n + 255) / 256, 256, 0, s>>>(p, g, m, v, n, lr, 0.9f, 0.999f, 1e-8f, t);
  return cudaGetLastError();
}

int mlp_nparams() { return MLP_NP; }

// von Neumann entropy in bits of every bond spectrum: S_b = -sum l^2 log2 l^2
__global__ void k_entropy(const double* const* __restrict__ lams, const int* __restrict__ chi, int nb,
                          double* __restrict__ out) {
  const int b = blockIdx.x;
  if (b >= nb) return;
  const double* l = lams[b];
  double acc = 0;
  for (int i = threadIdx.x; i < chi[b]; i += blockDim.x) {
    const double p = l[i] * l[i];
    if (p > 0) acc -= p * log2(p);
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double part[4];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) out[b] = part[0] + part[1] + part[2] + part[3];
}

cudaError_t launch_entropy(const double* const* d_lams, const int* d_chi, int nb, double* d_out, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  k_entropy<<<nb, 128, 0, s>>>(d_lams, d_chi, nb, d_out);
  return cudaGetLastError();
}

}  // namespace ctebd
