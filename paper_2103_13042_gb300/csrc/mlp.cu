// Learned tau: the FP32 network x(65) -> Linear(65,64) -> GELU -> Linear(64,64)
// -> GELU -> Linear(64,1) -> y = log10(tau / (||A||_F ||B||_F)), with x the
// 64-bin histogram of log2 relative norm products (each bin a fraction of
// all bm * bk * bn triples) followed by log10 of the target relative error.  The
// paper chooses tau by a valid-ratio search (Section 3.5.2); the network
// replaces that search with one forward pass, and plain bisection on the
// achieved error stays the fallback.
//
// Parameters: one flat FP32 array, W1 (64 x 65, row-major out x in), b1,
// W2 (64 x 64), b2, W3 (1 x 64), b3: 8449 values.  GELU is the exact
// 0.5 z (1 + erf(z / sqrt 2)).
//
// Kernels: a batched forward (one thread per sample, weights in shared
// memory), the pinball-loss gradient over a sample set, one Adam step, and a
// persistent training loop (one CTA runs every step: per minibatch, forward,
// backward and Adam, the weights kept in shared memory between steps).  The
// network is tiny (6.5 MFLOP per 256-sample step), so one CTA with the
// weights on chip beats any multi-CTA split that would need grid-wide
// reductions of the 8449 gradients.
#include <cmath>

#include "plan.cuh"

namespace spamm {
namespace mlp {

constexpr int kIn = 65, kH = 64;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH,
              kOffB2 = kOffW2 + kH * kH, kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH;
constexpr int kParams = kOffB3 + 1;   // 8449
static_assert(kParams == 8449, "parameter count");

constexpr int kThreads = 256;
constexpr int kChunk = 32;                                   // samples per backward chunk
constexpr int kOwned = (kParams + kThreads - 1) / kThreads;  // 34 parameters per thread

__device__ __forceinline__ float gelu(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// y for one sample x[65] with the weights W (shared or global).
__device__ float forward_one(const float* __restrict__ W, const float* __restrict__ x) {
  float h1[kH];
#pragma unroll 4
  for (int o = 0; o < kH; ++o) {
    float z = W[kOffB1 + o];
    for (int i = 0; i < kIn; ++i) z = fmaf(W[kOffW1 + o * kIn + i], x[i], z);
    h1[o] = gelu(z);
  }
  float y = W[kOffB3];
  for (int o = 0; o < kH; ++o) {
    float z = W[kOffB2 + o];
#pragma unroll 8
    for (int i = 0; i < kH; ++i) z = fmaf(W[kOffW2 + o * kH + i], h1[i], z);
    y = fmaf(W[kOffW3 + o], gelu(z), y);
  }
  return y;
}

__global__ void __launch_bounds__(128) forward_kernel(const float* __restrict__ Wg,
                                                      const float* __restrict__ X, int count,
                                                      float* __restrict__ Y) {
  extern __shared__ float W[];
  for (int q = threadIdx.x; q < kParams; q += blockDim.x) W[q] = Wg[q];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= count) return;
  float x[kIn];
  for (int i = 0; i < kIn; ++i) x[i] = X[(int64_t)s * kIn + i];
  Y[s] = forward_one(W, x);
}

// Shared-memory work area of the gradient pass (after the kParams weights).
struct Work {
  float* X;    // [kChunk][kIn]
  float* Z1;   // [kChunk][kH]
  float* Z2;
  float* H1;
  float* H2;
  float* G1;
  float* G2;
  float* g3;   // [kChunk]
  float* loss; // [1]
};
constexpr size_t kWorkFloats = (size_t)kChunk * kIn + 6 * (size_t)kChunk * kH + kChunk + 4;
constexpr size_t kSmemBytes = ((size_t)kParams + 3 + kWorkFloats) * sizeof(float);

__device__ __forceinline__ Work carve(float* base) {
  Work w;
  float* p = base;
  w.X = p;  p += kChunk * kIn;
  w.Z1 = p; p += kChunk * kH;
  w.Z2 = p; p += kChunk * kH;
  w.H1 = p; p += kChunk * kH;
  w.H2 = p; p += kChunk * kH;
  w.G1 = p; p += kChunk * kH;
  w.G2 = p; p += kChunk * kH;
  w.g3 = p; p += kChunk;
  w.loss = p;
  return w;
}

// Adds to acc[] (this thread's parameters t + 256 r) the gradient of
// (1 / norm) sum_s rho_q(Y[s] - y[s]) over the samples idx[0..count) (or
// 0..count when idx is null); returns nothing, adds the loss into *w.loss.
// Every thread of the CTA calls it.
__device__ void accumulate_grad(const float* __restrict__ W, const float* __restrict__ Xg,
                                const float* __restrict__ Yg, const int* __restrict__ idx,
                                int count, float norm, float q, Work w, float (&acc)[kOwned]) {
  const int t = threadIdx.x;
  for (int c0 = 0; c0 < count; c0 += kChunk) {
    const int nc = min(kChunk, count - c0);
    // samples of the chunk
    for (int e = t; e < kChunk * kIn; e += kThreads) {
      const int s = e / kIn, i = e % kIn;
      float v = 0.0f;
      if (s < nc) {
        const int row = idx ? idx[c0 + s] : c0 + s;
        v = Xg[(int64_t)row * kIn + i];
      }
      w.X[e] = v;
    }
    __syncthreads();
    // layer 1: thread (s, o) pairs, o fastest
    for (int e = t; e < kChunk * kH; e += kThreads) {
      const int s = e / kH, o = e % kH;
      float z = W[kOffB1 + o];
      for (int i = 0; i < kIn; ++i) z = fmaf(W[kOffW1 + o * kIn + i], w.X[s * kIn + i], z);
      w.Z1[e] = z;
      w.H1[e] = gelu(z);
    }
    __syncthreads();
    for (int e = t; e < kChunk * kH; e += kThreads) {
      const int s = e / kH, o = e % kH;
      float z = W[kOffB2 + o];
      for (int i = 0; i < kH; ++i) z = fmaf(W[kOffW2 + o * kH + i], w.H1[s * kH + i], z);
      w.Z2[e] = z;
      w.H2[e] = gelu(z);
    }
    __syncthreads();
    // output and d loss / d y (pinball slope q for r > 0, q - 1 otherwise)
    if (t < kChunk) {
      float g = 0.0f, l = 0.0f;
      if (t < nc) {
        float y = W[kOffB3];
        for (int i = 0; i < kH; ++i) y = fmaf(W[kOffW3 + i], w.H2[t * kH + i], y);
        const int row = idx ? idx[c0 + t] : c0 + t;
        const float r = Yg[row] - y;
        g = -(r > 0.0f ? q : q - 1.0f) / norm;
        l = fmaxf(q * r, (q - 1.0f) * r) / norm;
      }
      w.g3[t] = g;
      for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
      if (t == 0) *w.loss += l;
    }
    __syncthreads();
    for (int e = t; e < kChunk * kH; e += kThreads) {
      const int s = e / kH, o = e % kH;
      w.G2[e] = w.g3[s] * W[kOffW3 + o] * gelu_grad(w.Z2[e]);
    }
    __syncthreads();
    for (int e = t; e < kChunk * kH; e += kThreads) {
      const int s = e / kH, o = e % kH;
      float g = 0.0f;
      for (int j = 0; j < kH; ++j) g = fmaf(w.G2[s * kH + j], W[kOffW2 + j * kH + o], g);
      w.G1[e] = g * gelu_grad(w.Z1[e]);
    }
    __syncthreads();
    // this thread's parameters: sums over the chunk's samples
#pragma unroll
    for (int r = 0; r < kOwned; ++r) {
      const int p = t + r * kThreads;
      if (p >= kParams) break;
      float g = 0.0f;
      if (p < kOffB1) {
        const int o = p / kIn, i = p % kIn;
        for (int s = 0; s < nc; ++s) g = fmaf(w.G1[s * kH + o], w.X[s * kIn + i], g);
      } else if (p < kOffW2) {
        const int o = p - kOffB1;
        for (int s = 0; s < nc; ++s) g += w.G1[s * kH + o];
      } else if (p < kOffB2) {
        const int o = (p - kOffW2) / kH, i = (p - kOffW2) % kH;
        for (int s = 0; s < nc; ++s) g = fmaf(w.G2[s * kH + o], w.H1[s * kH + i], g);
      } else if (p < kOffW3) {
        const int o = p - kOffB2;
        for (int s = 0; s < nc; ++s) g += w.G2[s * kH + o];
      } else if (p < kOffB3) {
        const int i = p - kOffW3;
        for (int s = 0; s < nc; ++s) g = fmaf(w.g3[s], w.H2[s * kH + i], g);
      } else {
        for (int s = 0; s < nc; ++s) g += w.g3[s];
      }
      acc[r] += g;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads, 1)
    grad_kernel(const float* __restrict__ Wg, const float* __restrict__ X,
                const float* __restrict__ Y, int count, float q, float* __restrict__ grad,
                float* __restrict__ loss) {
  extern __shared__ float sm[];
  float* W = sm;
  Work w = carve(sm + kParams + 3);
  for (int p = threadIdx.x; p < kParams; p += kThreads) W[p] = Wg[p];
  if (threadIdx.x == 0) *w.loss = 0.0f;
  __syncthreads();
  float acc[kOwned];
#pragma unroll
  for (int r = 0; r < kOwned; ++r) acc[r] = 0.0f;
  accumulate_grad(W, X, Y, nullptr, count, (float)count, q, w, acc);
#pragma unroll
  for (int r = 0; r < kOwned; ++r) {
    const int p = threadIdx.x + r * kThreads;
    if (p < kParams) grad[p] = acc[r];
  }
  if (threadIdx.x == 0) *loss = *w.loss;
}

// Adam with bias-corrected moments (beta1 0.9, beta2 0.999, eps 1e-8).
__device__ __forceinline__ void adam_update(float& w, float g, float& m, float& v, float lr,
                                            float c1, float c2) {
  m = 0.9f * m + 0.1f * g;
  v = 0.999f * v + 0.001f * g * g;
  const float mhat = m / c1, vhat = v / c2;
  w -= lr * mhat / (sqrtf(vhat) + 1e-8f);
}

__global__ void adam_kernel(float* __restrict__ W, const float* __restrict__ grad,
                            float* __restrict__ m, float* __restrict__ v, int t, float lr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  const float c1 = 1.0f - powf(0.9f, (float)t), c2 = 1.0f - powf(0.999f, (float)t);
  float w = W[p], mm = m[p], vv = v[p];
  adam_update(w, grad[p], mm, vv, lr, c1, c2);
  W[p] = w;
  m[p] = mm;
  v[p] = vv;
}

// `steps` Adam steps; step s uses the samples idx[s * batch .. (s + 1) * batch).
__global__ void __launch_bounds__(kThreads, 1)
    train_kernel(float* __restrict__ Wg, float* __restrict__ mg, float* __restrict__ vg, int t0,
                 const float* __restrict__ X, const float* __restrict__ Y,
                 const int* __restrict__ idx, int steps, int batch, float lr, float q,
                 float* __restrict__ loss_hist) {
  extern __shared__ float sm[];
  float* W = sm;
  Work w = carve(sm + kParams + 3);
  const int t = threadIdx.x;
  for (int p = t; p < kParams; p += kThreads) W[p] = Wg[p];
  float m[kOwned], v[kOwned];
#pragma unroll
  for (int r = 0; r < kOwned; ++r) {
    const int p = t + r * kThreads;
    m[r] = p < kParams ? mg[p] : 0.0f;
    v[r] = p < kParams ? vg[p] : 0.0f;
  }
  __syncthreads();
  for (int s = 0; s < steps; ++s) {
    if (t == 0) *w.loss = 0.0f;
    __syncthreads();
    float acc[kOwned];
#pragma unroll
    for (int r = 0; r < kOwned; ++r) acc[r] = 0.0f;
    accumulate_grad(W, X, Y, idx + (int64_t)s * batch, batch, (float)batch, q, w, acc);
    const int step = t0 + s + 1;
    const float c1 = 1.0f - powf(0.9f, (float)step), c2 = 1.0f - powf(0.999f, (float)step);
#pragma unroll
    for (int r = 0; r < kOwned; ++r) {
      const int p = t + r * kThreads;
      if (p < kParams) adam_update(W[p], acc[r], m[r], v[r], lr, c1, c2);
    }
    if (t == 0 && loss_hist) loss_hist[s] = *w.loss;
    __syncthreads();
  }
  for (int p = t; p < kParams; p += kThreads) Wg[p] = W[p];
#pragma unroll
  for (int r = 0; r < kOwned; ++r) {
    const int p = t + r * kThreads;
    if (p < kParams) {
      mg[p] = m[r];
      vg[p] = v[r];
    }
  }
}

// Features of every instance from its histogram and the network's tau:
// tau = 10^y * ||A||_F ||B||_F, target relative error in Inst::target_rel.
__global__ void __launch_bounds__(128) tau_kernel(InstRef R, const float* __restrict__ Wg,
                                                  float* __restrict__ feats,
                                                  double* __restrict__ tau) {
  extern __shared__ float W[];
  for (int q = threadIdx.x; q < kParams; q += blockDim.x) W[q] = Wg[q];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= R.count) return;
  const Inst& in = R.at(i);
  const double cube = (double)in.bm * (double)in.bk * (double)in.bn;
  float x[kIn];
  for (int b = 0; b < kHistBins; ++b) x[b] = (float)((double)in.pd->hist[b] / cube);
  x[kHistBins] = (float)log10(in.target_rel);
  if (feats)
    for (int b = 0; b < kIn; ++b) feats[(int64_t)i * kIn + b] = x[b];
  const float y = forward_one(W, x);
  tau[i] = exp10((double)y) * (in.pd->norm_a * in.pd->norm_b);
}

}  // namespace mlp

int mlp_param_count() { return mlp::kParams; }

cudaError_t launch_mlp_forward(const float* W, const float* X, int count, float* Y,
                               cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = mlp::kParams * sizeof(float);
  cudaFuncSetAttribute(mlp::forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  mlp::forward_kernel<<<(count + 127) / 128, 128, smem, s>>>(W, X, count, Y);
  return cudaPeekAtLastError();
}

cudaError_t launch_mlp_grad(const float* W, const float* X, const float* Y, int count, float q,
                            float* grad, float* loss, cudaStream_t s) {
  cudaFuncSetAttribute(mlp::grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)mlp::kSmemBytes);
  mlp::grad_kernel<<<1, mlp::kThreads, mlp::kSmemBytes, s>>>(W, X, Y, count, q, grad, loss);
  return cudaPeekAtLastError();
}

cudaError_t launch_mlp_adam(float* W, const float* grad, float* m, float* v, int t, float lr,
                            cudaStream_t s) {
  mlp::adam_kernel<<<(mlp::kParams + 255) / 256, 256, 0, s>>>(W, grad, m, v, t, lr);
  return cudaPeekAtLastError();
}

cudaError_t launch_mlp_train(float* W, float* m, float* v, int t0, const float* X, const float* Y,
                             const int* idx, int steps, int batch, float lr, float q,
                             float* loss_hist, cudaStream_t s) {
  if (steps <= 0) return cudaSuccess;
  cudaFuncSetAttribute(mlp::train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)mlp::kSmemBytes);
  mlp::train_kernel<<<1, mlp::kThreads, mlp::kSmemBytes, s>>>(W, m, v, t0, X, Y, idx, steps,
                                                               batch, lr, q, loss_hist);
  return cudaPeekAtLastError();
}

cudaError_t launch_tau_from_hist(const InstRef& ref, const float* W, float* feats, double* tau,
                                 cudaStream_t s) {
  const size_t smem = mlp::kParams * sizeof(float);
  cudaFuncSetAttribute(mlp::tau_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  mlp::tau_kernel<<<(ref.count + 127) / 128, 128, smem, s>>>(ref, W, feats, tau);
  return cudaPeekAtLastError();
}

}  // namespace spamm
