// The cost model's kernels (include/onesweep_mlp.h): forward pass, mean
// squared error with its gradient, and an Adam update, for a
// one-hidden-layer ReLU perceptron small enough that its parameters live in
// shared memory. One thread per sample; per-block gradient sums in shared
// memory, then one global atomic per parameter per block. fp32 throughout.
// These matrices are tiny (at most 128 x 32), so the CUDA cores, not the
// tensor cores, are the right unit.
#include <cuda_runtime.h>

#include "../../include/onesweep_mlp.h"

namespace {

constexpr int kMaxFeatures = 32;
constexpr int kMaxHidden = 128;
constexpr int kThreads = 256;

__host__ __device__ inline int param_count(int f, int h) { return h * f + 2 * h + 1; }

// Loads the parameters into shared memory.
__device__ inline void load_params(float* sp, const float* params, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) sp[i] = params[i];
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) mlp_forward_kernel(const float* params, int f, int hdim, const float* x,
                                                                int n, float* y) {
  extern __shared__ float sp[];
  load_params(sp, params, param_count(f, hdim));
  const float* W1 = sp;
  const float* b1 = W1 + hdim * f;
  const float* w2 = b1 + hdim;
  const float b2 = w2[hdim];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float xi[kMaxFeatures];
  for (int k = 0; k < f; ++k) xi[k] = x[(size_t)i * f + k];
  float out = b2;
  for (int j = 0; j < hdim; ++j) {
    float pre = b1[j];
    for (int k = 0; k < f; ++k) pre += W1[j * f + k] * xi[k];
    out += w2[j] * fmaxf(pre, 0.0f);
  }
  y[i] = out;
}

__global__ void __launch_bounds__(kThreads) mlp_grad_kernel(const float* params, int f, int hdim, const float* x,
                                                             const float* t, int n, float* grads, float* loss) {
  extern __shared__ float sp[];
  const int count = param_count(f, hdim);
  float* sg = sp + count;       // per-block gradient sums
  float* sloss = sg + count;    // per-block loss sum
  for (int i = threadIdx.x; i < count; i += blockDim.x) sg[i] = 0.0f;
  if (threadIdx.x == 0) *sloss = 0.0f;
  load_params(sp, params, count);
  const float* W1 = sp;
  const float* b1 = W1 + hdim * f;
  const float* w2 = b1 + hdim;
  const float b2 = w2[hdim];
  float* gW1 = sg;
  float* gb1 = gW1 + hdim * f;
  float* gw2 = gb1 + hdim;
  float* gb2 = gw2 + hdim;

  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    float xi[kMaxFeatures];
    for (int k = 0; k < f; ++k) xi[k] = x[(size_t)i * f + k];
    float out = b2;
    for (int j = 0; j < hdim; ++j) {
      float pre = b1[j];
      for (int k = 0; k < f; ++k) pre += W1[j * f + k] * xi[k];
      out += w2[j] * fmaxf(pre, 0.0f);
    }
    const float r = out - t[i];
    const float dy = 2.0f * r / (float)n;  // dL/dy_i
    atomicAdd(sloss, r * r / (float)n);
    atomicAdd(gb2, dy);
    for (int j = 0; j < hdim; ++j) {
      float pre = b1[j];
      for (int k = 0; k < f; ++k) pre += W1[j * f + k] * xi[k];
      if (pre > 0.0f) {
        atomicAdd(gw2 + j, dy * pre);
        const float dpre = dy * w2[j];
        atomicAdd(gb1 + j, dpre);
        for (int k = 0; k < f; ++k) atomicAdd(gW1 + j * f + k, dpre * xi[k]);
      }
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < count; p += blockDim.x) atomicAdd(grads + p, sg[p]);
  if (threadIdx.x == 0) atomicAdd(loss, *sloss);
}

__global__ void mlp_adam_kernel(float* params, const float* grads, float* m, float* v, int count, float lr, float b1,
                                float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float g = grads[i];
  const float mi = b1 * m[i] + (1.0f - b1) * g;
  const float vi = b2 * v[i] + (1.0f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

bool sizes_ok(int f, int h) { return f >= 1 && f <= kMaxFeatures && h >= 1 && h <= kMaxHidden; }

}  // namespace

extern "C" {

int os_mlp_param_count(int features, int hidden) {
  return sizes_ok(features, hidden) ? param_count(features, hidden) : 0;
}

int os_mlp_forward(const float* params, int features, int hidden, const float* x, int n, float* y, void* stream) {
  if (!sizes_ok(features, hidden) || n < 0 || !params || (n > 0 && (!x || !y))) return OS_ERR_INVALID_ARG;
  if (n == 0) return OS_OK;
  const size_t smem = (size_t)param_count(features, hidden) * sizeof(float);
  mlp_forward_kernel<<<(n + kThreads - 1) / kThreads, kThreads, smem, static_cast<cudaStream_t>(stream)>>>(
      params, features, hidden, x, n, y);
  return cudaGetLastError() == cudaSuccess ? OS_OK : OS_ERR_CUDA;
}

int os_mlp_loss_grad(const float* params, int features, int hidden, const float* x, const float* t, int n,
                     float* grads, float* loss, void* stream) {
  if (!sizes_ok(features, hidden) || n <= 0 || !params || !x || !t || !grads || !loss) return OS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int count = param_count(features, hidden);
  if (cudaMemsetAsync(grads, 0, (size_t)count * sizeof(float), s) != cudaSuccess) return OS_ERR_CUDA;
  if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return OS_ERR_CUDA;
  const size_t smem = (2 * (size_t)count + 1) * sizeof(float);
  mlp_grad_kernel<<<(n + kThreads - 1) / kThreads, kThreads, smem, s>>>(params, features, hidden, x, t, n, grads,
                                                                         loss);
  return cudaGetLastError() == cudaSuccess ? OS_OK : OS_ERR_CUDA;
}

int os_mlp_adam_step(float* params, const float* grads, float* m, float* v, int count, float lr, float beta1,
                     float beta2, float eps, int step, void* stream) {
  if (count <= 0 || step < 1 || !params || !grads || !m || !v) return OS_ERR_INVALID_ARG;
  double p1 = 1.0, p2 = 1.0;
  for (int i = 0; i < step; ++i) {
    p1 *= beta1;
    p2 *= beta2;
  }
  const float c1 = (float)(1.0 - p1), c2 = (float)(1.0 - p2);
  mlp_adam_kernel<<<(count + kThreads - 1) / kThreads, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      params, grads, m, v, count, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? OS_OK : OS_ERR_CUDA;
}

}  // extern "C"
