// Kernels of the variant-predictor MLP: fully connected layers with an
// optional ReLU, their backward passes, the mean-squared-error loss and the
// Adam update.  Row-major FP32: X is n x din, W is dout x din, Y is n x dout.
// The network is tiny (tens of features, 64-wide layers), so plain CUDA-core
// kernels with one thread per output element suffice.
#include "internal.h"

namespace alto {

namespace {

__global__ void __launch_bounds__(256) linear_fwd_kernel(const float* __restrict__ X, const float* __restrict__ W,
                                                         const float* __restrict__ b, float* __restrict__ Y, int n,
                                                         int din, int dout, int relu) {
  const int64_t total = static_cast<int64_t>(n) * dout;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / dout;
    const int o = static_cast<int>(e - r * dout);
    float acc = b[o];
    const float* x = X + r * din;
    const float* w = W + static_cast<int64_t>(o) * din;
    for (int i = 0; i < din; ++i) acc = fmaf(x[i], w[i], acc);
    Y[e] = (relu && acc < 0.f) ? 0.f : acc;
  }
}

// G = dY * relu'(Y) (or dY when relu == 0)
__global__ void __launch_bounds__(256) relu_grad_kernel(const float* __restrict__ dY, const float* __restrict__ Y,
                                                        float* __restrict__ G, int64_t total, int relu) {
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    G[e] = (relu && Y[e] <= 0.f) ? 0.f : dY[e];
}

// dX = G W
__global__ void __launch_bounds__(256) linear_bwd_input_kernel(const float* __restrict__ G, const float* __restrict__ W,
                                                               float* __restrict__ dX, int n, int din, int dout) {
  const int64_t total = static_cast<int64_t>(n) * din;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / din;
    const int i = static_cast<int>(e - r * din);
    float acc = 0.f;
    const float* g = G + r * dout;
    for (int o = 0; o < dout; ++o) acc = fmaf(g[o], W[static_cast<int64_t>(o) * din + i], acc);
    dX[e] = acc;
  }
}

// dW = G^T X, db = column sums of G: one block per output unit o, threads
// stride over the rows and reduce in FP64.
__global__ void __launch_bounds__(256) linear_bwd_params_kernel(const float* __restrict__ G,
                                                                const float* __restrict__ X, float* __restrict__ dW,
                                                                float* __restrict__ db, int n, int din, int dout) {
  __shared__ double red[256];
  const int o = blockIdx.x;
  for (int i = -1; i < din; ++i) {  // i = -1: the bias
    double acc = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      const double g = G[static_cast<int64_t>(r) * dout + o];
      acc += i < 0 ? g : g * X[static_cast<int64_t>(r) * din + i];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (i < 0)
        db[o] = static_cast<float>(red[0]);
      else
        dW[static_cast<int64_t>(o) * din + i] = static_cast<float>(red[0]);
    }
    __syncthreads();
  }
}

// loss = sum(mask * (P - T)^2) / sum(mask); dP = 2 mask (P - T) / sum(mask)
__global__ void __launch_bounds__(256) mse_kernel(const float* __restrict__ P, const float* __restrict__ T,
                                                  const float* __restrict__ mask, float* __restrict__ dP,
                                                  int64_t total, double inv_count, double* loss) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double m = mask ? mask[e] : 1.0;
    const double d = static_cast<double>(P[e]) - T[e];
    acc += m * d * d;
    dP[e] = static_cast<float>(2.0 * m * d * inv_count);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] * inv_count);
}

__global__ void __launch_bounds__(256) adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                                                   float* __restrict__ m, float* __restrict__ v, int64_t n, float lr,
                                                   float b1, float b2, float eps, float c1, float c2) {
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

unsigned grid_of(int64_t total) {
  int64_t g = (total + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return static_cast<unsigned>(g);
}

}  // namespace

}  // namespace alto

using namespace alto;

extern "C" {

alto_status alto_nn_linear_forward(const float* X, const float* W, const float* b, float* Y, int n, int din,
                                   int dout, int relu, void* stream) {
  if (!X || !W || !b || !Y || n < 0 || din < 1 || dout < 1) return fail(ALTO_EINVAL, "bad linear arguments");
  if (n == 0) return ALTO_OK;
  linear_fwd_kernel<<<grid_of(static_cast<int64_t>(n) * dout), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      X, W, b, Y, n, din, dout, relu);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ALTO_OK : fail(ALTO_ECUDA, "linear forward: %s", cudaGetErrorString(e));
}

alto_status alto_nn_linear_backward(const float* X, const float* W, const float* Y, const float* dY, float* G,
                                    float* dX, float* dW, float* db, int n, int din, int dout, int relu,
                                    void* stream) {
  if (!X || !W || !Y || !dY || !G || !dW || !db || n < 1 || din < 1 || dout < 1)
    return fail(ALTO_EINVAL, "bad linear arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t ny = static_cast<int64_t>(n) * dout;
  relu_grad_kernel<<<grid_of(ny), 256, 0, s>>>(dY, Y, G, ny, relu);
  linear_bwd_params_kernel<<<dout, 256, 0, s>>>(G, X, dW, db, n, din, dout);
  note_launch(2);
  if (dX != nullptr) {
    linear_bwd_input_kernel<<<grid_of(static_cast<int64_t>(n) * din), 256, 0, s>>>(G, W, dX, n, din, dout);
    note_launch();
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ALTO_OK : fail(ALTO_ECUDA, "linear backward: %s", cudaGetErrorString(e));
}

alto_status alto_nn_mse(const float* P, const float* T, const float* mask, float* dP, int64_t count, double norm,
                        double* loss, void* stream) {
  if (!P || !T || !dP || !loss || count < 0 || !(norm > 0)) return fail(ALTO_EINVAL, "bad mse arguments");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), s);
  if (e == cudaSuccess && count > 0) {
    mse_kernel<<<grid_of(count), 256, 0, s>>>(P, T, mask, dP, count, 1.0 / norm, loss);
    note_launch();
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? ALTO_OK : fail(ALTO_ECUDA, "mse: %s", cudaGetErrorString(e));
}

alto_status alto_nn_adam(float* param, const float* grad, float* m, float* v, int64_t count, float lr, float beta1,
                         float beta2, float eps, int step, void* stream) {
  if (!param || !grad || !m || !v || count < 0 || step < 1) return fail(ALTO_EINVAL, "bad adam arguments");
  if (count == 0) return ALTO_OK;
  const float c1 = 1.f - powf(beta1, static_cast<float>(step));
  const float c2 = 1.f - powf(beta2, static_cast<float>(step));
  adam_kernel<<<grid_of(count), 256, 0, static_cast<cudaStream_t>(stream)>>>(param, grad, m, v, count, lr, beta1,
                                                                            beta2, eps, c1, c2);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ALTO_OK : fail(ALTO_ECUDA, "adam: %s", cudaGetErrorString(e));
}

}  // extern "C"
