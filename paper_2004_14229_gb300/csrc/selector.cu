// Learned parameter selector: a 4 -> 64 -> 64 -> 64 -> 2 perceptron (tanh
// hidden layers, linear output) with FP16 weights and FP32 accumulation,
// trained on the GPU by full-batch Adam with the kernels below, and used to
// pick the Chebyshev order and the high-frequency level of a plan.  The paper
// has no selector (it fixes m = 4 for all levels, Sect. 4, and l_hf by the
// rule of Sect. 2.5); this is the library's own addition.
//
// Parameter vector (8770 floats): W1 (64 x 4, row-major), b1, W2 (64 x 64),
// b2, W3 (64 x 64), b3, W4 (2 x 64), b4.  The forward pass reads every
// parameter rounded to FP16; gradients are taken w.r.t. the FP32 master copy
// (straight through the rounding); the weight-gradient sums over the batch
// are FP64, one thread per parameter, so training is deterministic.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <string>
#include <vector>

#include "dfdm_internal.cuh"

namespace dfdm {
namespace {

constexpr int kIn = 4, kH = 64, kOut = 2;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn;
constexpr int kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH;
constexpr int kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + kOut * kH;
constexpr int kNParams = kOffB4 + kOut;
static_assert(kNParams == 8770, "parameter layout");

__global__ void k_params_to_half(const float *theta, __half *wh) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kNParams) wh[p] = __float2half_rn(theta[p]);
}

__device__ __forceinline__ float wf(const __half *wh, int i) { return __half2float(wh[i]); }

// One block of 64 threads per sample (grid-stride over samples): thread j is
// hidden neuron j of every layer; activations go through shared memory.
__global__ void __launch_bounds__(kH) k_mlp_forward(const __half *wh, const float *x, int64_t B, float *h1,
                                                    float *h2, float *h3, float *y) {
  __shared__ float in[kH];
  const int j = threadIdx.x;
  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    float z = wf(wh, kOffB1 + j);
#pragma unroll
    for (int i = 0; i < kIn; ++i) z = fmaf(wf(wh, kOffW1 + j * kIn + i), x[b * kIn + i], z);
    float a = tanhf(z);
    if (h1) h1[b * kH + j] = a;
    __syncthreads();
    in[j] = a;
    __syncthreads();
    z = wf(wh, kOffB2 + j);
    for (int i = 0; i < kH; ++i) z = fmaf(wf(wh, kOffW2 + j * kH + i), in[i], z);
    a = tanhf(z);
    if (h2) h2[b * kH + j] = a;
    __syncthreads();
    in[j] = a;
    __syncthreads();
    z = wf(wh, kOffB3 + j);
    for (int i = 0; i < kH; ++i) z = fmaf(wf(wh, kOffW3 + j * kH + i), in[i], z);
    a = tanhf(z);
    if (h3) h3[b * kH + j] = a;
    __syncthreads();
    in[j] = a;
    __syncthreads();
    if (j < kOut) {
      z = wf(wh, kOffB4 + j);
      for (int i = 0; i < kH; ++i) z = fmaf(wf(wh, kOffW4 + j * kH + i), in[i], z);
      y[b * kOut + j] = z;
    }
    __syncthreads();
  }
}

// Per-sample error signals dL/dz of every layer (backpropagation):
// d4 = (y - t) / B, d3 = (W4^T d4) (1 - h3^2), d2 = (W3^T d3) (1 - h2^2),
// d1 = (W2^T d2) (1 - h1^2).
__global__ void __launch_bounds__(kH) k_mlp_deltas(const __half *wh, const float *h1, const float *h2,
                                                   const float *h3, const float *y, const float *t, int64_t B,
                                                   float *d1, float *d2, float *d3, float *d4) {
  __shared__ float dn[kH];
  const int j = threadIdx.x;
  const float invB = 1.0f / (float)B;
  for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
    __syncthreads();
    if (j < kOut) {
      const float v = (y[b * kOut + j] - t[b * kOut + j]) * invB;
      d4[b * kOut + j] = v;
      dn[j] = v;
    }
    __syncthreads();
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kOut; ++k) s = fmaf(wf(wh, kOffW4 + k * kH + j), dn[k], s);
    float h = h3[b * kH + j];
    float d = s * (1.f - h * h);
    d3[b * kH + j] = d;
    __syncthreads();
    dn[j] = d;
    __syncthreads();
    s = 0.f;
    for (int k = 0; k < kH; ++k) s = fmaf(wf(wh, kOffW3 + k * kH + j), dn[k], s);
    h = h2[b * kH + j];
    d = s * (1.f - h * h);
    d2[b * kH + j] = d;
    __syncthreads();
    dn[j] = d;
    __syncthreads();
    s = 0.f;
    for (int k = 0; k < kH; ++k) s = fmaf(wf(wh, kOffW2 + k * kH + j), dn[k], s);
    h = h1[b * kH + j];
    d1[b * kH + j] = s * (1.f - h * h);
  }
}

// grad[p] = sum_b delta_b[row(p)] * input_b[col(p)] (bias: input 1), FP64 sum.
__global__ void k_mlp_wgrad(const float *x, const float *h1, const float *h2, const float *h3, const float *d1,
                            const float *d2, const float *d3, const float *d4, int64_t B, float *grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNParams) return;
  const float *dl, *in;
  int nd, ni, row, col;   // col < 0: bias
  if (p < kOffB1) { dl = d1; nd = kH; in = x; ni = kIn; row = p / kIn; col = p % kIn; }
  else if (p < kOffW2) { dl = d1; nd = kH; in = nullptr; ni = 0; row = p - kOffB1; col = -1; }
  else if (p < kOffB2) { dl = d2; nd = kH; in = h1; ni = kH; row = (p - kOffW2) / kH; col = (p - kOffW2) % kH; }
  else if (p < kOffW3) { dl = d2; nd = kH; in = nullptr; ni = 0; row = p - kOffB2; col = -1; }
  else if (p < kOffB3) { dl = d3; nd = kH; in = h2; ni = kH; row = (p - kOffW3) / kH; col = (p - kOffW3) % kH; }
  else if (p < kOffW4) { dl = d3; nd = kH; in = nullptr; ni = 0; row = p - kOffB3; col = -1; }
  else if (p < kOffB4) { dl = d4; nd = kOut; in = h3; ni = kH; row = (p - kOffW4) / kH; col = (p - kOffW4) % kH; }
  else { dl = d4; nd = kOut; in = nullptr; ni = 0; row = p - kOffB4; col = -1; }
  double s = 0.0;
  for (int64_t b = 0; b < B; ++b) {
    const float a = (col < 0) ? 1.f : in[b * ni + col];
    s += (double)dl[b * nd + row] * (double)a;
  }
  grad[p] = (float)s;
}

// L = (1 / B) sum_b 1/2 |y_b - t_b|^2 (one block, FP64 partial sums).
__global__ void __launch_bounds__(256) k_mlp_loss(const float *y, const float *t, int64_t B, float *loss) {
  __shared__ double part[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < B * kOut; i += blockDim.x) {
    const double r = (double)y[i] - (double)t[i];
    s += 0.5 * r * r;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = (float)(part[0] / (double)B);
}

// Adam step k (from 1) on the FP32 master parameters, refreshing the FP16 copy.
__global__ void k_adam(float *theta, const float *grad, float *m, float *v, __half *wh, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNParams) return;
  const float g = grad[p];
  const float mm = b1 * m[p] + (1.f - b1) * g;
  const float vv = b2 * v[p] + (1.f - b2) * g * g;
  m[p] = mm;
  v[p] = vv;
  const float th = theta[p] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  theta[p] = th;
  wh[p] = __float2half_rn(th);
}

struct Buffers {
  float *theta = nullptr, *x = nullptr, *t = nullptr, *y = nullptr;
  float *h1 = nullptr, *h2 = nullptr, *h3 = nullptr, *d1 = nullptr, *d2 = nullptr, *d3 = nullptr, *d4 = nullptr;
  float *grad = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
  __half *wh = nullptr;
  std::vector<void *> all;
  cudaStream_t st;
  explicit Buffers(cudaStream_t s) : st(s) {}
  template <typename T>
  T *get(size_t count) {
    void *p = nullptr;
    if (cudaMallocAsync(&p, std::max<size_t>(count, 1) * sizeof(T), st) != cudaSuccess)
      throw Error{DFDM_ERR_OOM, "selector buffer allocation failed"};
    all.push_back(p);
    return static_cast<T *>(p);
  }
  ~Buffers() {
    for (void *p : all) cudaFreeAsync(p, st);
  }
};

int grid_samples(int64_t B) { return (int)std::min<int64_t>(B, 152 * 16); }

void forward_all(Buffers &b, int64_t B, bool keep) {
  k_mlp_forward<<<grid_samples(B), kH, 0, b.st>>>(b.wh, b.x, B, keep ? b.h1 : nullptr, keep ? b.h2 : nullptr,
                                                  keep ? b.h3 : nullptr, b.y);
  DFDM_LAUNCH_CHECK();
}

void gradient(Buffers &b, int64_t B) {
  forward_all(b, B, true);
  k_mlp_loss<<<1, 256, 0, b.st>>>(b.y, b.t, B, b.loss);
  DFDM_LAUNCH_CHECK();
  k_mlp_deltas<<<grid_samples(B), kH, 0, b.st>>>(b.wh, b.h1, b.h2, b.h3, b.y, b.t, B, b.d1, b.d2, b.d3, b.d4);
  DFDM_LAUNCH_CHECK();
  k_mlp_wgrad<<<(kNParams + 127) / 128, 128, 0, b.st>>>(b.x, b.h1, b.h2, b.h3, b.d1, b.d2, b.d3, b.d4, B, b.grad);
  DFDM_LAUNCH_CHECK();
}

void load_inputs(Buffers &b, const float *theta, const float *x, const float *t, int64_t B) {
  b.theta = b.get<float>(kNParams);
  b.wh = b.get<__half>(kNParams);
  b.x = b.get<float>(B * kIn);
  b.y = b.get<float>(B * kOut);
  DFDM_CUDA_TRY(cudaMemcpyAsync(b.theta, theta, kNParams * 4, cudaMemcpyHostToDevice, b.st));
  DFDM_CUDA_TRY(cudaMemcpyAsync(b.x, x, B * kIn * 4, cudaMemcpyHostToDevice, b.st));
  if (t) {
    b.t = b.get<float>(B * kOut);
    DFDM_CUDA_TRY(cudaMemcpyAsync(b.t, t, B * kOut * 4, cudaMemcpyHostToDevice, b.st));
    b.h1 = b.get<float>(B * kH);
    b.h2 = b.get<float>(B * kH);
    b.h3 = b.get<float>(B * kH);
    b.d1 = b.get<float>(B * kH);
    b.d2 = b.get<float>(B * kH);
    b.d3 = b.get<float>(B * kH);
    b.d4 = b.get<float>(B * kOut);
    b.grad = b.get<float>(kNParams);
    b.loss = b.get<float>(1);
  }
  k_params_to_half<<<(kNParams + 255) / 256, 256, 0, b.st>>>(b.theta, b.wh);
  DFDM_LAUNCH_CHECK();
}

}  // namespace

void selector_forward(const float *theta, const float *x, int64_t B, float *y, cudaStream_t st) {
  Buffers b(st);
  load_inputs(b, theta, x, nullptr, B);
  forward_all(b, B, false);
  DFDM_CUDA_TRY(cudaMemcpyAsync(y, b.y, B * kOut * 4, cudaMemcpyDeviceToHost, st));
  DFDM_CUDA_TRY(cudaStreamSynchronize(st));
}

void selector_grad(const float *theta, const float *x, const float *t, int64_t B, float *grad, float *loss,
                   cudaStream_t st) {
  Buffers b(st);
  load_inputs(b, theta, x, t, B);
  gradient(b, B);
  DFDM_CUDA_TRY(cudaMemcpyAsync(grad, b.grad, kNParams * 4, cudaMemcpyDeviceToHost, st));
  DFDM_CUDA_TRY(cudaMemcpyAsync(loss, b.loss, 4, cudaMemcpyDeviceToHost, st));
  DFDM_CUDA_TRY(cudaStreamSynchronize(st));
}

void selector_train(const float *theta0, const float *x, const float *t, int64_t B, int epochs, float lr,
                    float *theta_out, float *losses, cudaStream_t st) {
  Buffers b(st);
  load_inputs(b, theta0, x, t, B);
  b.m = b.get<float>(kNParams);
  b.v = b.get<float>(kNParams);
  float *loss_hist = b.get<float>(std::max(epochs, 1));
  DFDM_CUDA_TRY(cudaMemsetAsync(b.m, 0, kNParams * 4, st));
  DFDM_CUDA_TRY(cudaMemsetAsync(b.v, 0, kNParams * 4, st));
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  double p1 = 1.0, p2 = 1.0;
  for (int k = 1; k <= epochs; ++k) {
    gradient(b, B);
    DFDM_CUDA_TRY(cudaMemcpyAsync(loss_hist + (k - 1), b.loss, 4, cudaMemcpyDeviceToDevice, st));
    p1 *= b1;
    p2 *= b2;
    k_adam<<<(kNParams + 255) / 256, 256, 0, st>>>(b.theta, b.grad, b.m, b.v, b.wh, lr, b1, b2, eps,
                                                    (float)(1.0 - p1), (float)(1.0 - p2));
    DFDM_LAUNCH_CHECK();
  }
  DFDM_CUDA_TRY(cudaMemcpyAsync(theta_out, b.theta, kNParams * 4, cudaMemcpyDeviceToHost, st));
  if (losses && epochs > 0)
    DFDM_CUDA_TRY(cudaMemcpyAsync(losses, loss_hist, epochs * 4, cudaMemcpyDeviceToHost, st));
  DFDM_CUDA_TRY(cudaStreamSynchronize(st));
}

int selector_param_count() { return kNParams; }

}  // namespace dfdm

// ------------------------------------------------------------------ C ABI
namespace {
dfdm_status sel_guard(const char *what, const std::function<void()> &f) {
  try {
    f();
    return DFDM_OK;
  } catch (const dfdm::Error &e) {
    dfdm::set_error(std::string(what) + ": " + e.msg);
    return e.status;
  } catch (const std::exception &e) {
    dfdm::set_error(std::string(what) + ": " + e.what());
    return DFDM_ERR_CUDA;
  }
}
}  // namespace

extern "C" {

int dfdm_selector_param_count(void) { return dfdm::selector_param_count(); }

dfdm_status dfdm_selector_features(double kappa, double root_side, int level, int64_t n_points, double tol,
                                   float *out) {
  if (!out || !(kappa > 0) || !(root_side > 0) || level < 0 || level > 30 || n_points < 1 || !(tol > 0)) {
    dfdm::set_error("dfdm_selector_features: invalid argument");
    return DFDM_ERR_INVALID_ARG;
  }
  const double w = root_side / std::ldexp(1.0, level);
  const double per_box = (double)n_points / std::ldexp(1.0, 3 * level);
  out[0] = (float)(level / 10.0);
  out[1] = (float)(std::log2(kappa * std::sqrt(3.0) * w) / 8.0);
  out[2] = (float)(std::log2(1.0 + per_box) / 16.0);
  out[3] = (float)(-std::log10(tol) / 10.0);
  return DFDM_OK;
}

dfdm_status dfdm_selector_forward(const float *theta, const float *x, int64_t n, float *y, void *stream) {
  if (!theta || !x || !y || n < 1) {
    dfdm::set_error("dfdm_selector_forward: invalid argument");
    return DFDM_ERR_INVALID_ARG;
  }
  return sel_guard("dfdm_selector_forward",
                   [&] { dfdm::selector_forward(theta, x, n, y, static_cast<cudaStream_t>(stream)); });
}

dfdm_status dfdm_selector_grad(const float *theta, const float *x, const float *t, int64_t n, float *grad,
                               float *loss, void *stream) {
  if (!theta || !x || !t || !grad || !loss || n < 1) {
    dfdm::set_error("dfdm_selector_grad: invalid argument");
    return DFDM_ERR_INVALID_ARG;
  }
  return sel_guard("dfdm_selector_grad",
                   [&] { dfdm::selector_grad(theta, x, t, n, grad, loss, static_cast<cudaStream_t>(stream)); });
}

dfdm_status dfdm_selector_train(const float *theta0, const float *x, const float *t, int64_t n, int epochs,
                                float lr, float *theta_out, float *losses, void *stream) {
  if (!theta0 || !x || !t || !theta_out || n < 1 || epochs < 0 || !(lr > 0)) {
    dfdm::set_error("dfdm_selector_train: invalid argument");
    return DFDM_ERR_INVALID_ARG;
  }
  return sel_guard("dfdm_selector_train", [&] {
    dfdm::selector_train(theta0, x, t, n, epochs, lr, theta_out, losses, static_cast<cudaStream_t>(stream));
  });
}

dfdm_status dfdm_select_params(const float *theta, double kappa, double tol, int64_t n_points, dfdm_params *p,
                               void *stream) {
  if (!theta || !p || !(kappa > 0) || !(tol > 0) || n_points < 1 || !(p->root_side > 0) || p->max_depth < 0 ||
      p->max_depth > 10) {
    dfdm::set_error("dfdm_select_params: invalid argument");
    return DFDM_ERR_INVALID_ARG;
  }
  const int lo = std::min(2, p->max_depth), hi = p->max_depth;
  const int nl = hi - lo + 1;
  std::vector<float> x(4 * nl), y(2 * nl);
  for (int l = lo; l <= hi; ++l) {
    const dfdm_status s = dfdm_selector_features(kappa, p->root_side, l, n_points, tol, &x[4 * (l - lo)]);
    if (s != DFDM_OK) return s;
  }
  const dfdm_status s = dfdm_selector_forward(theta, x.data(), nl, y.data(), stream);
  if (s != DFDM_OK) return s;
  double osum = 0.0;
  int lhf = -1;
  for (int i = 0; i < nl; ++i) {
    if (!std::isfinite(y[2 * i]) || !std::isfinite(y[2 * i + 1])) {
      dfdm::set_error("dfdm_select_params: the network produced a non-finite output");
      return DFDM_ERR_NUMERIC;
    }
    osum += 2.0 + 8.0 * (double)y[2 * i];
    if (y[2 * i + 1] > 0.5f) lhf = lo + i;
  }
  p->order = std::min(10, std::max(2, (int)std::floor(osum / nl + 0.5)));
  p->l_hf = lhf;
  return DFDM_OK;
}

}  // extern "C"
