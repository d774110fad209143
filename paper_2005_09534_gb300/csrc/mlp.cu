// Learned predictor of spectral bounds and density of states: a small fully
// connected FP32 network, x -> tanh(W1 x' + b1) -> tanh(W2 . + b2) -> W3 . + b3,
// with x' = (x - x_mean) / x_std and outputs in standardized target units.
// Forward, backward (hand-derived; deterministic reductions, no atomics) and
// the Adam update are plain CUDA kernels: the network is tiny (about 20k
// parameters), so each kernel maps one thread to one output, one parameter
// gradient or one activation.
//
// Parameter layout (one contiguous float array):
//   W1 [H x d_in] row-major, b1 [H], W2 [H x H], b2 [H], W3 [d_out x H], b3 [d_out].
#include <cmath>
#include <cstring>
#include <vector>

#include "polfed_internal.h"

struct polfed_mlp {
  int d_in = 0, H = 0, d_out = 0, n_params = 0;
  float* params = nullptr;  // device
  float* m = nullptr;       // Adam first moment
  float* v = nullptr;       // Adam second moment
  float* grad = nullptr;    // device, n_params
  float* scale = nullptr;   // device: x_mean [d_in], 1/x_std [d_in], y_mean [d_out], y_std [d_out]
  float* io = nullptr;      // device: one input row and one output row (polfed_mlp_predict)
  float* work = nullptr;    // activations and deltas
  size_t work_floats = 0;
  std::vector<float> h_scale;  // host copy of scale
  int64_t t = 0;               // Adam step counter
  int device = 0;
};

namespace polfed {
namespace {

// xs[b][i] = (x[b][i] - mean[i]) * inv_std[i]
__global__ void k_mlp_standardize(const float* __restrict__ x, const float* __restrict__ mean,
                                  const float* __restrict__ inv_std, int B, int d, float* __restrict__ xs) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * d) return;
  const int i = e % d;
  xs[e] = (x[e] - mean[i]) * inv_std[i];
}

// out[b][j] = act(sum_i W[j][i] in[b][i] + bias[j]); act = tanh (hidden) or identity
__global__ void k_mlp_layer(const float* __restrict__ W, const float* __restrict__ bias, const float* __restrict__ in,
                            int B, int n_in, int n_out, int tanh_act, float* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * n_out) return;
  const int b = e / n_out, j = e % n_out;
  float s = bias[j];
  const float* w = W + (size_t)j * n_in;
  const float* x = in + (size_t)b * n_in;
  for (int i = 0; i < n_in; i++) s = fmaf(w[i], x[i], s);
  out[e] = tanh_act ? tanhf(s) : s;
}

// y[b][o] = ys[b][o] * y_std[o] + y_mean[o]
__global__ void k_mlp_unscale(const float* __restrict__ ys, const float* __restrict__ mean,
                              const float* __restrict__ sd, int B, int d, float* __restrict__ y) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * d) return;
  const int o = e % d;
  y[e] = fmaf(ys[e], sd[o], mean[o]);
}

// r = y - (t - y_mean) / y_std;  dy = r / B;  lp = 0.5 r^2 / B
__global__ void k_mlp_out_delta(const float* __restrict__ y, const float* __restrict__ t,
                                const float* __restrict__ mean, const float* __restrict__ sd, int B, int d_out,
                                float* __restrict__ dy, float* __restrict__ lp) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * d_out) return;
  const int o = e % d_out;
  const float r = y[e] - (t[e] - mean[o]) / sd[o];
  dy[e] = r / (float)B;
  lp[e] = 0.5f * r * r / (float)B;
}

// dW[j][i] = sum_b dz[b][j] in[b][i];  db[j] = sum_b dz[b][j]  (one thread per parameter)
__global__ void k_mlp_wgrad(const float* __restrict__ dz, const float* __restrict__ in, int B, int n_in, int n_out,
                            float* __restrict__ dW, float* __restrict__ db) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int nw = n_out * n_in;
  if (e < nw) {
    const int j = e / n_in, i = e % n_in;
    float s = 0.f;
    for (int b = 0; b < B; b++) s = fmaf(dz[(size_t)b * n_out + j], in[(size_t)b * n_in + i], s);
    dW[e] = s;
  } else if (e < nw + n_out) {
    const int j = e - nw;
    float s = 0.f;
    for (int b = 0; b < B; b++) s += dz[(size_t)b * n_out + j];
    db[j] = s;
  }
}

// dz_prev[b][i] = (sum_j W[j][i] dz[b][j]) * (1 - a_prev[b][i]^2)   (tanh' = 1 - tanh^2)
__global__ void k_mlp_back(const float* __restrict__ W, const float* __restrict__ dz, const float* __restrict__ a_prev,
                           int B, int n_in, int n_out, float* __restrict__ dz_prev) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * n_in) return;
  const int b = e / n_in, i = e % n_in;
  float s = 0.f;
  for (int j = 0; j < n_out; j++) s = fmaf(W[(size_t)j * n_in + i], dz[(size_t)b * n_out + j], s);
  const float a = a_prev[e];
  dz_prev[e] = s * (1.f - a * a);
}

// Adam with bias correction (Kingma & Ba, ICLR 2015, Algorithm 1).
__global__ void k_mlp_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                           float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gi = g[e];
  const float mi = b1 * m[e] + (1.f - b1) * gi;
  const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
  m[e] = mi;
  v[e] = vi;
  p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// *out = sum x[0..n), one block, fixed order
__global__ void k_mlp_sum(const float* __restrict__ x, int n, float* __restrict__ out) {
  __shared__ float sh[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// uniform in [-a, a] from splitmix64, a = sqrt(6 / (fan_in + fan_out)) per weight matrix; biases 0
__global__ void k_mlp_init(float* p, int n, uint64_t seed, int d_in, int H, int d_out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(e + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const float u = (float)((double)(z >> 40) * (1.0 / 16777216.0)) * 2.f - 1.f;
  const int n1 = H * d_in, n2 = n1 + H, n3 = n2 + H * H, n4 = n3 + H, n5 = n4 + d_out * H;
  float a = 0.f;
  if (e < n1)
    a = sqrtf(6.f / (d_in + H));
  else if (e >= n2 && e < n3)
    a = sqrtf(6.f / (2 * H));
  else if (e >= n4 && e < n5)
    a = sqrtf(6.f / (H + d_out));
  p[e] = a * u;
}

unsigned nblk(int n) { return (unsigned)((n + 255) / 256); }

struct Views {
  const float *W1, *b1, *W2, *b2, *W3, *b3;
  float *gW1, *gb1, *gW2, *gb2, *gW3, *gb3;
  const float *xm, *xinv, *ym, *ysd;
};

Views views(const polfed_mlp* n) {
  Views v;
  v.W1 = n->params;
  v.b1 = v.W1 + (size_t)n->H * n->d_in;
  v.W2 = v.b1 + n->H;
  v.b2 = v.W2 + (size_t)n->H * n->H;
  v.W3 = v.b2 + n->H;
  v.b3 = v.W3 + (size_t)n->d_out * n->H;
  v.gW1 = n->grad;
  v.gb1 = v.gW1 + (size_t)n->H * n->d_in;
  v.gW2 = v.gb1 + n->H;
  v.gb2 = v.gW2 + (size_t)n->H * n->H;
  v.gW3 = v.gb2 + n->H;
  v.gb3 = v.gW3 + (size_t)n->d_out * n->H;
  v.xm = n->scale;
  v.xinv = v.xm + n->d_in;
  v.ym = v.xinv + n->d_in;
  v.ysd = v.ym + n->d_out;
  return v;
}

// Work buffer: xs [B d_in] | a1 [B H] | a2 [B H] | y [B d_out] | dy [B d_out] | dz2 [B H] | dz1 [B H] | loss [1]
struct Work {
  float *xs, *a1, *a2, *y, *dy, *dz2, *dz1, *loss;
};

int ensure_work(polfed_mlp* n, int B, Work* w) {
  const size_t need = (size_t)B * (n->d_in + 4 * n->H + 2 * n->d_out) + 64;
  if (!n->work || n->work_floats < need) {
    if (n->work) cudaFree(n->work);
    n->work = nullptr;
    n->work_floats = 0;
    if (cudaMalloc(&n->work, need * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return fail(POLFED_ENOMEM, "MLP work allocation failed");
    }
    n->work_floats = need;
  }
  w->xs = n->work;
  w->a1 = w->xs + (size_t)B * n->d_in;
  w->a2 = w->a1 + (size_t)B * n->H;
  w->y = w->a2 + (size_t)B * n->H;
  w->dy = w->y + (size_t)B * n->d_out;
  w->dz2 = w->dy + (size_t)B * n->d_out;
  w->dz1 = w->dz2 + (size_t)B * n->H;
  w->loss = w->dz1 + (size_t)B * n->H;
  return POLFED_OK;
}

// standardized forward pass into the work buffer
int forward(polfed_mlp* n, const float* x, int B, cudaStream_t s, Work* w) {
  PF_CHECK(ensure_work(n, B, w));
  const Views v = views(n);
  k_mlp_standardize<<<nblk(B * n->d_in), 256, 0, s>>>(x, v.xm, v.xinv, B, n->d_in, w->xs);
  k_mlp_layer<<<nblk(B * n->H), 256, 0, s>>>(v.W1, v.b1, w->xs, B, n->d_in, n->H, 1, w->a1);
  k_mlp_layer<<<nblk(B * n->H), 256, 0, s>>>(v.W2, v.b2, w->a1, B, n->H, n->H, 1, w->a2);
  k_mlp_layer<<<nblk(B * n->d_out), 256, 0, s>>>(v.W3, v.b3, w->a2, B, n->H, n->d_out, 0, w->y);
  PF_CUDA(cudaGetLastError());
  count_launch(4);
  return POLFED_OK;
}

// gradient of 0.5/B sum |y - t'|^2 into n->grad; the loss partials go to dz1
// before it is overwritten (d_out <= H)
int backward(polfed_mlp* n, const float* x, const float* t, int B, cudaStream_t s, float* loss_host) {
  Work w;
  PF_CHECK(forward(n, x, B, s, &w));
  const Views v = views(n);
  k_mlp_out_delta<<<nblk(B * n->d_out), 256, 0, s>>>(w.y, t, v.ym, v.ysd, B, n->d_out, w.dy, w.dz1);
  k_mlp_sum<<<1, 256, 0, s>>>(w.dz1, B * n->d_out, w.loss);
  k_mlp_wgrad<<<nblk(n->d_out * n->H + n->d_out), 256, 0, s>>>(w.dy, w.a2, B, n->H, n->d_out, v.gW3, v.gb3);
  k_mlp_back<<<nblk(B * n->H), 256, 0, s>>>(v.W3, w.dy, w.a2, B, n->H, n->d_out, w.dz2);
  k_mlp_wgrad<<<nblk(n->H * n->H + n->H), 256, 0, s>>>(w.dz2, w.a1, B, n->H, n->H, v.gW2, v.gb2);
  k_mlp_back<<<nblk(B * n->H), 256, 0, s>>>(v.W2, w.dz2, w.a1, B, n->H, n->H, w.dz1);
  k_mlp_wgrad<<<nblk(n->H * n->d_in + n->H), 256, 0, s>>>(w.dz1, w.xs, B, n->d_in, n->H, v.gW1, v.gb1);
  PF_CUDA(cudaGetLastError());
  count_launch(7);
  if (loss_host) PF_CUDA(cudaMemcpyAsync(loss_host, w.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
  return POLFED_OK;
}

struct DeviceGuard {
  int prev = 0;
  explicit DeviceGuard(int d) {
    cudaGetDevice(&prev);
    cudaSetDevice(d);
  }
  ~DeviceGuard() { cudaSetDevice(prev); }
};

}  // namespace
}  // namespace polfed

using namespace polfed;

extern "C" {

void polfed_mlp_destroy(polfed_mlp* n) {
  if (!n) return;
  DeviceGuard g(n->device);
  cudaFree(n->params);
  cudaFree(n->m);
  cudaFree(n->v);
  cudaFree(n->grad);
  cudaFree(n->scale);
  cudaFree(n->io);
  cudaFree(n->work);
  delete n;
}

int polfed_mlp_create(int32_t d_in, int32_t hidden, int32_t d_out, uint64_t seed, polfed_mlp** out) {
  if (!out) return fail(POLFED_EINVAL, "out is NULL");
  if (d_in < 1 || d_in > 1024 || d_out < 1 || d_out > 64 || hidden < d_out || hidden > 4096)
    return fail(POLFED_EINVAL, "need 1 <= d_in <= 1024, 1 <= d_out <= 64, d_out <= hidden <= 4096");
  polfed_mlp* n = new polfed_mlp();
  n->d_in = d_in;
  n->H = hidden;
  n->d_out = d_out;
  n->n_params = hidden * d_in + hidden + hidden * hidden + hidden + d_out * hidden + d_out;
  cudaGetDevice(&n->device);
  const size_t bytes = (size_t)n->n_params * sizeof(float);
  const size_t sbytes = (size_t)(2 * d_in + 2 * d_out) * sizeof(float);
  if (cudaMalloc(&n->params, bytes) != cudaSuccess || cudaMalloc(&n->m, bytes) != cudaSuccess ||
      cudaMalloc(&n->v, bytes) != cudaSuccess || cudaMalloc(&n->grad, bytes) != cudaSuccess ||
      cudaMalloc(&n->scale, sbytes) != cudaSuccess ||
      cudaMalloc(&n->io, (size_t)(d_in + d_out) * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    polfed_mlp_destroy(n);
    return fail(POLFED_ENOMEM, "MLP allocation failed");
  }
  n->h_scale.assign(2 * d_in + 2 * d_out, 0.f);
  for (int i = 0; i < d_in; i++) n->h_scale[d_in + i] = 1.f;
  for (int o = 0; o < d_out; o++) n->h_scale[2 * d_in + d_out + o] = 1.f;
  int rc = POLFED_OK;
  if (cudaMemset(n->m, 0, bytes) != cudaSuccess || cudaMemset(n->v, 0, bytes) != cudaSuccess ||
      cudaMemset(n->grad, 0, bytes) != cudaSuccess ||
      cudaMemcpy(n->scale, n->h_scale.data(), sbytes, cudaMemcpyHostToDevice) != cudaSuccess)
    rc = POLFED_ECUDA;
  if (rc == POLFED_OK) {
    k_mlp_init<<<nblk(n->n_params), 256>>>(n->params, n->n_params, seed, d_in, hidden, d_out);
    count_launch();
    if (cudaDeviceSynchronize() != cudaSuccess) rc = POLFED_ECUDA;
  }
  if (rc != POLFED_OK) {
    cudaGetLastError();
    polfed_mlp_destroy(n);
    return fail(rc, "MLP initialization failed");
  }
  *out = n;
  return POLFED_OK;
}

int32_t polfed_mlp_num_params(const polfed_mlp* n) { return n ? n->n_params : 0; }

int polfed_mlp_set_params(polfed_mlp* n, const float* host) {
  if (!n || !host) return fail(POLFED_EINVAL, "NULL argument");
  DeviceGuard g(n->device);
  const size_t bytes = (size_t)n->n_params * sizeof(float);
  PF_CUDA(cudaMemcpy(n->params, host, bytes, cudaMemcpyHostToDevice));
  PF_CUDA(cudaMemset(n->m, 0, bytes));
  PF_CUDA(cudaMemset(n->v, 0, bytes));
  n->t = 0;
  return POLFED_OK;
}

int polfed_mlp_get_params(const polfed_mlp* n, float* host) {
  if (!n || !host) return fail(POLFED_EINVAL, "NULL argument");
  DeviceGuard g(n->device);
  PF_CUDA(cudaMemcpy(host, n->params, (size_t)n->n_params * sizeof(float), cudaMemcpyDeviceToHost));
  return POLFED_OK;
}

int polfed_mlp_set_scaling(polfed_mlp* n, const float* x_mean, const float* x_std, const float* y_mean,
                           const float* y_std) {
  if (!n || !x_mean || !x_std || !y_mean || !y_std) return fail(POLFED_EINVAL, "NULL argument");
  for (int i = 0; i < n->d_in; i++)
    if (!(x_std[i] > 0.f) || !std::isfinite(x_std[i]) || !std::isfinite(x_mean[i]))
      return fail(POLFED_EINVAL, "x_std must be finite and > 0");
  for (int o = 0; o < n->d_out; o++)
    if (!(y_std[o] > 0.f) || !std::isfinite(y_std[o]) || !std::isfinite(y_mean[o]))
      return fail(POLFED_EINVAL, "y_std must be finite and > 0");
  for (int i = 0; i < n->d_in; i++) {
    n->h_scale[i] = x_mean[i];
    n->h_scale[n->d_in + i] = 1.f / x_std[i];
  }
  for (int o = 0; o < n->d_out; o++) {
    n->h_scale[2 * n->d_in + o] = y_mean[o];
    n->h_scale[2 * n->d_in + n->d_out + o] = y_std[o];
  }
  DeviceGuard g(n->device);
  PF_CUDA(cudaMemcpy(n->scale, n->h_scale.data(), n->h_scale.size() * sizeof(float), cudaMemcpyHostToDevice));
  return POLFED_OK;
}

int polfed_mlp_forward(polfed_mlp* n, const float* d_x, int32_t B, float* d_y, polfed_stream_t stream) {
  if (!n || !d_x || !d_y || B < 1 || B > (1 << 20)) return fail(POLFED_EINVAL, "bad MLP forward arguments");
  DeviceGuard g(n->device);
  cudaStream_t s = (cudaStream_t)stream;
  Work w;
  PF_CHECK(forward(n, d_x, B, s, &w));
  const Views v = views(n);
  k_mlp_unscale<<<nblk(B * n->d_out), 256, 0, s>>>(w.y, v.ym, v.ysd, B, n->d_out, d_y);
  PF_CUDA(cudaGetLastError());
  count_launch();
  PF_CUDA(cudaStreamSynchronize(s));
  return POLFED_OK;
}

int polfed_mlp_grad(polfed_mlp* n, const float* d_x, const float* d_t, int32_t B, float* d_grad, float* loss,
                    polfed_stream_t stream) {
  if (!n || !d_x || !d_t || B < 1 || B > (1 << 20)) return fail(POLFED_EINVAL, "bad MLP gradient arguments");
  DeviceGuard g(n->device);
  cudaStream_t s = (cudaStream_t)stream;
  PF_CHECK(backward(n, d_x, d_t, B, s, loss));
  if (d_grad)
    PF_CUDA(cudaMemcpyAsync(d_grad, n->grad, (size_t)n->n_params * sizeof(float), cudaMemcpyDeviceToDevice, s));
  PF_CUDA(cudaStreamSynchronize(s));
  return POLFED_OK;
}

int polfed_mlp_train_step(polfed_mlp* n, const float* d_x, const float* d_t, int32_t B, float lr, float* loss,
                          polfed_stream_t stream) {
  if (!n || !d_x || !d_t || B < 1 || B > (1 << 20) || !(lr > 0.f))
    return fail(POLFED_EINVAL, "bad MLP training arguments");
  DeviceGuard g(n->device);
  cudaStream_t s = (cudaStream_t)stream;
  PF_CHECK(backward(n, d_x, d_t, B, s, loss));
  n->t++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)n->t), c2 = 1.f - std::pow(b2, (float)n->t);
  k_mlp_adam<<<nblk(n->n_params), 256, 0, s>>>(n->params, n->m, n->v, n->grad, n->n_params, lr, b1, b2, 1e-8f, c1,
                                                c2);
  PF_CUDA(cudaGetLastError());
  count_launch();
  PF_CUDA(cudaStreamSynchronize(s));
  return POLFED_OK;
}

int polfed_mlp_features(const polfed_model* model, double W, float* x) {
  if (!model || !model->h || !x) return fail(POLFED_EINVAL, "NULL argument");
  if (model->L < 2 || model->L > 32) return fail(POLFED_EINVAL, "L must be in 2..32");
  for (int i = 0; i < model->L; i++) x[i] = (float)model->h[i];
  x[model->L] = (float)W;
  return POLFED_OK;
}

int polfed_mlp_targets(int32_t L, const double* labels, float* y) {
  if (!labels || !y) return fail(POLFED_EINVAL, "NULL argument");
  if (L < 2 || L > 32) return fail(POLFED_EINVAL, "L must be in 2..32");
  if (!(labels[2] > 0.0) || !std::isfinite(labels[2])) return fail(POLFED_EINVAL, "rho_eps must be > 0");
  y[0] = (float)(labels[0] / L);
  y[1] = (float)(labels[1] / L);
  y[2] = (float)std::log(labels[2]);
  return POLFED_OK;
}

int polfed_mlp_predict(polfed_mlp* n, const polfed_model* model, double W, double* out) {
  if (!n || !model || !out) return fail(POLFED_EINVAL, "NULL argument");
  if (n->d_in != model->L + 1 || n->d_out != 3) return fail(POLFED_EINVAL, "predictor needs d_in = L + 1, d_out = 3");
  std::vector<float> x(n->d_in);
  PF_CHECK(polfed_mlp_features(model, W, x.data()));
  DeviceGuard g(n->device);
  PF_CUDA(cudaMemcpy(n->io, x.data(), n->d_in * sizeof(float), cudaMemcpyHostToDevice));
  PF_CHECK(polfed_mlp_forward(n, n->io, 1, n->io + n->d_in, nullptr));
  float y[3];
  PF_CUDA(cudaMemcpy(y, n->io + n->d_in, sizeof(y), cudaMemcpyDeviceToHost));
  out[0] = (double)y[0] * model->L;
  out[1] = (double)y[1] * model->L;
  out[2] = std::exp((double)y[2]);
  return POLFED_OK;
}

}  // extern "C"
