// Density of states of H~ by the kernel polynomial method (Weisse, Wellein,
// Alvermann, Fehske, Rev. Mod. Phys. 78, 275 (2006)): stochastic Chebyshev
// moments mu_n = (1/R) sum_r r^T T_n(H~) r of R random vectors, from the same
// H~ step kernel as the filter, and the Jackson-damped eigenvalue count of an
// interval.  The paper sets K from the density of states at the target
// ("POLFED algorithm" section and the Supplement's estimate of rho(0)) and
// cites iterative estimators of it; this is such an estimator.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "polfed_internal.h"

namespace polfed {

// Jackson damping factors g_n, n = 0..N-1 (Weisse et al., Eq. (71)).
void jackson_coeffs(int N, std::vector<double>& g) {
  g.assign(N, 1.0);
  const double q = M_PI / (N + 1);
  for (int n = 0; n < N; n++)
    g[n] = ((N - n + 1) * std::cos(q * n) + std::sin(q * n) / std::tan(q)) / (N + 1);
}

namespace {

constexpr int kDotBlocks = 152 * 2;
constexpr int kDotThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;
}

// part[2b] = sum a*a, part[2b+1] = sum a*c over this block's grid-stride share
template <class T>
__global__ void k_kpm_dots(const T* __restrict__ a, const T* __restrict__ c, int64_t n, double* __restrict__ part) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = (double)a[i];
    s0 += x * x;
    s1 += x * (double)c[i];
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s0;
    part[2 * blockIdx.x + 1] = s1;
  }
}

// t_{n+1} = 2 y - t_{n-1} (written over t_{n-1}), y = H~ t_n; partial sums of
// t_n . t_n and t_{n+1} . t_n
template <class T>
__global__ void k_kpm_step(const T* __restrict__ y, T* __restrict__ prev, const T* __restrict__ cur, int64_t n,
                           double* __restrict__ part) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T nx = (T)2 * y[i] - prev[i];
    prev[i] = nx;
    const double c = (double)cur[i];
    s0 += c * c;
    s1 += (double)nx * c;
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s0;
    part[2 * blockIdx.x + 1] = s1;
  }
}

// out[0..1] = column sums of the [nb x 2] partials, in fixed order
__global__ void k_kpm_reduce(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    s0 += part[2 * i];
    s1 += part[2 * i + 1];
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    out[0] = s0;
    out[1] = s1;
  }
}

template <class T>
int kpm_run(HamPlan& plan, int kind, const T* r, int R, int n_mom, double* mu, const KpmBuffers& b, FilterScratch& scr,
            cudaStream_t s) {
  const int64_t n = plan.geo.dim * (int64_t)R;
  const int abi = std::is_same<T, float>::value ? POLFED_F32 : POLFED_F64;
  T* prev = (T*)b.t0;
  T* cur = (T*)b.t1;
  T* y = (T*)b.y;
  const int lpr = choose_lpr(kind, R);
  PF_CUDA(cudaMemcpyAsync(prev, r, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, s));
  PF_CHECK(apply_block(plan, kind, prev, cur, R, abi, scr, s, lpr));
  k_kpm_dots<T><<<kDotBlocks, kDotThreads, 0, s>>>(prev, cur, n, b.part);
  k_kpm_reduce<<<1, kDotThreads, 0, s>>>(b.part, kDotBlocks, b.mu);
  count_launch(2);
  const int half = (n_mom + 1) / 2;  // t_0 .. t_half are needed
  for (int k = 1; k < half; k++) {
    PF_CHECK(apply_block(plan, kind, cur, y, R, abi, scr, s, lpr));
    k_kpm_step<T><<<kDotBlocks, kDotThreads, 0, s>>>(y, prev, cur, n, b.part);
    k_kpm_reduce<<<1, kDotThreads, 0, s>>>(b.part, kDotBlocks, b.mu + 2 * k);
    count_launch(2);
    std::swap(prev, cur);
  }
  PF_CUDA(cudaGetLastError());
  std::vector<double> raw((size_t)2 * half);
  PF_CUDA(cudaMemcpyAsync(raw.data(), b.mu, raw.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  // raw[0] = r.r, raw[1] = r.H~r; raw[2k] = t_k.t_k, raw[2k+1] = t_{k+1}.t_k
  //   T_{2k} = 2 T_k^2 - T_0,  T_{2k+1} = 2 T_{k+1} T_k - T_1
  const double m0 = raw[0], m1 = raw[1];
  for (int j = 0; j < n_mom; j++) {
    double v;
    if (j < 2)
      v = raw[j];
    else
      v = 2.0 * raw[j] - ((j & 1) ? m1 : m0);
    mu[j] = v / R;
  }
  for (int j = 0; j < n_mom; j++)
    if (!std::isfinite(mu[j]) || std::fabs(mu[j]) > 1.01 * std::fabs(mu[0]) + 1e-300)
      return fail(POLFED_EBOUNDS, "KPM moment |mu_n| > mu_0: spectrum outside [e_lo, e_hi]");
  return POLFED_OK;
}

}  // namespace

size_t kpm_buffer_bytes(int64_t dim, int R, int abi_kind) {
  const size_t es = abi_kind == POLFED_F32 ? 4 : 8;
  const size_t v = ((size_t)dim * R * es + 255) & ~(size_t)255;
  return 3 * v + 2 * kDotBlocks * sizeof(double) + 256 + (size_t)(2 * (kMaxKpmMoments / 2 + 1)) * sizeof(double);
}

KpmBuffers kpm_carve(void* base, int64_t dim, int R, int abi_kind) {
  const size_t es = abi_kind == POLFED_F32 ? 4 : 8;
  const size_t v = ((size_t)dim * R * es + 255) & ~(size_t)255;
  char* p = (char*)base;
  KpmBuffers b;
  b.t0 = p;
  b.t1 = p + v;
  b.y = p + 2 * v;
  b.part = (double*)(p + 3 * v);
  b.mu = b.part + 2 * kDotBlocks;
  return b;
}

int kpm_moments(HamPlan& plan, int kind, const void* r, int R, int n_mom, double* mu, const KpmBuffers& b,
                FilterScratch& scr, cudaStream_t s) {
  if (kind == POLFED_F32) return kpm_run<float>(plan, kind, (const float*)r, R, n_mom, mu, b, scr, s);
  return kpm_run<double>(plan, kind, (const double*)r, R, n_mom, mu, b, scr, s);
}

// Fraction of the spectrum in [x_a, x_b] from Jackson-damped moments:
// the indicator's Chebyshev coefficients are c_0 = (th_a - th_b) / pi and
// c_n = 2 (sin n th_a - sin n th_b) / (n pi), th = arccos x.
double kpm_count_fraction(const double* mu, int n_mom, double x_a, double x_b) {
  std::vector<double> g;
  jackson_coeffs(n_mom, g);
  const double ta = std::acos(std::max(-1.0, std::min(1.0, x_a)));
  const double tb = std::acos(std::max(-1.0, std::min(1.0, x_b)));
  double f = (ta - tb) / M_PI * mu[0];
  for (int k = 1; k < n_mom; k++) f += g[k] * 2.0 * (std::sin(k * ta) - std::sin(k * tb)) / (k * M_PI) * mu[k];
  return f / mu[0];
}

}  // namespace polfed

using namespace polfed;

extern "C" {

int polfed_kpm_moments(const polfed_model* model, const uint32_t* d_states, int64_t dim, double e_lo, double e_hi,
                       int32_t n_mom, const void* d_R, int32_t R, int32_t dtype, double* mu, polfed_stream_t stream) {
  if (!model) return fail(POLFED_EINVAL, "model is NULL");
  if (model->L < 4 || model->L > 32 || (model->L & 1)) return fail(POLFED_EINVAL, "L must be even, 4 <= L <= 32");
  if (dim != (int64_t)binom_host(model->L, model->L / 2)) return fail(POLFED_EINVAL, "dim != C(L, L/2)");
  if (!d_states || !d_R || !mu) return fail(POLFED_EINVAL, "NULL argument");
  if (n_mom < 2 || n_mom > kMaxKpmMoments) return fail(POLFED_EINVAL, "n_mom must be in 2..65536");
  if (R < 1 || R > 128) return fail(POLFED_EINVAL, "R must be in 1..128");
  if (dtype != POLFED_F32 && dtype != POLFED_F64 && dtype != POLFED_DF64) return fail(POLFED_EINVAL, "bad dtype");
  if (!std::isfinite(e_lo) || !std::isfinite(e_hi) || !(e_lo < e_hi)) return fail(POLFED_EINVAL, "need e_lo < e_hi");
  cudaStream_t s = (cudaStream_t)stream;
  HamPlan plan;
  PF_CHECK(plan.init(model, s, true));
  PF_CHECK(plan.prepare_typed(dtype, e_lo, e_hi));
  const int abi = dtype == POLFED_F32 ? POLFED_F32 : POLFED_F64;
  const int lpr = choose_lpr(dtype, R);
  const size_t fb = (filter_scratch_bytes(plan, dtype, lpr) + 255) & ~(size_t)255;
  void* mem = nullptr;
  PF_CUDA(cudaMallocAsync(&mem, fb + kpm_buffer_bytes(dim, R, abi), s));
  FilterScratch scr;
  scr.xs = mem;
  scr.bytes = fb;
  const KpmBuffers b = kpm_carve((char*)mem + fb, dim, R, abi);
  const int rc = kpm_moments(plan, dtype, d_R, R, n_mom, mu, b, scr, s);
  cudaFreeAsync(mem, s);
  cudaStreamSynchronize(s);
  return rc;
}

int polfed_kpm_count(const double* mu, int32_t n_mom, double x_a, double x_b, double* fraction) {
  if (!mu || !fraction) return fail(POLFED_EINVAL, "NULL argument");
  if (n_mom < 1 || n_mom > kMaxKpmMoments) return fail(POLFED_EINVAL, "n_mom must be in 1..65536");
  if (!(x_a <= x_b) || !(mu[0] != 0.0)) return fail(POLFED_EINVAL, "need x_a <= x_b and mu[0] != 0");
  *fraction = kpm_count_fraction(mu, n_mom, x_a, x_b);
  return POLFED_OK;
}

}  // extern "C"
