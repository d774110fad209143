// C ABI entry points: error reporting, basis, H~ application and the filter.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "polfed_internal.h"

namespace polfed {

static thread_local std::string t_err;
static thread_local Counters g_counters;  // per host thread: a call reports its own launches
Counters& counters() { return g_counters; }

void set_error(int code, const std::string& msg) { t_err = "[" + std::to_string(code) + "] " + msg; }

int fail(int code, const std::string& msg) {
  set_error(code, msg);
  return code;
}

void clear_error() { t_err.clear(); }

static int check_block_args(const polfed_model* model, const uint32_t* d_states, int64_t dim, const void* X,
                            const void* Y, int n_b, int dtype) {
  if (!model) return fail(POLFED_EINVAL, "model is NULL");
  if (model->L < 4 || model->L > 32 || (model->L & 1)) return fail(POLFED_EINVAL, "L must be even, 4 <= L <= 32");
  if (dim != (int64_t)binom_host(model->L, model->L / 2)) return fail(POLFED_EINVAL, "dim != C(L, L/2)");
  if (!d_states) return fail(POLFED_EINVAL, "d_states is NULL");
  if (!X || !Y) return fail(POLFED_EINVAL, "X or Y is NULL");
  if (X == Y) return fail(POLFED_EINVAL, "X and Y must not overlap");
  if (n_b < 1 || n_b > 128) return fail(POLFED_EINVAL, "n_b must be in 1..128");
  if (dtype != POLFED_F32 && dtype != POLFED_F64 && dtype != POLFED_DF64) return fail(POLFED_EINVAL, "bad dtype");
  const size_t es = dtype == POLFED_F32 ? 4 : 8;
  const char* x = (const char*)X;
  const char* y = (const char*)Y;
  const size_t nbytes = (size_t)dim * n_b * es;
  if (x < y + nbytes && y < x + nbytes) return fail(POLFED_EINVAL, "X and Y must not overlap");
  return POLFED_OK;
}

static int check_bounds(double e_lo, double e_hi) {
  if (!std::isfinite(e_lo) || !std::isfinite(e_hi)) return fail(POLFED_EINVAL, "non-finite e_lo/e_hi");
  if (!(e_lo == 0.0 && e_hi == 0.0) && !(e_lo < e_hi)) return fail(POLFED_EINVAL, "need e_lo < e_hi");
  return POLFED_OK;
}

struct StreamScratch {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  ~StreamScratch() {
    if (p) cudaFreeAsync(p, s);
  }
};

}  // namespace polfed

using namespace polfed;

extern "C" {

const char* polfed_last_error(void) { return t_err.c_str(); }

int polfed_get_counters(polfed_counters* out) {
  if (!out) return fail(POLFED_EINVAL, "out is NULL");
  const Counters& c = counters();
  out->launches = c.launches;
  out->step_launches = c.step_launches;
  out->step_gpu_s = c.step_gpu_s;
  out->step_alg_bytes = c.step_alg_bytes;
  for (int k = 0; k < 3; k++) {
    out->kind_launches[k] = c.kind_launches[k];
    out->kind_gpu_s[k] = c.kind_gpu_s[k];
    out->kind_alg_bytes[k] = c.kind_alg_bytes[k];
  }
  return POLFED_OK;
}

void polfed_opts_default(polfed_opts* o) {
  if (!o) return;
  o->p = 0.17;
  o->k_margin = 0.2;
  o->tol_conv = 1e-7;
  o->tol_resid = 1e-8;
  o->cols_factor = 2.8;
  o->precision = POLFED_DF64;
  o->bounds_steps = 600;
  o->verbose = 0;
  o->dos_rule = POLFED_DOS_MOMENTS;
  o->seed = 1234;
  o->rho_hint = 0.0;
  o->emin_hint = 0.0;
  o->emax_hint = 0.0;
  o->kpm_moments = 256;
  o->kpm_vectors = 16;
  o->tol_refine = 0.0;
}

int polfed_basis_build(int32_t L, int32_t n_up, uint32_t* d_states, int64_t* dim, polfed_stream_t stream) {
  t_err.clear();
  if (L < 2 || L > 32) return fail(POLFED_EINVAL, "L must be in 2..32");
  if (n_up < 0 || n_up > L) return fail(POLFED_EINVAL, "n_up must be in 0..L");
  if (!dim) return fail(POLFED_EINVAL, "dim is NULL");
  const int64_t d = (int64_t)binom_host(L, n_up);
  *dim = d;
  if (!d_states) return POLFED_OK;
  return launch_basis(L, n_up, d_states, d, (cudaStream_t)stream);
}

int polfed_h_apply(const polfed_model* model, const uint32_t* d_states, int64_t dim, double e_lo, double e_hi,
                   const void* d_X, void* d_Y, int32_t n_b, int32_t dtype, polfed_stream_t stream) {
  t_err.clear();
  PF_CHECK(check_block_args(model, d_states, dim, d_X, d_Y, n_b, dtype));
  PF_CHECK(check_bounds(e_lo, e_hi));
  cudaStream_t s = (cudaStream_t)stream;
  HamPlan plan;
  PF_CHECK(plan.init(model, s, true));
  PF_CHECK(plan.prepare_typed(dtype, e_lo, e_hi));
  const int lpr = choose_lpr(dtype, n_b);
  StreamScratch mem;
  mem.s = s;
  FilterScratch scr;
  scr.bytes = filter_scratch_bytes(plan, dtype, lpr);
  PF_CUDA(cudaMallocAsync(&mem.p, scr.bytes, s));
  scr.xs = mem.p;
  PF_CHECK(apply_block(plan, dtype, d_X, d_Y, n_b, dtype == POLFED_F32 ? POLFED_F32 : POLFED_F64, scr, s, lpr));
  PF_CUDA(cudaStreamSynchronize(s));
  return POLFED_OK;
}

int polfed_cheb_filter(const polfed_model* model, const uint32_t* d_states, int64_t dim, double e_lo, double e_hi,
                       double sigma, int32_t K, const double* coeffs, const void* d_X, void* d_Y, int32_t n_b,
                       int32_t dtype, polfed_stream_t stream) {
  t_err.clear();
  PF_CHECK(check_block_args(model, d_states, dim, d_X, d_Y, n_b, dtype));
  PF_CHECK(check_bounds(e_lo, e_hi));
  if (K < 0 || K > 10000000) return fail(POLFED_EINVAL, "K must be in 0..1e7");
  if (!coeffs && !(sigma > -1.0 && sigma < 1.0)) return fail(POLFED_EINVAL, "sigma must be in (-1, 1)");
  std::vector<double> c;
  double invD = 1.0;
  if (coeffs) {
    c.assign(coeffs, coeffs + K + 1);
    for (double v : c)
      if (!std::isfinite(v)) return fail(POLFED_EINVAL, "non-finite coefficient");
  } else {
    double D = 1.0;
    cheb_coeffs(sigma, K, c, D);
    invD = 1.0 / D;
  }
  double csum = 0.0;
  for (double v : c) csum += std::fabs(v);
  cudaStream_t s = (cudaStream_t)stream;
  HamPlan plan;
  PF_CHECK(plan.init(model, s, true));
  PF_CHECK(plan.prepare_typed(dtype, e_lo, e_hi));
  const int lpr = choose_lpr(dtype, n_b);
  StreamScratch mem;
  mem.s = s;
  FilterScratch scr;
  scr.bytes = filter_scratch_bytes(plan, dtype, lpr);
  PF_CUDA(cudaMallocAsync(&mem.p, scr.bytes, s));
  scr.xs = mem.p;
  PF_CHECK(filter_block(plan, dtype, c.data(), K, invD, d_X, d_Y, n_b, dtype == POLFED_F32 ? POLFED_F32 : POLFED_F64,
                        scr, s, lpr));
  float flag[3] = {0, 0, 0};
  PF_CUDA(cudaMemcpyAsync(flag, scr.flag, sizeof(flag), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  int bad = 0;
  memcpy(&bad, &flag[2], 4);
  // |T_n| <= 1 on [-1, 1]  =>  ||y||_2 <= (sum |c_n| / D) ||x||_2 <= (sum |c_n| / D) sqrt(N) max|x|
  const double bound = csum * invD * std::sqrt((double)dim) * (double)flag[0] * 1.01 + 1e-300;
  if (bad || (double)flag[1] > bound)
    return fail(POLFED_EBOUNDS, "filter output grew beyond the Chebyshev bound: spectrum outside [e_lo, e_hi]");
  return POLFED_OK;
}

int polfed_cheb_filter_cols(const polfed_model* model, const uint32_t* d_states, int64_t dim, double e_lo,
                            double e_hi, int32_t K, const double* coeffs, const void* d_X, void* d_Y, int32_t n_b,
                            polfed_stream_t stream) {
  clear_error();
  PF_CHECK(check_block_args(model, d_states, dim, d_X, d_Y, n_b, POLFED_F32));
  PF_CHECK(check_bounds(e_lo, e_hi));
  if (K < 1 || K > 10000000) return fail(POLFED_EINVAL, "K must be in 1..1e7");
  if (!coeffs) return fail(POLFED_EINVAL, "coeffs is NULL");
  const int W = slice_width(POLFED_F32, choose_lpr(POLFED_F32, n_b));
  const int nsl = (n_b + W - 1) / W;
  std::vector<float> cf((size_t)nsl * (K + 1) * W, 0.f);
  for (int j = 0; j < n_b; j++)
    for (int n = 0; n <= K; n++) {
      const double v = coeffs[(size_t)j * (K + 1) + n];
      if (!std::isfinite(v)) return fail(POLFED_EINVAL, "non-finite coefficient");
      cf[((size_t)(j / W) * (K + 1) + n) * W + (j % W)] = (float)v;
    }
  cudaStream_t s = (cudaStream_t)stream;
  HamPlan plan;
  PF_CHECK(plan.init(model, s, true));
  PF_CHECK(plan.prepare_typed(POLFED_F32, e_lo, e_hi));
  const int lpr = choose_lpr(POLFED_F32, n_b);
  StreamScratch mem, cmem;
  mem.s = s;
  cmem.s = s;
  FilterScratch scr;
  scr.bytes = filter_scratch_bytes(plan, POLFED_F32, lpr);
  PF_CUDA(cudaMallocAsync(&mem.p, scr.bytes, s));
  scr.xs = mem.p;
  PF_CUDA(cudaMallocAsync(&cmem.p, cf.size() * sizeof(float), s));
  PF_CUDA(cudaMemcpyAsync(cmem.p, cf.data(), cf.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  PF_CHECK(filter_block_cols(plan, (const float*)cmem.p, K, d_X, d_Y, n_b, POLFED_F32, scr, s));
  float flag[3] = {0, 0, 0};
  PF_CUDA(cudaMemcpyAsync(flag, scr.flag, sizeof(flag), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  int bad = 0;
  memcpy(&bad, &flag[2], 4);
  if (bad) return fail(POLFED_EBOUNDS, "filter output is not finite: spectrum outside [e_lo, e_hi]");
  return POLFED_OK;
}

}  // extern "C"
