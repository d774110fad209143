// Block Lanczos on P^K_sigma(H~) (Eqs. (3)-(4)) and the whole POLFED run.
//
//   U_j = P Q_j - Q_{j-1} B_j^T,  A_j = Q_j^T U_j,  R_{j+1} = U_j - Q_j A_j,  Q_{j+1} B_{j+1} = R_{j+1}
//
// with U_j re-orthogonalized against all of Q_1..Q_j "between (3) and (4)"
// (block classical Gram-Schmidt, two passes; the first pass's Q_j block is
// A_j and its Q_{j-1} block is B_j^T, since Q_j^T Q_{j-1} = 0), QR by
// Cholesky QR applied twice, and the block tridiagonal
// T_m = Q_m^T P Q_m (A_j on the diagonal, B_j below, B_j^T above).
// Convergence: ||B_{j+1} t~_i|| for Ritz values theta_i >= p, t~_i the last
// s components of the eigenvector t_i of T_m (text after Eq. (4)).
// Ritz vectors u_i = Q_m t_i; eigenvalues u_i^T H~ u_i after a Rayleigh-Ritz
// step with H~ on the span of the converged Ritz vectors; residuals
// ||H~ u_i - eps_i u_i||.
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "dense.h"
#include "polfed_internal.h"

using namespace polfed;

namespace {

bool debug_on() {
  static const bool v = [] {
    const char* e = getenv("POLFED_DEBUG");
    return e && e[0] == '1';
  }();
  return v;
}

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  int ensure(size_t need, size_t* total, size_t limit) {
    if (p && n >= need) return POLFED_OK;
    if (p) {
      cudaFree(p);
      if (total) *total -= n;
    }
    p = nullptr;
    n = 0;
    if (limit && total && *total + need > limit) return fail(POLFED_ENOMEM, "context workspace limit exceeded");
    if (cudaMalloc(&p, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(POLFED_ENOMEM, "cudaMalloc of " + std::to_string(need) + " bytes failed");
    }
    n = need;
    if (total) *total += need;
    return POLFED_OK;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  template <class T>
  T* as() const {
    return (T*)p;
  }
};

}  // namespace

struct polfed_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cusolverDnHandle_t solver = nullptr;
  size_t ws_limit = 0, ws_total = 0;
  polfed_opts opts;
  bool have_opts = false;
  DevBuf basis, U, R, fscr, ritz, small, evbuf, work, vecs, kpm, coefbuf;
  Dense dense;
  polfed_stats last;
  polfed_progress_fn progress = nullptr;
  void* progress_user = nullptr;
  int block_steps = 0;  // block-Lanczos steps of the current run (over restarts), for the hook's index
  std::vector<polfed_conv_point> hist;  // convergence checks of the last call
  int attempt = 0;                      // attempt index recorded in hist
};

namespace {

struct ScopedDevice {
  int prev = 0;
  explicit ScopedDevice(int d) {
    cudaGetDevice(&prev);
    cudaSetDevice(d);
  }
  ~ScopedDevice() { cudaSetDevice(prev); }
};

// Phase boundary: the stream is drained first so that the hook sees the step's work complete.
void notify(polfed_ctx* c, int phase, int index) {
  if (!c->progress) return;
  cudaStreamSynchronize(c->stream);
  c->progress(c->progress_user, phase, index);
}

// Symmetric eigen-solve of the n x n column-major matrix A (lda) on the
// device with cuSOLVER (the projected problem); A is overwritten by the
// eigenvectors, w receives the eigenvalues ascending.
int syevd(polfed_ctx* c, double* A, int n, int lda, double* w) {
  int lwork = 0;
  if (cusolverDnDsyevd_bufferSize(c->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, A, lda, w,
                                  &lwork) != CUSOLVER_STATUS_SUCCESS)
    return fail(POLFED_ECUDA, "cusolverDnDsyevd_bufferSize failed");
  PF_CHECK(c->work.ensure((size_t)(lwork + 16) * sizeof(double), &c->ws_total, c->ws_limit));
  int* info = (int*)(c->work.as<double>() + lwork);
  if (cusolverDnDsyevd(c->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n, A, lda, w,
                       c->work.as<double>(), lwork, info) != CUSOLVER_STATUS_SUCCESS)
    return fail(POLFED_ECUDA, "cusolverDnDsyevd failed");
  int hinfo = 0;
  PF_CUDA(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PF_CUDA(cudaStreamSynchronize(c->stream));
  if (hinfo != 0) return fail(POLFED_ECUDA, "syevd info = " + std::to_string(hinfo));
  return POLFED_OK;
}

int round_block(int n_b) {
  if (n_b <= 16) return 16;
  if (n_b <= 32) return 32;
  if (n_b <= 64) return 64;
  return 128;
}

// gather columns idx of a column-major matrix V (ld) into a column-major out (ld_out)
__global__ void k_gather_cols(const double* V, int ld, const int* idx, int ncol, int nrow, double* out, int ld_out) {
  const int64_t tot = (int64_t)ncol * nrow;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / nrow), r = (int)(e % nrow);
    out[(int64_t)c * ld_out + r] = V[(int64_t)idx[c] * ld + r];
  }
}

// Exact mean and variance of the spectrum of the block: Tr H / N and
// Tr H^2 / N - mean^2 = <d^2> + <sum of squared off-diagonals per row> - mean^2.
__global__ void k_moments(const HamGeometry g, const uint16_t* U_lo, const int32_t* T_hi, const double* F_lo,
                          const double* F_hi, const double* C_x, double* out) {
  double s1 = 0.0, s2 = 0.0, so = 0.0;
  const double w1 = 0.25 * g.J1 * g.J1, w2 = 0.25 * g.J2 * g.J2;
  for (int grp = blockIdx.x; grp < (1 << g.nh); grp += gridDim.x) {
    if (T_hi[grp] < 0) continue;
    const int n_lo = g.n_up - __popc(grp);
    const int n_g = g.cls_off[n_lo + 1] - g.cls_off[n_lo];
    for (int loc = threadIdx.x; loc < n_g; loc += blockDim.x) {
      const uint32_t s_lo = U_lo[g.cls_off[n_lo] + loc];
      uint32_t pattern = 0;
      double off = 0.0;
      for (int k = 0; k < g.n_cross; k++) {
        const int hb = (grp >> g.cross_hi[k]) & 1;
        if ((int)((s_lo >> g.cross_lo[k]) & 1) != hb) {
          pattern |= 1u << k;
          off += g.cross_cls[k] == 1 ? w1 : w2;
        }
      }
      for (int k = 0; k < g.n_low1 + g.n_low2; k++)
        if (__popc(s_lo & g.low_mask[k]) == 1) off += k < g.n_low1 ? w1 : w2;
      for (int k = 0; k < g.n_high1 + g.n_high2; k++)
        if (__popc((uint32_t)grp & g.high_mask[k]) == 1) off += k < g.n_high1 ? w1 : w2;
      const double d = F_lo[s_lo] + F_hi[grp] + C_x[pattern];
      s1 += d;
      s2 += d * d;
      so += off;
    }
  }
  atomicAdd(out + 0, s1);
  atomicAdd(out + 1, s2);
  atomicAdd(out + 2, so);
}

double lobe_root(double p) {
  // first positive root of sin(y)/y = p (main lobe of the Dirichlet kernel)
  double a = 1e-6, b = M_PI;
  for (int i = 0; i < 200; i++) {
    double m = 0.5 * (a + b);
    if (std::sin(m) / m > p)
      a = m;
    else
      b = m;
  }
  return 0.5 * (a + b);
}

struct LanczosParams {
  double e_lo, e_hi, sigma;
  int K, S, N_ev;
  polfed_opts o;
  double tol_resid_t;  // acceptance threshold on ||H~ u - eps u||
  bool accept_any;     // accept the first verified set (FP32 stage before refinement)
  bool fill_panels;    // top the converged set up to whole panels (input of the refinement)
  FilterHook* hook = nullptr;  // batched runner: filter calls go through it
  double guard_dp = 0.02;      // Ritz vectors with theta >= p - guard_dp enter the Rayleigh-Ritz step
                               // (wider guards, tried for strict refinement targets, made the sweeps stall)
};

// Y_q = invD sum_n coef[n] T_n(H~) X_q for the panels q (dim x S each), directly
// or through the batched runner's rendezvous.
int run_filter(HamPlan& plan, const LanczosParams& P, int kind, const double* coef, int K, double invD,
               const double* const* in, double* const* out, int npan, int S, FilterScratch& scr, cudaStream_t s,
               int lpr) {
  if (P.hook && (kind == POLFED_F32 || kind == POLFED_DF64))
    return P.hook->filter(plan, kind, coef, K, invD, in, out, npan, S, s);
  for (int q = 0; q < npan; q++)
    PF_CHECK(filter_block(plan, kind, coef, K, invD, in[q], out[q], S, POLFED_F64, scr, s, lpr));
  return POLFED_OK;
}

struct LanczosOut {
  std::vector<double> evals_t;  // H~ units, ascending
  std::vector<double> resid_t;  // H~ units
  int n_out = 0, m = 0, n_conv = 0, checks = 0, ritz_cols = 0, n_refine = 0, refine_K = 0;
  int n_acc = -1;  // Ritz values theta >= p at the last check (converged or not); -1 = no check yet
  int64_t matvec_cols = 0;
  double t_filter = 0, t_reorth = 0, t_qr = 0, t_teig = 0, t_ritz = 0;
};

int extract(polfed_ctx* c, HamPlan& plan, const LanczosParams& P, const double* Qb, int m_done,
            const std::vector<double>& theta, const std::vector<double>& tres, double tol_sel, double* d_evecs,
            LanczosOut& out);

int run_lanczos(polfed_ctx* c, HamPlan& plan, const LanczosParams& P, double* d_evecs, LanczosOut& out) {
  cudaStream_t s = c->stream;
  const int64_t dim = plan.geo.dim;
  const int S = P.S;
  const int kind = P.o.precision == POLFED_F32 ? POLFED_F32 : (P.o.precision == POLFED_F64 ? POLFED_F64 : POLFED_DF64);
  if (P.N_ev < 1 || P.N_ev > dim) return fail(POLFED_EINVAL, "N_ev must be in 1..dim");
  int m_max = (int)std::ceil(P.o.cols_factor * (1.0 + P.o.k_margin) * P.N_ev / S) + 1;
  // block Lanczos needs polynomial degree (steps) as well as columns: the
  // accessible pairs start converging once ms ~ 2.2 (1 + k_margin) N_ev and
  // then gain one to two digits per step, so allow 12 steps past that onset
  const int onset = (int)std::ceil(2.2 * (1.0 + P.o.k_margin) * P.N_ev / S);
  m_max = std::max(std::max(m_max, 24), onset + 12);
  m_max = (int)std::min<int64_t>(m_max, dim / S);
  if (m_max < 1) return fail(POLFED_EINVAL, "dimension too small for this block size");
  Dense& D = c->dense;
  D.dim = dim;
  D.S = S;
  PF_CHECK(D.configure());
  const int64_t pstride = dim * S;
  PF_CHECK(c->basis.ensure((size_t)(m_max + 1) * pstride * sizeof(double), &c->ws_total, c->ws_limit));
  PF_CHECK(c->U.ensure((size_t)pstride * sizeof(double), &c->ws_total, c->ws_limit));
  const int lpr = choose_lpr(kind, S);
  PF_CHECK(c->fscr.ensure(filter_scratch_bytes(plan, kind, lpr), &c->ws_total, c->ws_limit));
  PF_CHECK(plan.prepare_typed(kind, P.e_lo, P.e_hi));
  FilterScratch scr;
  scr.xs = c->fscr.p;
  scr.bytes = c->fscr.n;
  std::vector<double> coef;
  double Dn = 1.0;
  cheb_coeffs(P.sigma, P.K, coef, Dn);
  const double invD = 1.0 / Dn;
  double* Qb = c->basis.as<double>();
  double* Ub = c->U.as<double>();
  // Q_1: random orthonormal N x s
  PF_CHECK(D.random_fill(Qb, pstride, P.o.seed, s));
  bool brk = false;
  PF_CHECK(D.cholqr(Qb, Qb, nullptr, 2, s, &brk));
  if (brk) return fail(POLFED_ECUDA, "random start block is rank deficient");
  std::vector<std::vector<double>> A, B;  // A_j, B_{j+1} (row-major S x S)
  // device buffers for projections (max (m_max+1) S x S) and T
  const size_t cmax = (size_t)(m_max + 1) * S * S;
  PF_CHECK(c->small.ensure((cmax + 16) * sizeof(double), &c->ws_total, c->ws_limit));
  double* Cdev = c->small.as<double>();
  std::vector<double> Chost((size_t)S * S);
  std::vector<double> theta, tres;
  std::vector<int> conv_idx;
  int status = POLFED_OK;
  int m_done = 0;
  bool stopped = false;
  const double p = P.o.p;
  double tol_cur = P.o.tol_conv;
  std::vector<double> colnrm(S);
  auto step_done = [&] { notify(c, POLFED_PHASE_BLOCK, c->block_steps++); };
  for (int j = 0; j < m_max; j++) {
    double* Qj = Qb + (int64_t)j * pstride;
    double t0 = now_s();
    {
      const double* in1[1] = {Qj};
      double* out1[1] = {Ub};
      PF_CHECK(run_filter(plan, P, kind, coef.data(), P.K, invD, in1, out1, 1, S, scr, s, lpr));
    }
    PF_CHECK(D.coldot(Ub, Ub, S, colnrm.data(), s));  // synchronizes
    out.matvec_cols += (int64_t)P.K * S;
    double t1 = now_s();
    out.t_filter += t1 - t0;
    for (int q = 0; q < S; q++)
      if (!std::isfinite(colnrm[q]) || colnrm[q] > 1.0 + 1e-6)
        return fail(POLFED_EBOUNDS, "filtered block norm exceeds 1: spectrum outside [e_lo, e_hi]");
    // pass 1: C = Q_{0..j}^T U; A_j = sym(C_j); U -= Q C
    PF_CHECK(D.gram(Qb, pstride, j + 1, Ub, Cdev, S, 0, s));
    PF_CUDA(cudaMemcpyAsync(Chost.data(), Cdev + (size_t)j * S * S, (size_t)S * S * sizeof(double),
                            cudaMemcpyDeviceToHost, s));
    PF_CHECK(D.update(Qb, pstride, j + 1, Cdev, S, 1, S, Ub, 0, -1.0, 1.0, s));
    // pass 2
    PF_CHECK(D.gram(Qb, pstride, j + 1, Ub, Cdev, S, 0, s));
    PF_CHECK(D.update(Qb, pstride, j + 1, Cdev, S, 1, S, Ub, 0, -1.0, 1.0, s));
    PF_CUDA(cudaStreamSynchronize(s));
    std::vector<double> Aj((size_t)S * S);
    for (int a = 0; a < S; a++)
      for (int b = 0; b < S; b++) Aj[(size_t)a * S + b] = 0.5 * (Chost[(size_t)a * S + b] + Chost[(size_t)b * S + a]);
    A.push_back(Aj);
    double t2 = now_s();
    out.t_reorth += t2 - t1;
    // QR: Q_{j+1} B_{j+1} = R
    std::vector<double> Bn((size_t)S * S);
    double* Qn = Qb + (int64_t)(j + 1) * pstride;
    PF_CHECK(D.cholqr(Ub, Qn, Bn.data(), 2, s, &brk));
    B.push_back(Bn);
    if (debug_on()) {
      // orthogonality of the new panel against Q_0 and itself
      double* Ct = Cdev;
      std::vector<double> h((size_t)S * S), h0((size_t)S * S);
      PF_CHECK(D.gram(Qn, 0, 1, Qn, Ct, S, 0, s));
      PF_CUDA(cudaMemcpyAsync(h.data(), Ct, (size_t)S * S * 8, cudaMemcpyDeviceToHost, s));
      PF_CUDA(cudaStreamSynchronize(s));
      PF_CHECK(D.gram(Qb, 0, 1, Qn, Ct, S, 0, s));
      PF_CUDA(cudaMemcpyAsync(h0.data(), Ct, (size_t)S * S * 8, cudaMemcpyDeviceToHost, s));
      PF_CUDA(cudaStreamSynchronize(s));
      double e1 = 0, e0 = 0, bn = 0, tr = 0, cm = 0;
      for (int a = 0; a < S; a++)
        for (int b = 0; b < S; b++) {
          e1 = std::max(e1, std::fabs(h[(size_t)a * S + b] - (a == b)));
          e0 = std::max(e0, std::fabs(h0[(size_t)a * S + b]));
          bn += Bn[(size_t)a * S + b] * Bn[(size_t)a * S + b];
        }
      for (int a = 0; a < S; a++) tr += Aj[(size_t)a * S + a], cm = std::max(cm, colnrm[a]);
      fprintf(stderr, "[polfed dbg] j=%d  max|U col|^2=%.3e  trA=%.4e  |B|_F=%.3e  |QnQn-I|=%.2e  |Q0Qn|=%.2e\n", j, cm,
              tr, std::sqrt(bn), e1, e0);
    }
    double t3 = now_s();
    out.t_qr += t3 - t2;
    m_done = j + 1;
    if (brk) {
      status = fail(POLFED_ENOCONV, "Lanczos breakdown (rank-deficient residual block)");
      step_done();
      break;
    }
    // convergence check
    const int n = m_done * S;
    const bool last = (j == m_max - 1);
    if (n < (int)((1.0 + P.o.k_margin) * P.N_ev) && !last) {
      step_done();
      continue;
    }
    std::vector<double> T((size_t)n * n, 0.0);  // column-major, symmetric
    for (int i = 0; i < m_done; i++) {
      for (int a = 0; a < S; a++)
        for (int b = 0; b < S; b++) T[(size_t)(i * S + b) * n + i * S + a] = A[i][(size_t)a * S + b];
      if (i + 1 < m_done)
        for (int a = 0; a < S; a++)
          for (int b = 0; b < S; b++) {
            const double v = B[i][(size_t)a * S + b];  // B_{i+1}: block (i+1, i)
            T[(size_t)(i * S + b) * n + (i + 1) * S + a] = v;
            T[(size_t)((i + 1) * S + a) * n + i * S + b] = v;
          }
    }
    PF_CHECK(c->evbuf.ensure(((size_t)n * n + n) * sizeof(double), &c->ws_total, c->ws_limit));
    double* Td = c->evbuf.as<double>();
    double* wd = Td + (size_t)n * n;
    PF_CUDA(cudaMemcpyAsync(Td, T.data(), (size_t)n * n * sizeof(double), cudaMemcpyHostToDevice, s));
    PF_CHECK(syevd(c, Td, n, n, wd));
    out.checks++;
    theta.assign(n, 0.0);
    PF_CUDA(cudaMemcpyAsync(theta.data(), wd, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
    // last S rows of every eigenvector
    std::vector<double> tail((size_t)S * n);
    PF_CUDA(cudaMemcpy2DAsync(tail.data(), S * sizeof(double), Td + (size_t)(m_done - 1) * S, (size_t)n * sizeof(double),
                              S * sizeof(double), n, cudaMemcpyDeviceToHost, s));
    PF_CUDA(cudaStreamSynchronize(s));
    tres.assign(n, 0.0);
    const std::vector<double>& Bl = B.back();
    for (int i = 0; i < n; i++) {
      double ss = 0.0;
      for (int a = 0; a < S; a++) {
        double v = 0.0;
        for (int b = 0; b < S; b++) v += Bl[(size_t)a * S + b] * tail[(size_t)i * S + b];
        ss += v * v;
      }
      tres[i] = std::sqrt(ss);
    }
    out.t_teig += now_s() - t3;
    // stopping rule: the N_ev largest Ritz values are >= p and all converged
    std::vector<int> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return theta[x] > theta[y]; });
    int nconv_p = 0;
    for (int i = 0; i < n; i++)
      if (theta[i] >= p && tres[i] <= tol_cur) nconv_p++;
    const bool ok_theta = n >= P.N_ev && theta[ord[P.N_ev - 1]] >= p;  // N_ev accessible values found
    double maxres_top = 0.0;
    for (int k = 0; k < std::min(n, P.N_ev); k++) maxres_top = std::max(maxres_top, tres[ord[k]]);
    const bool ok = ok_theta && maxres_top <= tol_cur;
    out.n_conv = nconv_p;
    out.n_acc = 0;
    for (int i = 0; i < n; i++) out.n_acc += theta[i] >= p;
    {
      polfed_conv_point cp;
      memset(&cp, 0, sizeof(cp));
      cp.step = j + 1;
      cp.cols = n;
      cp.n_conv = nconv_p;
      cp.n_acc = out.n_acc;
      cp.attempt = c->attempt;
      cp.theta_nev = n >= P.N_ev ? theta[ord[P.N_ev - 1]] : -1.0;
      cp.max_res_top = maxres_top;
      c->hist.push_back(cp);
    }
    if (debug_on()) {
      fprintf(stderr, "[polfed dbg] check n=%d: top theta/res:", n);
      for (int k = 0; k < std::min(n, 12); k++) fprintf(stderr, " %.4f/%.1e", theta[ord[k]], tres[ord[k]]);
      fprintf(stderr, "\n   around N_ev:");
      for (int k = std::max(0, P.N_ev - 4); k < std::min(n, P.N_ev + 4); k++)
        fprintf(stderr, " %.4f/%.1e", theta[ord[k]], tres[ord[k]]);
      fprintf(stderr, "\n");
    }
    if (P.o.verbose)
      fprintf(stderr, "[polfed] step %d  cols %d  n_conv(theta>=p) %d  theta_Nev %.4f  max_res_top %.2e\n", j + 1, n,
              nconv_p, n >= P.N_ev ? theta[ord[P.N_ev - 1]] : -1.0,
              [&] {
                double mr = 0;
                for (int k = 0; k < std::min(n, P.N_ev); k++) mr = std::max(mr, tres[ord[k]]);
                return mr;
              }());
    if (ok || (last && ok_theta)) {
      // verify by the residuals of the Rayleigh-Ritz pairs (text after Eq. (4))
      const double t5 = now_s();
      const double tol_sel = std::max(tol_cur, maxres_top);  // all N_ev top pairs, plus converged guards
      const int erc = extract(c, plan, P, Qb, m_done, theta, tres, tol_sel, d_evecs, out);
      out.t_ritz += now_s() - t5;
      if (erc != POLFED_OK) return erc;
      double mr = 0.0;
      for (double r : out.resid_t) mr = std::max(mr, r);
      if (P.o.verbose || debug_on())
        fprintf(stderr, "[polfed] verify at step %d: %d pairs, max resid (H~) %.3e, target %.3e\n", j + 1, out.n_out, mr,
                P.tol_resid_t);
      if (out.n_out >= P.N_ev && (mr <= P.tol_resid_t || P.accept_any)) {
        stopped = true;
        step_done();
        break;
      }
      tol_cur = 0.1 * std::min(tol_cur, maxres_top);  // not accurate enough yet: demand smaller Ritz residuals
    }
    step_done();
  }
  out.m = m_done;
  if (!stopped && status == POLFED_OK) status = fail(POLFED_ENOCONV, "column budget exhausted before convergence");
  if (status == POLFED_OK && out.n_out < P.N_ev) status = fail(POLFED_ENOCONV, "fewer converged pairs than requested");
  return status;
}

// Ritz vectors of the converged pairs (theta >= p - 0.02, ||B t~|| <= tol_sel),
// Rayleigh-Ritz with H~ on their span, the N_ev pairs nearest sigma, residuals.
// The Lanczos basis is left intact (outputs live in the ritz buffer).
// Rayleigh-Ritz with H~ on the span of the nr (orthonormal) columns of U
// (panel-major, ncols padded to panels with zero columns), the N_ev pairs
// nearest sigma, their residual norms ||H~ u - eps u|| (text after Eq. (4)).
// Uses the Wr/Uo/Wo regions of the ritz buffer; writes out.* and d_evecs.
// Regions of the ritz buffer, in panels of dim x S doubles (npan = ceil(nr / S),
// opan = ceil(min(nr, N_ev) / S)): U [npan] | W = H~ U [npan] | F, a filtered
// block [npan] | the selected pairs Uo [opan] and their images Wo [opan].  The
// refinement's residual block T [npan] shares the last region with Uo / Wo
// (T is consumed before they are written).
struct RitzLayout {
  double *U, *Wr, *F, *Uo, *Wo, *T;
  static size_t panels(int S, int nr, int N_ev) {
    const size_t npan = (nr + S - 1) / S, opan = (std::min(nr, N_ev) + S - 1) / S;
    return 3 * npan + std::max(2 * opan, npan);
  }
  RitzLayout(double* base, int64_t dim, int S, int nr, int N_ev) {
    const size_t pst = (size_t)dim * S, npan = (nr + S - 1) / S, opan = (std::min(nr, N_ev) + S - 1) / S;
    U = base;
    Wr = base + npan * pst;
    F = base + 2 * npan * pst;
    Uo = base + 3 * npan * pst;
    Wo = Uo + opan * pst;
    T = Uo;
  }
};

int rr_select(polfed_ctx* c, HamPlan& plan, const LanczosParams& P, const double* U, int nr, double* d_evecs,
              LanczosOut& out) {
  cudaStream_t s = c->stream;
  Dense& D = c->dense;
  const int64_t dim = plan.geo.dim;
  const int S = P.S;
  const int64_t pstride = dim * S;
  const int npan = (nr + S - 1) / S;
  const int nr_pad = npan * S;
  const int nout = std::min(nr, P.N_ev);
  const int opan = (nout + S - 1) / S;
  double* base = c->ritz.as<double>();
  const RitzLayout Rl(base, dim, S, nr, P.N_ev);
  double* Wr = Rl.Wr;  // H~ U
  double* Uo = Rl.Uo;  // selected eigenvectors
  double* Wo = Rl.Wo;  // their images
  PF_CHECK(plan.prepare_typed(POLFED_F64, P.e_lo, P.e_hi));
  const int lpr64 = choose_lpr(POLFED_F64, S);
  PF_CHECK(c->fscr.ensure(std::max(c->fscr.n, filter_scratch_bytes(plan, POLFED_F64, lpr64)), &c->ws_total,
                          c->ws_limit));
  FilterScratch scr64;
  scr64.xs = c->fscr.p;
  scr64.bytes = c->fscr.n;
  for (int q = 0; q < npan; q++)
    PF_CHECK(apply_block(plan, POLFED_F64, U + (size_t)q * pstride, Wr + (size_t)q * pstride, S, POLFED_F64, scr64, s,
                         lpr64));
  out.matvec_cols += nr_pad;
  // G = U^T W (nr_pad x nr_pad); the eigen-solve of its leading nr x nr block
  PF_CHECK(c->evbuf.ensure(((size_t)nr_pad * nr_pad + nr_pad) * sizeof(double), &c->ws_total, c->ws_limit));
  double* G = c->evbuf.as<double>();
  double* lam = G + (size_t)nr_pad * nr_pad;
  for (int q = 0; q < npan; q++) PF_CHECK(D.gram(U, pstride, npan, Wr + (size_t)q * pstride, G, nr_pad, q * S, s));
  PF_CHECK(syevd(c, G, nr, nr_pad, lam));
  std::vector<double> lamh(nr);
  PF_CUDA(cudaMemcpyAsync(lamh.data(), lam, nr * sizeof(double), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  // the N_ev nearest sigma, ascending
  std::vector<int> sel(nr);
  std::iota(sel.begin(), sel.end(), 0);
  std::stable_sort(sel.begin(), sel.end(),
                   [&](int x, int y) { return std::fabs(lamh[x] - P.sigma) < std::fabs(lamh[y] - P.sigma); });
  sel.resize(nout);
  std::sort(sel.begin(), sel.end());
  PF_CHECK(c->vecs.ensure(((size_t)nr_pad * nout + 64) * sizeof(double) + (size_t)nr_pad * sizeof(int), &c->ws_total,
                          c->ws_limit));
  double* Ysel = c->vecs.as<double>();
  int* idx_d = (int*)(Ysel + (size_t)nr_pad * nout + 64);
  PF_CUDA(cudaMemcpyAsync(idx_d, sel.data(), nout * sizeof(int), cudaMemcpyHostToDevice, s));
  // rows nr..nr_pad-1 multiply the zero padding columns of U/W: make them 0, not stale memory
  PF_CUDA(cudaMemsetAsync(Ysel, 0, (size_t)nr_pad * nout * sizeof(double), s));
  k_gather_cols<<<1024, 256, 0, s>>>(G, nr_pad, idx_d, nout, nr, Ysel, nr_pad);
  PF_CUDA(cudaGetLastError());
  count_launch();
  PF_CHECK(D.update(U, pstride, npan, Ysel, 1, nr_pad, nout, Uo, pstride, 1.0, 0.0, s));
  PF_CHECK(D.update(Wr, pstride, npan, Ysel, 1, nr_pad, nout, Wo, pstride, 1.0, 0.0, s));
  std::vector<double> lsel(opan * S, 0.0);
  for (int i = 0; i < nout; i++) lsel[i] = lamh[sel[i]];
  double* lsel_d = lam;  // reuse
  PF_CUDA(cudaMemcpyAsync(lsel_d, lsel.data(), lsel.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  out.evals_t.assign(nout, 0.0);
  out.resid_t.assign(nout, 0.0);
  std::vector<double> rn(S);
  for (int q = 0; q < opan; q++) {
    PF_CHECK(D.resid(Uo + (size_t)q * pstride, Wo + (size_t)q * pstride, lsel_d + q * S, s));
    PF_CHECK(D.coldot(Wo + (size_t)q * pstride, Wo + (size_t)q * pstride, S, rn.data(), s));
    for (int k = 0; k < S && q * S + k < nout; k++) out.resid_t[q * S + k] = std::sqrt(std::max(0.0, rn[k]));
  }
  for (int i = 0; i < nout; i++) out.evals_t[i] = lsel[i];
  if (d_evecs) PF_CHECK(D.panels_to_colmajor(Uo, nout, d_evecs, s));
  PF_CUDA(cudaStreamSynchronize(s));
  out.n_out = nout;
  return POLFED_OK;
}

// Room in the ritz buffer for U, H~U, the selected pairs and a filtered copy of U.
int ensure_ritz(polfed_ctx* c, int64_t dim, int S, int nr, int N_ev) {
  return c->ritz.ensure(RitzLayout::panels(S, nr, N_ev) * (size_t)dim * S * sizeof(double), &c->ws_total,
                        c->ws_limit);
}

// Ritz vectors u_i = Q_m t_i of the converged pairs (theta >= p - 0.02,
// ||B t~|| <= tol_sel), then rr_select.  With fill_panels the set is topped up
// with the next Ritz vectors by theta to whole panels (a full-rank block for
// the refinement sweeps).  The Lanczos basis is left intact.
int extract(polfed_ctx* c, HamPlan& plan, const LanczosParams& P, const double* Qb, int m_done,
            const std::vector<double>& theta, const std::vector<double>& tres, double tol_sel, double* d_evecs,
            LanczosOut& out) {
  cudaStream_t s = c->stream;
  Dense& D = c->dense;
  const int64_t dim = plan.geo.dim;
  const int S = P.S;
  const int64_t pstride = dim * S;
  const int n = m_done * S;
  const double p_rr = P.o.p - P.guard_dp;
  std::vector<int> conv_idx;
  std::vector<char> used(n, 0);
  // the FP32 stage (accept_any) hands every accessible Ritz vector to the
  // refinement: subspace iteration needs the window's neighbours in the block
  for (int i = 0; i < n; i++)
    if (theta[i] >= p_rr && (tres[i] <= tol_sel || P.accept_any)) {
      conv_idx.push_back(i);
      used[i] = 1;
    }
  if (conv_idx.empty()) {
    out.n_out = 0;
    out.evals_t.clear();
    out.resid_t.clear();
    return POLFED_OK;
  }
  if (P.fill_panels) {
    std::vector<int> rest;
    for (int i = 0; i < n; i++)
      if (!used[i]) rest.push_back(i);
    std::sort(rest.begin(), rest.end(), [&](int x, int y) { return theta[x] > theta[y]; });
    size_t k = 0;
    while (conv_idx.size() % S && k < rest.size()) conv_idx.push_back(rest[k++]);
  }
  const int nr = (int)conv_idx.size();
  const int npan = (nr + S - 1) / S;
  // T eigenvectors are in c->evbuf (column-major n x n)
  double* Td = c->evbuf.as<double>();
  PF_CHECK(c->vecs.ensure(((size_t)n * npan * S + 64) * sizeof(double) + (size_t)npan * S * sizeof(int), &c->ws_total,
                          c->ws_limit));
  double* Vsel = c->vecs.as<double>();
  int* idx_d = (int*)(Vsel + (size_t)n * npan * S + 64);
  PF_CUDA(cudaMemcpyAsync(idx_d, conv_idx.data(), nr * sizeof(int), cudaMemcpyHostToDevice, s));
  k_gather_cols<<<1024, 256, 0, s>>>(Td, n, idx_d, nr, n, Vsel, n);
  PF_CUDA(cudaGetLastError());
  count_launch();
  PF_CHECK(ensure_ritz(c, dim, S, nr, P.N_ev));
  double* Ur = c->ritz.as<double>();  // npan panels
  PF_CHECK(D.update(Qb, pstride, m_done, Vsel, 1, n, nr, Ur, pstride, 1.0, 0.0, s));
  out.ritz_cols = nr;
  return rr_select(c, plan, P, Ur, nr, d_evecs, out);
}

// Jackson damping factors g_n of an order-N Chebyshev expansion (kernel
// polynomial method; Weisse, Wellein, Alvermann, Fehske, Rev. Mod. Phys. 78,
// 275 (2006), Eq. (71)).
static void jackson(int N, std::vector<double>& g) {
  g.resize(N + 1);
  const double a = M_PI / (N + 1);
  for (int n = 0; n <= N; n++) g[n] = ((N - n + 1) * std::cos(a * n) + std::sin(a * n) / std::tan(a)) / (N + 1);
}

// End of a refinement sweep: the filtered block F (nr columns in panels, ritz
// buffer region F) is orthonormalized panel by panel (block Gram-Schmidt twice
// + Cholesky QR twice), copied to region 0 and handed to rr_select.  The
// padding columns of the last panel are exactly zero and stay zero.
int finish_sweep(polfed_ctx* c, HamPlan& plan, const LanczosParams& P, double* F, int nr, double* d_evecs,
                 LanczosOut& out) {
  cudaStream_t s = c->stream;
  Dense& D = c->dense;
  const int S = P.S;
  const int64_t pstride = plan.geo.dim * S;
  const int npan = (nr + S - 1) / S;
  const double t1 = now_s();
  PF_CHECK(c->small.ensure(std::max(c->small.n, ((size_t)npan * S * S + 16) * sizeof(double)), &c->ws_total,
                           c->ws_limit));
  double* Cd = c->small.as<double>();
  bool brk = false;
  for (int q = 0; q < npan; q++) {
    double* Fq = F + (size_t)q * pstride;
    for (int pass = 0; pass < 2 && q > 0; pass++) {
      PF_CHECK(D.gram(F, pstride, q, Fq, Cd, S, 0, s));
      PF_CHECK(D.update(F, pstride, q, Cd, S, 1, S, Fq, 0, -1.0, 1.0, s));
    }
    PF_CHECK(D.cholqr(Fq, Fq, nullptr, 2, s, &brk));
    const bool padded = (q == npan - 1) && (nr % S != 0);  // zero columns trip the pivot test by design
    if (brk && !padded) return fail(POLFED_ENOCONV, "refinement block lost rank");
  }
  out.t_reorth += now_s() - t1;
  double* U = c->ritz.as<double>();
  PF_CUDA(cudaMemcpyAsync(U, F, (size_t)npan * pstride * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return rr_select(c, plan, P, U, nr, d_evecs, out);
}

// One refinement sweep by defect correction, with the filter in FP32.  For a
// unit vector u with Rayleigh value lam and residual r = H~ u - lam u, and any
// polynomial P, P(H~) u = P(lam) u + g(H~) r with g(x) = (P(x) - P(lam)) /
// (x - lam), a polynomial of degree Kr - 1.  Only g(H~) r goes through the
// FP32 Chebyshev filter; since |r| is small (the FP32 stage leaves |r| about
// 1e-6), its FP32 rounding error is that much smaller than that of an FP32
// filter of u, and the sweep costs an FP32 filter of the block.  Steps: the
// Rayleigh-Ritz basis of span(U) with H~ in FP64 (u_i, lam_i, r_i for all nr
// columns), the Chebyshev coefficients of each column's g by synthetic
// division (FP64, host), the per-column FP32 filter of the residual block,
// W = U diag(P(lam)) + g(H~) R, then orthonormalization and Rayleigh-Ritz
// (finish_sweep).  P is the Jackson-damped order-Kr transform of Eq. (2).
// Columns whose residual is already at most tol_lock are locked: they skip
// the filter (W_i = P(lam_i) u_i, the same scale) and stay in the block for
// the orthonormalization and Rayleigh-Ritz, so a sweep filters only the
// columns still converging.
int refine_dd(polfed_ctx* c, HamPlan& plan, const LanczosParams& P, int Kr, int nr, double tol_lock,
              double* d_evecs, LanczosOut& out, int* n_filtered) {
  cudaStream_t s = c->stream;
  Dense& D = c->dense;
  const int64_t dim = plan.geo.dim;
  const int S = P.S;
  const int64_t pstride = dim * S;
  const int npan = (nr + S - 1) / S;
  const int nr_pad = npan * S;
  PF_CHECK(ensure_ritz(c, dim, S, nr, P.N_ev));
  const RitzLayout R(c->ritz.as<double>(), dim, S, nr, P.N_ev);
  const double t0 = now_s();
  // 1. Rayleigh-Ritz basis of span(U): W = H~ U (FP64), G = U^T W = Y diag(lam) Y^T
  PF_CHECK(plan.prepare_typed(POLFED_F64, P.e_lo, P.e_hi));
  const int lpr64 = choose_lpr(POLFED_F64, S);
  PF_CHECK(c->fscr.ensure(std::max(c->fscr.n, filter_scratch_bytes(plan, POLFED_F64, lpr64)), &c->ws_total,
                          c->ws_limit));
  FilterScratch scr64;
  scr64.xs = c->fscr.p;
  scr64.bytes = c->fscr.n;
  for (int q = 0; q < npan; q++)
    PF_CHECK(apply_block(plan, POLFED_F64, R.U + (size_t)q * pstride, R.Wr + (size_t)q * pstride, S, POLFED_F64, scr64,
                         s, lpr64));
  out.matvec_cols += nr_pad;
  PF_CHECK(c->evbuf.ensure(((size_t)nr_pad * nr_pad + nr_pad) * sizeof(double), &c->ws_total, c->ws_limit));
  double* G = c->evbuf.as<double>();
  double* lam_d = G + (size_t)nr_pad * nr_pad;
  for (int q = 0; q < npan; q++) PF_CHECK(D.gram(R.U, pstride, npan, R.Wr + (size_t)q * pstride, G, nr_pad, q * S, s));
  PF_CHECK(syevd(c, G, nr, nr_pad, lam_d));
  std::vector<double> lam(nr_pad, 0.0);
  PF_CUDA(cudaMemcpyAsync(lam.data(), lam_d, nr * sizeof(double), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  // 2. F = U Y, T = W Y - F diag(lam): the Ritz vectors and their residuals (padding columns zero)
  PF_CUDA(cudaMemsetAsync(R.F, 0, (size_t)npan * pstride * sizeof(double), s));
  PF_CUDA(cudaMemsetAsync(R.T, 0, (size_t)npan * pstride * sizeof(double), s));
  PF_CHECK(D.update(R.U, pstride, npan, G, 1, nr_pad, nr, R.F, pstride, 1.0, 0.0, s));
  PF_CHECK(D.update(R.Wr, pstride, npan, G, 1, nr_pad, nr, R.T, pstride, 1.0, 0.0, s));
  PF_CUDA(cudaMemcpyAsync(lam_d, lam.data(), nr_pad * sizeof(double), cudaMemcpyHostToDevice, s));
  for (int q = 0; q < npan; q++) PF_CHECK(D.resid(R.F + (size_t)q * pstride, R.T + (size_t)q * pstride, lam_d + q * S, s));
  // 3. residual norms: the columns above the lock threshold are filtered, packed into whole panels
  std::vector<double> rn(nr_pad, 0.0);
  for (int q = 0; q < npan; q++)
    PF_CHECK(D.coldot(R.T + (size_t)q * pstride, R.T + (size_t)q * pstride, S, rn.data() + (size_t)q * S, s));
  std::vector<int> idx, pos(nr_pad, -1);
  for (int i = 0; i < nr; i++)
    if (!(std::sqrt(std::max(0.0, rn[i])) <= tol_lock)) {
      pos[i] = (int)idx.size();
      idx.push_back(i);
    }
  const int nc = (int)idx.size();
  const int npc = (nc + S - 1) / S;
  *n_filtered = nc;
  if (debug_on())
    fprintf(stderr, "[polfed] defect-correction sweep (Kr %d): %d of %d columns filtered, %d locked\n", Kr, nc, nr,
            nr - nc);
  // 4. coefficients: a_n of the damped transform, and per filtered column the synthetic
  //    division g = (P - P(lam)) / (x - lam) in the Chebyshev basis, from the top:
  //    d_{Kr-1} = 2 a_Kr, d_{n-1} = 2 (a_n + lam d_n) - d_{n+1} (n >= 2), d_0 = a_1 + lam d_1 - d_2 / 2
  //    (x T_0 = T_1, x T_m = (T_{m+1} + T_{m-1}) / 2)
  std::vector<double> a, gj;
  double Dn = 1.0;
  cheb_coeffs(P.sigma, Kr, a, Dn);
  jackson(Kr, gj);
  for (int n = 0; n <= Kr; n++) a[n] *= gj[n] / Dn;
  const int Kg = Kr - 1;                                                // degree of g
  const int W32 = slice_width(POLFED_F32, choose_lpr(POLFED_F32, S));  // columns per FP32 slice
  const int nsl = (S + W32 - 1) / W32;                                  // slices per panel
  const size_t per_panel = (size_t)nsl * (Kg + 1) * W32;
  std::vector<float> coef((size_t)npc * per_panel, 0.f);
  std::vector<double> pl(nr_pad, 0.0), d(Kr + 2);
  for (int i = 0; i < nr; i++) {
    const double l = lam[i];
    // P(lam) by Clenshaw in FP64
    double b1 = 0.0, b2 = 0.0;
    for (int n = Kr; n >= 1; n--) {
      const double b0 = a[n] + 2.0 * l * b1 - b2;
      b2 = b1;
      b1 = b0;
    }
    pl[i] = a[0] + l * b1 - b2;
    if (pos[i] < 0) continue;
    std::fill(d.begin(), d.end(), 0.0);
    d[Kr - 1] = 2.0 * a[Kr];
    for (int n = Kr - 1; n >= 2; n--) d[n - 1] = 2.0 * (a[n] + l * d[n]) - d[n + 1];
    if (Kr >= 2) d[0] = a[1] + l * d[1] - 0.5 * d[2];
    const int j = pos[i], q = j / S, col = j % S, sl = col / W32, jj = col % W32;
    float* base = coef.data() + (size_t)q * per_panel + (size_t)sl * (Kg + 1) * W32;
    for (int n = 0; n <= Kg; n++) base[(size_t)n * W32 + jj] = (float)d[n];
  }
  const size_t coef_bytes = (coef.size() * sizeof(float) + 255) & ~(size_t)255;
  PF_CHECK(c->coefbuf.ensure(coef_bytes + ((size_t)nr_pad + nc + 64) * sizeof(int), &c->ws_total, c->ws_limit));
  float* coef_d = c->coefbuf.as<float>();
  int* pos_d = reinterpret_cast<int*>(reinterpret_cast<char*>(coef_d) + coef_bytes);
  int* idx_d = pos_d + nr_pad;
  if (!coef.empty())
    PF_CUDA(cudaMemcpyAsync(coef_d, coef.data(), coef.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  PF_CUDA(cudaMemcpyAsync(pos_d, pos.data(), (size_t)nr_pad * sizeof(int), cudaMemcpyHostToDevice, s));
  if (nc > 0) PF_CUDA(cudaMemcpyAsync(idx_d, idx.data(), (size_t)nc * sizeof(int), cudaMemcpyHostToDevice, s));
  PF_CUDA(cudaMemcpyAsync(lam_d, pl.data(), nr_pad * sizeof(double), cudaMemcpyHostToDevice, s));
  const double t1 = now_s();
  out.t_ritz += t1 - t0;
  // 5. Wr = the filtered columns of T, packed; T = g(H~) Wr per column, FP32
  if (nc > 0) {
    PF_CHECK(D.gather_cols(R.T, idx_d, nc, npc * S, R.Wr, s));
    PF_CHECK(plan.prepare_typed(POLFED_F32, P.e_lo, P.e_hi));
    const int lpr32 = choose_lpr(POLFED_F32, S);
    PF_CHECK(c->fscr.ensure(std::max(c->fscr.n, filter_scratch_bytes(plan, POLFED_F32, lpr32)), &c->ws_total,
                            c->ws_limit));
    FilterScratch scr;
    scr.xs = c->fscr.p;
    scr.bytes = c->fscr.n;
    for (int q = 0; q < npc; q++)
      PF_CHECK(filter_block_cols(plan, coef_d + (size_t)q * per_panel, Kg, R.Wr + (size_t)q * pstride,
                                 R.T + (size_t)q * pstride, S, POLFED_F64, scr, s));
    out.matvec_cols += (int64_t)Kg * nc;
  }
  // 6. F_i = P(lam_i) u_i + g_i(H~) r_i (locked columns: P(lam_i) u_i), the filtered block
  PF_CHECK(D.scale_add_cols(R.F, R.T, pos_d, lam_d, npan, s));
  PF_CUDA(cudaStreamSynchronize(s));
  out.t_filter += now_s() - t1;
  return finish_sweep(c, plan, P, R.F, nr, d_evecs, out);
}

// Single-vector Lanczos on H for E_min and E_max (text before Eq. (3)).
int spectral_bounds(polfed_ctx* c, HamPlan& plan, const polfed_opts& o, double* emin, double* emax, double* err,
                    int64_t* matvecs) {
  cudaStream_t s = c->stream;
  const int64_t dim = plan.geo.dim;
  PF_CHECK(plan.prepare_typed(POLFED_F64, 0.0, 0.0));
  const int lpr = choose_lpr(POLFED_F64, 1);
  PF_CHECK(c->fscr.ensure(std::max(c->fscr.n, filter_scratch_bytes(plan, POLFED_F64, lpr)), &c->ws_total, c->ws_limit));
  FilterScratch scr;
  scr.xs = c->fscr.p;
  scr.bytes = c->fscr.n;
  PF_CHECK(c->R.ensure((size_t)3 * dim * sizeof(double), &c->ws_total, c->ws_limit));
  double* v0 = c->R.as<double>();
  double* v1 = v0 + dim;
  double* w = v1 + dim;
  Dense& D = c->dense;
  D.dim = dim;
  PF_CHECK(D.random_fill(v1, dim, o.seed ^ 0x5bd1e995ull, s));
  double nrm = 0.0;
  PF_CHECK(D.coldot(v1, v1, 1, &nrm, s));
  PF_CHECK(D.axpbypcz(dim, 0.0, v1, 1.0 / std::sqrt(nrm), v1, 0.0, nullptr, s));
  PF_CUDA(cudaMemsetAsync(v0, 0, dim * sizeof(double), s));
  std::vector<double> al, be;  // be[k] couples k and k+1
  double beta = 0.0;
  const int kmax = (int)std::min<int64_t>(o.bounds_steps, dim);
  double lo = 0, hi = 0, e_lo = 1e300, e_hi = 1e300;
  for (int k = 0; k < kmax; k++) {
    PF_CHECK(apply_block(plan, POLFED_F64, v1, w, 1, POLFED_F64, scr, s, lpr));
    (*matvecs)++;
    double a = 0.0;
    PF_CHECK(D.coldot(v1, w, 1, &a, s));
    al.push_back(a);
    PF_CHECK(D.axpbypcz(dim, -a, v1, 1.0, w, -beta, v0, s));
    double bb = 0.0;
    PF_CHECK(D.coldot(w, w, 1, &bb, s));
    beta = std::sqrt(std::max(bb, 0.0));
    be.push_back(beta);
    const int m = k + 1;
    const bool check = (m >= 20 && m % 20 == 0) || m == kmax || beta < 1e-300;
    if (check) {
      // eigen-solve of the m x m tridiagonal
      std::vector<double> T((size_t)m * m, 0.0);
      for (int i = 0; i < m; i++) {
        T[(size_t)i * m + i] = al[i];
        if (i + 1 < m) T[(size_t)i * m + i + 1] = T[(size_t)(i + 1) * m + i] = be[i];
      }
      PF_CHECK(c->evbuf.ensure(((size_t)m * m + m) * sizeof(double), &c->ws_total, c->ws_limit));
      double* Td = c->evbuf.as<double>();
      PF_CUDA(cudaMemcpyAsync(Td, T.data(), (size_t)m * m * sizeof(double), cudaMemcpyHostToDevice, s));
      PF_CHECK(syevd(c, Td, m, m, Td + (size_t)m * m));
      std::vector<double> ev(m), y0(m), y1(m);
      PF_CUDA(cudaMemcpyAsync(ev.data(), Td + (size_t)m * m, m * sizeof(double), cudaMemcpyDeviceToHost, s));
      double last_lo = 0, last_hi = 0;
      PF_CUDA(cudaMemcpyAsync(&last_lo, Td + (size_t)0 * m + (m - 1), sizeof(double), cudaMemcpyDeviceToHost, s));
      PF_CUDA(cudaMemcpyAsync(&last_hi, Td + (size_t)(m - 1) * m + (m - 1), sizeof(double), cudaMemcpyDeviceToHost, s));
      PF_CUDA(cudaStreamSynchronize(s));
      lo = ev[0];
      hi = ev[m - 1];
      e_lo = std::fabs(beta * last_lo);
      e_hi = std::fabs(beta * last_hi);
      const double scale = std::max(std::fabs(lo), std::fabs(hi));
      if ((e_lo <= 1e-12 * scale && e_hi <= 1e-12 * scale) || beta < 1e-300) break;
    }
    if (beta < 1e-300) break;
    // v0 <- v1, v1 <- w / beta
    std::swap(v0, v1);
    PF_CHECK(D.axpbypcz(dim, 1.0 / beta, w, 0.0, v1, 0.0, nullptr, s));
  }
  *emin = lo;
  *emax = hi;
  *err = std::max(e_lo, e_hi);
  return POLFED_OK;
}

// Density of states per unit of H~ at sigma (whole sector) from the KPM
// eigenvalue count of the window [sigma - d, sigma + d], d = max(0.01, 8 / n_mom)
// (a few Jackson widths pi / n_mom), with R random vectors of seed.
int kpm_rho(polfed_ctx* c, HamPlan& plan, double e_lo, double e_hi, double sigma, int n_mom, int R, uint64_t seed,
            double* rho_t, int64_t* matvecs) {
  cudaStream_t s = c->stream;
  const int64_t dim = plan.geo.dim;
  const int kind = POLFED_DF64;
  PF_CHECK(plan.prepare_typed(kind, e_lo, e_hi));
  const int lpr = choose_lpr(kind, R);
  PF_CHECK(c->fscr.ensure(std::max(c->fscr.n, filter_scratch_bytes(plan, kind, lpr)), &c->ws_total, c->ws_limit));
  FilterScratch scr;
  scr.xs = c->fscr.p;
  scr.bytes = c->fscr.n;
  const size_t vb = ((size_t)dim * R * sizeof(double) + 255) & ~(size_t)255;
  PF_CHECK(c->kpm.ensure(vb + kpm_buffer_bytes(dim, R, POLFED_F64), &c->ws_total, c->ws_limit));
  double* r = c->kpm.as<double>();
  PF_CHECK(c->dense.random_fill(r, dim * R, seed ^ 0x6b706d5f646f73ull, s));
  const KpmBuffers b = kpm_carve((char*)c->kpm.p + vb, dim, R, POLFED_F64);
  std::vector<double> mu(n_mom);
  PF_CHECK(kpm_moments(plan, kind, r, R, n_mom, mu.data(), b, scr, s));
  *matvecs += (int64_t)R * ((n_mom + 1) / 2);
  const double d = std::max(0.01, 8.0 / n_mom);
  const double xa = std::max(-1.0, sigma - d), xb = std::min(1.0, sigma + d);
  const double f = kpm_count_fraction(mu.data(), n_mom, xa, xb);
  *rho_t = std::max(f, 1e-12) * (double)dim / (xb - xa);
  return POLFED_OK;
}

int moments(polfed_ctx* c, HamPlan& plan, double* mean, double* var) {
  cudaStream_t s = c->stream;
  PF_CHECK(c->small.ensure(std::max(c->small.n, (size_t)64), &c->ws_total, c->ws_limit));
  double* out = c->small.as<double>();
  PF_CUDA(cudaMemsetAsync(out, 0, 3 * sizeof(double), s));
  k_moments<<<std::min(plan.geo.n_groups + 0, 152 * 4), 256, 0, s>>>(plan.geo, plan.tab.U_lo, plan.tab.T_hi,
                                                                      plan.tab.F_lo, plan.tab.F_hi, plan.tab.C_x, out);
  PF_CUDA(cudaGetLastError());
  count_launch();
  double h[3];
  PF_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  const double n = (double)plan.geo.dim;
  *mean = h[0] / n;
  *var = h[1] / n - (*mean) * (*mean) + h[2] / n;
  return POLFED_OK;
}

}  // namespace

extern "C" {

int polfed_ctx_create(int32_t device, size_t workspace_bytes, polfed_ctx** out) {
  if (!out) return fail(POLFED_EINVAL, "out is NULL");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return fail(POLFED_EINVAL, "invalid CUDA device");
  }
  ScopedDevice sd(device);
  polfed_ctx* c = new polfed_ctx();
  c->device = device;
  c->ws_limit = workspace_bytes;
  polfed_opts_default(&c->opts);
  memset(&c->last, 0, sizeof(c->last));
  if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return fail(POLFED_ECUDA, "cudaStreamCreate failed");
  }
  c->own_stream = true;
  if (cusolverDnCreate(&c->solver) != CUSOLVER_STATUS_SUCCESS) {
    cudaStreamDestroy(c->stream);
    delete c;
    return fail(POLFED_ECUDA, "cusolverDnCreate failed");
  }
  cusolverDnSetStream(c->solver, c->stream);
  *out = c;
  return POLFED_OK;
}

void polfed_ctx_destroy(polfed_ctx* c) {
  if (!c) return;
  ScopedDevice sd(c->device);
  cudaStreamSynchronize(c->stream);
  c->basis.release();
  c->U.release();
  c->R.release();
  c->fscr.release();
  c->ritz.release();
  c->small.release();
  c->evbuf.release();
  c->work.release();
  c->vecs.release();
  c->kpm.release();
  c->coefbuf.release();
  c->dense.release();
  if (c->solver) cusolverDnDestroy(c->solver);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

int polfed_ctx_set_stream(polfed_ctx* c, polfed_stream_t stream) {
  if (!c) return fail(POLFED_EINVAL, "ctx is NULL");
  ScopedDevice sd(c->device);
  if (c->own_stream && c->stream) {
    cudaStreamSynchronize(c->stream);
    cudaStreamDestroy(c->stream);
  }
  c->stream = (cudaStream_t)stream;
  c->own_stream = false;
  cusolverDnSetStream(c->solver, c->stream);
  return POLFED_OK;
}

int polfed_block_lanczos(polfed_ctx* c, const polfed_model* model, double e_lo, double e_hi, double sigma, int32_t K,
                         int32_t n_b, int32_t N_ev, double* d_evecs, double* evals, double* resid, int32_t* n_conv) {
  if (!c) return fail(POLFED_EINVAL, "ctx is NULL");
  if (!evals) return fail(POLFED_EINVAL, "evals is NULL");
  if (!(e_lo < e_hi) || !std::isfinite(e_lo) || !std::isfinite(e_hi)) return fail(POLFED_EINVAL, "need e_lo < e_hi");
  if (!(sigma > -1.0 && sigma < 1.0)) return fail(POLFED_EINVAL, "sigma must be in (-1, 1)");
  if (K < 1 || K > 10000000) return fail(POLFED_EINVAL, "K must be in 1..1e7");
  if (n_b < 1 || n_b > 128) return fail(POLFED_EINVAL, "n_b must be in 1..128");
  ScopedDevice sd(c->device);
  HamPlan plan;
  PF_CHECK(plan.init(model, c->stream, false));
  const double hn = std::max(std::fabs(e_lo), std::fabs(e_hi));
  LanczosParams P{e_lo, e_hi, sigma, K, round_block(n_b), N_ev, c->opts, c->opts.tol_resid * hn / (0.5 * (e_hi - e_lo)),
                  false, false};
  LanczosOut o;
  const double t0 = now_s();
  c->block_steps = 0;
  c->hist.clear();
  c->attempt = 0;
  int rc = run_lanczos(c, plan, P, d_evecs, o);
  if (rc != POLFED_OK && rc != POLFED_ENOCONV) return rc;
  const double half = 0.5 * (e_hi - e_lo), mid = 0.5 * (e_hi + e_lo);
  for (int i = 0; i < o.n_out; i++) {
    evals[i] = o.evals_t[i] * half + mid;
    if (resid) resid[i] = o.resid_t[i] * half;
  }
  if (n_conv) *n_conv = o.n_out;
  polfed_stats& st = c->last;
  memset(&st, 0, sizeof(st));
  st.K = K;
  st.m = o.m;
  st.n_b = P.S;
  st.n_conv = o.n_conv;
  st.n_ritz_checks = o.checks;
  st.dim = plan.geo.dim;
  st.matvec_cols = o.matvec_cols;
  st.e_lo = e_lo;
  st.e_hi = e_hi;
  st.sigma = sigma;
  st.t_filter = o.t_filter;
  st.t_reorth = o.t_reorth;
  st.t_qr = o.t_qr;
  st.t_teig = o.t_teig;
  st.t_ritz = o.t_ritz;
  st.t_total = now_s() - t0;
  st.status = rc;
  for (int i = 0; i < o.n_out; i++) st.max_resid = std::max(st.max_resid, o.resid_t[i] * half);
  notify(c, POLFED_PHASE_END, rc);
  return rc;
}

int polfed_ctx_history(polfed_ctx* c, polfed_conv_point* out, int32_t max, int32_t* n) {
  if (!c || !n) return fail(POLFED_EINVAL, "ctx or n is NULL");
  *n = (int32_t)c->hist.size();
  if (out)
    for (int32_t i = 0; i < std::min<int32_t>(max, *n); i++) out[i] = c->hist[i];
  return POLFED_OK;
}

int polfed_ctx_set_progress(polfed_ctx* c, polfed_progress_fn fn, void* user) {
  if (!c) return fail(POLFED_EINVAL, "ctx is NULL");
  c->progress = fn;
  c->progress_user = user;
  return POLFED_OK;
}

int polfed_eigs(polfed_ctx* c, const polfed_model* model, double eps_target, int32_t N_ev, int32_t K, int32_t n_b,
                const polfed_opts* opts, double* evals, double* d_evecs, double* resid, polfed_stats* stats) {
  return polfed::eigs_impl(c, model, eps_target, N_ev, K, n_b, opts, evals, d_evecs, resid, stats, nullptr);
}

}  // extern "C"

namespace polfed {

cudaStream_t ctx_stream(polfed_ctx* c) { return c->stream; }
void* ctx_solver(polfed_ctx* c) { return c->solver; }
int ctx_device(polfed_ctx* c) { return c->device; }

int eigs_impl(polfed_ctx* c, const polfed_model* model, double eps_target, int32_t N_ev, int32_t K, int32_t n_b,
              const polfed_opts* opts, double* evals, double* d_evecs, double* resid, polfed_stats* stats,
              FilterHook* hook) {
  if (!c) return fail(POLFED_EINVAL, "ctx is NULL");
  if (!evals) return fail(POLFED_EINVAL, "evals is NULL");
  if (!(eps_target >= 0.0 && eps_target <= 1.0)) return fail(POLFED_EINVAL, "eps_target must be in [0, 1]");
  if (n_b < 1 || n_b > 128) return fail(POLFED_EINVAL, "n_b must be in 1..128");
  if (K < 0 || K > 10000000) return fail(POLFED_EINVAL, "K must be in 0..1e7");
  polfed_opts o;
  if (opts)
    o = *opts;
  else
    polfed_opts_default(&o);
  if (!(o.p > 0.0 && o.p < 1.0)) return fail(POLFED_EINVAL, "opts.p must be in (0, 1)");
  if (o.precision != POLFED_F64 && o.precision != POLFED_F32 && o.precision != POLFED_DF64)
    return fail(POLFED_EINVAL, "bad opts.precision");
  c->opts = o;
  c->have_opts = true;
  ScopedDevice sd(c->device);
  const double t0 = now_s();
  const Counters cn0 = counters();
  HamPlan plan;
  PF_CHECK(plan.init(model, c->stream, false, hook ? hook->plan_b(model->L) : -1));
  count_launch(4);  // table kernels
  const int64_t dim = plan.geo.dim;
  if (N_ev < 1 || N_ev > dim) return fail(POLFED_EINVAL, "N_ev must be in 1..dim");
  // 1. spectral bounds
  double Emin = 0, Emax = 0, berr = 0;
  int64_t mv = 0;
  PF_CHECK(spectral_bounds(c, plan, o, &Emin, &Emax, &berr, &mv));
  const double t_b = now_s() - t0;
  if (!(Emax > Emin)) return fail(POLFED_EINVAL, "degenerate spectrum (E_max == E_min)");
  const double width = Emax - Emin;
  const double pad = 1e-6 * width + 10.0 * berr;
  double e_lo = Emin - pad, e_hi = Emax + pad;
  int bounds_from_hint = 0;
  if (o.dos_rule == POLFED_DOS_HINT && o.emin_hint < o.emax_hint) {
    // predicted bounds: kept only if the probe confirms they contain the
    // spectrum (a bound inside it would make the recurrence grow) and they are
    // not looser than 5% of the width
    if (o.emin_hint <= Emin - 10.0 * berr && o.emax_hint >= Emax + 10.0 * berr &&
        o.emax_hint - o.emin_hint <= 1.05 * width) {
      e_lo = o.emin_hint;
      e_hi = o.emax_hint;
      bounds_from_hint = 1;
    }
  }
  const double Estar = Emin + eps_target * width;
  double sigma = (2.0 * Estar - e_lo - e_hi) / (e_hi - e_lo);
  if (std::fabs(sigma) < 1e-14) sigma = 0.0;
  if (!(sigma > -1.0 && sigma < 1.0)) return fail(POLFED_EINVAL, "target outside the spectrum");
  // 2. order K from the density of states at the target
  double mean = 0, var = 0, rho = 0.0, rho_t = 0.0;
  switch (o.dos_rule) {
    case POLFED_DOS_MOMENTS: {
      PF_CHECK(moments(c, plan, &mean, &var));
      const double gam = std::sqrt(std::max(var, 1e-300));
      rho = (double)dim / (std::sqrt(2.0 * M_PI) * gam) * std::exp(-0.5 * (Estar - mean) * (Estar - mean) / (gam * gam));
      rho_t = rho * 0.5 * (e_hi - e_lo);
      break;
    }
    case POLFED_DOS_GAMMA: {
      // analytic infinite-temperature width of Eq. (1) (Supplement: Gamma^2 =
      // L [(1 + J2^2)/8 + Delta^2 (1 + J2^2)/16 + W^2/12] for J1 = 1), per
      // realization (sum h_i^2 / 4 in place of L W^2 / 12) and per bond count
      // (nb_l terms of class l), centred at the exact sector mean: in the
      // S^z = 0 sector <S^z_i S^z_j> = -1 / (4 (L - 1)) for i != j.
      const polfed_model& md = *model;
      const double nb1 = md.periodic ? md.L : md.L - 1, nb2 = md.periodic ? md.L : md.L - 2;
      double hh = 0.0;
      for (int i = 0; i < md.L; i++) hh += md.h[i] * md.h[i];
      var = (nb1 * md.J1 * md.J1 + nb2 * md.J2 * md.J2) * (1.0 / 8.0 + md.Delta * md.Delta / 16.0) + hh / 4.0;
      mean = -md.Delta * (nb1 * md.J1 + nb2 * md.J2) / (4.0 * (md.L - 1));
      const double gam = std::sqrt(var);
      rho = (double)dim / (std::sqrt(2.0 * M_PI) * gam) * std::exp(-0.5 * (Estar - mean) * (Estar - mean) / (gam * gam));
      rho_t = rho * 0.5 * (e_hi - e_lo);
      break;
    }
    case POLFED_DOS_KPM: {
      const int nm = o.kpm_moments > 0 ? o.kpm_moments : 256;
      const int nv = o.kpm_vectors > 0 ? o.kpm_vectors : 16;
      if (nm < 16 || nm > kMaxKpmMoments || nv > 128) return fail(POLFED_EINVAL, "bad kpm_moments / kpm_vectors");
      PF_CHECK(kpm_rho(c, plan, e_lo, e_hi, sigma, nm, nv, o.seed, &rho_t, &mv));
      rho = rho_t / (0.5 * (e_hi - e_lo));
      break;
    }
    case POLFED_DOS_HINT: {
      if (!(o.rho_hint > 0.0) || !std::isfinite(o.rho_hint)) return fail(POLFED_EINVAL, "rho_hint must be > 0");
      rho = o.rho_hint * (double)dim / width;
      rho_t = rho * 0.5 * (e_hi - e_lo);
      break;
    }
    default:
      return fail(POLFED_EINVAL, "bad opts.dos_rule");
  }
  const double gam = std::sqrt(std::max(var, 0.0));
  const int K_auto = (K == 0);
  if (K == 0) {
    const double y = lobe_root(o.p);
    const double n_target = (1.0 + o.k_margin) * N_ev;
    double k1 = 2.0 * y * std::sqrt(1.0 - sigma * sigma) * rho_t / n_target;  // K + 1
    int k = (int)std::floor(k1 - 1.0);
    if (sigma == 0.0) k &= ~1;
    K = std::max(2, std::min(k, 10000000));
  }
  if (o.verbose || debug_on())
    fprintf(stderr, "[polfed] dim %lld  E_min %.12f  E_max %.12f (err %.1e)  sigma %.3e  mean %.4f  Gamma %.4f  rho~ %.4e  K %d\n",
            (long long)dim, Emin, Emax, berr, sigma, mean, gam, rho_t, K);
  // 3. block Lanczos
  c->block_steps = 0;
  c->hist.clear();
  c->attempt = 0;
  notify(c, POLFED_PHASE_START, K);
  const int S = round_block(n_b);
  const double hnorm0 = std::max(std::fabs(Emin), std::fabs(Emax));
  const bool mixed = o.precision == POLFED_F32;
  LanczosParams P{e_lo, e_hi, sigma, K, S, N_ev, o, o.tol_resid * hnorm0 / (0.5 * (e_hi - e_lo)), mixed, false};
  P.hook = hook;
  if (mixed) P.o.tol_conv = std::max(o.tol_conv, 2e-5);  // FP32 filter: stop at its noise floor
  LanczosOut lo;
  int rc = POLFED_OK, restarts = 0, fallback = 0;
  for (;;) {
    LanczosOut cur;
    rc = run_lanczos(c, plan, P, d_evecs, cur);
    if (restarts > 0) {  // the work of the abandoned attempts still counts
      cur.matvec_cols += lo.matvec_cols;
      cur.checks += lo.checks;
      cur.t_filter += lo.t_filter;
      cur.t_reorth += lo.t_reorth;
      cur.t_qr += lo.t_qr;
      cur.t_teig += lo.t_teig;
      cur.t_ritz += lo.t_ritz;
    }
    lo = std::move(cur);
    if (rc != POLFED_ENOCONV || K_auto == 0 || restarts >= 2 || lo.n_acc < 0 || lo.n_acc >= N_ev) break;
    // Fewer than N_ev eigenvalues have P >= p: the density of states was
    // overestimated and K is too large for the window to hold N_ev.  Shrink K
    // so that the window holds about (1 + k_margin) N_ev of the values seen.
    const double f = std::max(0.25, 0.9 * std::max(lo.n_acc, 1) / ((1.0 + o.k_margin) * N_ev));
    int Kn = std::min((int)(K * f), (int)(0.8 * K));
    if (sigma == 0.0) Kn &= ~1;
    Kn = std::max(2, Kn);
    if (o.verbose || debug_on())
      fprintf(stderr, "[polfed] %d accessible eigenvalues < N_ev = %d: restart with K %d -> %d\n", lo.n_acc, N_ev, K,
              Kn);
    K = Kn;
    P.K = K;
    restarts++;
    c->attempt++;
  }
  if (rc != POLFED_OK && rc != POLFED_ENOCONV) return rc;
  if (mixed && lo.n_out > 0) {
    // refinement sweeps (defect correction with FP32 filters) until the residuals pass
    int Kr = std::max(16, K / 2);
    if (sigma == 0.0) Kr &= ~1;
    double mr_prev = 1e300;
    // sweeps continue to the refinement target (tol_refine, default tol_resid)
    const double tol_ref_t =
        (o.tol_refine > 0.0 ? std::min(o.tol_refine, o.tol_resid) : o.tol_resid) * hnorm0 / (0.5 * (e_hi - e_lo));
    // a target below tol_resid (eigenvector-derived observables) allows more sweeps; the
    // wanted pairs near the window's edge gain a roughly constant factor per sweep
    const bool strict = tol_ref_t < P.tol_resid_t;
    // a column whose residual is already half the target skips the next sweep's filter
    constexpr double kLockFrac = 0.5;
    const int max_sweeps = strict ? 40 : 24;
    // a float-float run in place of the sweeps costs about twice the FP32 stage's filter work
    const double fallback_cost = 2.0 * (double)std::max(lo.m, 1) * S * K;
    int n_filt = lo.ritz_cols;  // columns the next sweep filters, about
    for (int sweep = 0; sweep < max_sweeps; sweep++) {
      double mr = 0.0;
      for (double r : lo.resid_t) mr = std::max(mr, r);
      if (lo.n_out >= N_ev && mr <= tol_ref_t && sweep > 0) break;
      if (sweep >= 2 && mr > 0.0 && mr_prev > 0.0) {
        // from the second sweep on (order K) the worst residual falls by a steady factor per sweep
        const double r = mr / mr_prev;
        if (r > 0.95) break;  // stagnating: the block misses part of the wanted subspace
        // converging too slowly: the sweeps still needed at this rate, each filtering about as many
        // columns as the last one, would cost more than the float-float run
        if (!strict && mr > tol_ref_t &&
            std::log(tol_ref_t / mr) / std::log(r) * (double)n_filt * Kr > fallback_cost)
          break;
      }
      mr_prev = mr;
      if (o.verbose || debug_on())
        fprintf(stderr, "[polfed] refinement sweep %d: Kr %d, max resid (H~) before %.3e\n", sweep + 1, Kr, mr);
      const double tr0 = now_s();
      // the sweep's per-column filters launch on the context's own stream: a batched runner's
      // rendezvous stops waiting for this realization meanwhile
      if (hook) hook->suspend();
      const int rrc = refine_dd(c, plan, P, Kr, lo.ritz_cols, kLockFrac * tol_ref_t, d_evecs, lo, &n_filt);
      if (hook) hook->resume();
      lo.t_ritz += now_s() - tr0;
      if (rrc != POLFED_OK) return rrc;
      notify(c, POLFED_PHASE_REFINE, sweep);
      lo.n_refine++;
      lo.refine_K = Kr;
      Kr = std::min(2 * Kr, K);
      if (sigma == 0.0) Kr &= ~1;
    }
    double mr = 0.0;
    for (double r : lo.resid_t) mr = std::max(mr, r);
    rc = (lo.n_out >= N_ev && mr <= P.tol_resid_t) ? POLFED_OK
                                                   : fail(POLFED_ENOCONV, "refinement did not reach the residual target");
    if (rc != POLFED_OK) {
      // The FP32 stage missed part of the wanted subspace (refinement cannot
      // recover a direction the block does not contain): run the plain
      // float-float method instead.
      if (o.verbose || debug_on())
        fprintf(stderr, "[polfed] refinement stalled at %.3e (H~): float-float POLFED run\n", mr);
      LanczosParams P2 = P;
      P2.o.precision = POLFED_DF64;
      P2.o.tol_conv = o.tol_conv;
      P2.accept_any = false;
      c->attempt++;
      LanczosOut l2;
      rc = run_lanczos(c, plan, P2, d_evecs, l2);
      if (rc != POLFED_OK && rc != POLFED_ENOCONV) return rc;
      l2.matvec_cols += lo.matvec_cols;
      l2.checks += lo.checks;
      l2.t_filter += lo.t_filter;
      l2.t_reorth += lo.t_reorth;
      l2.t_qr += lo.t_qr;
      l2.t_teig += lo.t_teig;
      l2.t_ritz += lo.t_ritz;
      l2.n_refine = lo.n_refine;
      l2.refine_K = lo.refine_K;
      lo = std::move(l2);
      fallback = 1;
    }
  }
  const double half = 0.5 * (e_hi - e_lo), mid = 0.5 * (e_hi + e_lo);
  const double hnorm = std::max(std::fabs(Emin), std::fabs(Emax));
  polfed_stats st;
  memset(&st, 0, sizeof(st));
  for (int i = 0; i < lo.n_out; i++) {
    evals[i] = lo.evals_t[i] * half + mid;
    const double r = lo.resid_t[i] * half;
    if (resid) resid[i] = r;
    st.max_resid = std::max(st.max_resid, r);
  }
  st.K = K;
  st.m = lo.m;
  st.n_b = S;
  st.n_conv = lo.n_conv;
  st.n_ritz_checks = lo.checks;
  st.status = rc;
  st.n_refine = lo.n_refine;
  st.refine_K = lo.refine_K;
  st.dim = dim;
  st.matvec_cols = lo.matvec_cols + mv;
  st.E_min = Emin;
  st.E_max = Emax;
  st.e_lo = e_lo;
  st.e_hi = e_hi;
  st.sigma = sigma;
  st.target = Estar;
  st.rho_sigma = rho_t;
  st.t_bounds = t_b;
  st.n_restarts = restarts;
  st.fallback_df64 = fallback;
  st.dos_rule = o.dos_rule;
  st.bounds_from_hint = bounds_from_hint;
  st.t_filter = lo.t_filter;
  st.t_reorth = lo.t_reorth;
  st.t_qr = lo.t_qr;
  st.t_teig = lo.t_teig;
  st.t_ritz = lo.t_ritz;
  st.t_total = now_s() - t0;
  const Counters cn1 = counters();
  st.n_launches = cn1.launches - cn0.launches;
  st.n_step_launches = cn1.step_launches - cn0.step_launches;
  st.step_gpu_s = cn1.step_gpu_s - cn0.step_gpu_s;
  st.step_alg_bytes = cn1.step_alg_bytes - cn0.step_alg_bytes;
  for (int k = 0; k < 3; k++) {
    st.kind_launches[k] = cn1.kind_launches[k] - cn0.kind_launches[k];
    st.kind_gpu_s[k] = cn1.kind_gpu_s[k] - cn0.kind_gpu_s[k];
    st.kind_alg_bytes[k] = cn1.kind_alg_bytes[k] - cn0.kind_alg_bytes[k];
  }
  c->last = st;
  if (stats) *stats = st;
  if (rc == POLFED_OK && st.max_resid > o.tol_resid * hnorm && o.verbose)
    fprintf(stderr, "[polfed] warning: max residual %.3e exceeds tol %.3e\n", st.max_resid, o.tol_resid * hnorm);
  notify(c, POLFED_PHASE_END, rc);
  return rc;
}

}  // namespace polfed

extern "C" {

int polfed_spectral_bounds(polfed_ctx* c, const polfed_model* model, double* bounds) {
  if (!c) return fail(POLFED_EINVAL, "ctx is NULL");
  if (!bounds) return fail(POLFED_EINVAL, "bounds is NULL");
  ScopedDevice sd(c->device);
  HamPlan plan;
  PF_CHECK(plan.init(model, c->stream, false));
  polfed_opts o = c->opts;
  if (!c->have_opts) polfed_opts_default(&o);
  int64_t mv = 0;
  PF_CHECK(spectral_bounds(c, plan, o, &bounds[0], &bounds[1], &bounds[2], &mv));
  return POLFED_OK;
}

int polfed_spectral_labels(polfed_ctx* c, const polfed_model* model, double eps_target, int32_t n_mom, int32_t R,
                           double* out) {
  if (!c) return fail(POLFED_EINVAL, "ctx is NULL");
  if (!out) return fail(POLFED_EINVAL, "out is NULL");
  if (!(eps_target > 0.0 && eps_target < 1.0)) return fail(POLFED_EINVAL, "eps_target must be in (0, 1)");
  if (n_mom < 16 || n_mom > kMaxKpmMoments) return fail(POLFED_EINVAL, "n_mom must be in 16..65536");
  if (R < 1 || R > 128) return fail(POLFED_EINVAL, "R must be in 1..128");
  ScopedDevice sd(c->device);
  HamPlan plan;
  PF_CHECK(plan.init(model, c->stream, false));
  polfed_opts o = c->opts;
  if (!c->have_opts) polfed_opts_default(&o);
  double Emin = 0, Emax = 0, berr = 0;
  int64_t mv = 0;
  PF_CHECK(spectral_bounds(c, plan, o, &Emin, &Emax, &berr, &mv));
  if (!(Emax > Emin)) return fail(POLFED_EINVAL, "degenerate spectrum (E_max == E_min)");
  const double width = Emax - Emin;
  const double pad = 1e-6 * width + 10.0 * berr;
  const double e_lo = Emin - pad, e_hi = Emax + pad;
  const double Estar = Emin + eps_target * width;
  const double sigma = (2.0 * Estar - e_lo - e_hi) / (e_hi - e_lo);
  double rho_t = 0.0;
  PF_CHECK(kpm_rho(c, plan, e_lo, e_hi, sigma, n_mom, R, o.seed, &rho_t, &mv));
  out[0] = Emin;
  out[1] = Emax;
  out[2] = rho_t / (0.5 * (e_hi - e_lo)) * width / (double)plan.geo.dim;
  return POLFED_OK;
}

}  // extern "C"
