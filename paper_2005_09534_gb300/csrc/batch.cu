// Batched runner: many disorder realizations solved together on one GPU.
//
// The paper runs realizations independently (one per node or core set).  On
// one GB300 a single small realization (L = 16 or 18: 12870 or 48620 rows)
// fills a fraction of the 152 SMs and pays a kernel launch per Chebyshev
// step.  Here every realization runs the polfed_eigs driver on its own host
// thread, context and stream, and their filter calls meet at a rendezvous:
// once every running realization has asked for its filter, one cooperative
// launch (filter_batched) advances all of their Clenshaw recurrences, each
// with its own operator, order K and block.  Everything else (bounds, block
// Gram-Schmidt, Cholesky QR, the projected eigenproblem, Rayleigh-Ritz) runs
// concurrently on the realizations' own streams.
//
// Autotuner: before the run, the batched filter kernel is timed on the
// realizations' own operators for each candidate block width (16, 32, 64
// columns) and grid (1 or 2 CTAs per SM); each realization then takes the
// width that minimizes (measured time per filter step of width S) x (steps
// its Lanczos run needs, about max(16, ceil(2.64 N_ev / S) + 8)).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "polfed_internal.h"

namespace polfed {
namespace {

double wall_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// low/high split of the batched plans: large groups keep the per-CTA work
// items big when many small realizations share the GPU
int batch_b(int L) { return std::max(2, std::min(10, L - 4)); }

struct DeviceBuffer {
  void* p = nullptr;
  size_t n = 0;
  int ensure(size_t need) {
    if (need <= n) return POLFED_OK;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    if (cudaMalloc(&p, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(POLFED_ENOMEM, "batched runner: cudaMalloc of " + std::to_string(need) + " bytes failed");
    }
    n = need;
    return POLFED_OK;
  }
  ~DeviceBuffer() {
    if (p) cudaFree(p);
  }
};

// Rendezvous of the realizations' filter calls (see the file comment).
class Rendezvous : public FilterHook {
 public:
  explicit Rendezvous(int ctas_per_sm) : ctas_(ctas_per_sm) {}
  int init() {
    if (cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking) != cudaSuccess)
      return fail(POLFED_ECUDA, "batched runner: cudaStreamCreate failed");
    return POLFED_OK;
  }
  ~Rendezvous() override {
    if (stream_) {
      cudaStreamSynchronize(stream_);
      cudaStreamDestroy(stream_);
    }
  }
  int plan_b(int L) override { return batch_b(L); }
  // a realization in its refinement sweeps launches on its own stream: the others' filters need not wait for it
  void suspend() override { leave(); }
  void resume() override { enter(); }

  void enter() {
    std::unique_lock<std::mutex> lk(mu_);
    active_++;
  }
  void leave() {
    std::unique_lock<std::mutex> lk(mu_);
    active_--;
    drain(lk);
  }

  int filter(HamPlan& plan, int kind, const double* coef, int K, double invD, const double* const* in,
             double* const* out, int npan, int S, cudaStream_t s) override {
    Req r;
    r.plan = &plan;
    r.kind = kind;
    r.coef = coef;
    r.K = K;
    r.invD = invD;
    r.in.assign(in, in + npan);
    r.out.assign(out, out + npan);
    r.S = S;
    if (cudaEventCreateWithFlags(&r.ready, cudaEventDisableTiming) != cudaSuccess)
      return fail(POLFED_ECUDA, "cudaEventCreate failed");
    cudaEventRecord(r.ready, s);
    std::unique_lock<std::mutex> lk(mu_);
    pending_.push_back(&r);
    drain(lk);
    cv_.wait(lk, [&] { return r.done; });
    lk.unlock();
    cudaEventDestroy(r.ready);
    if (r.rc != POLFED_OK) set_error(r.rc, r.msg);
    return r.rc;
  }

  int rounds() const { return rounds_; }
  double gpu_s() const { return gpu_s_; }
  double alg_bytes() const { return alg_; }
  int64_t launches() const { return launches_; }

 private:
  struct Req {
    HamPlan* plan = nullptr;
    int kind = 0;
    const double* coef = nullptr;
    int K = 0;
    double invD = 1.0;
    std::vector<const double*> in;
    std::vector<double*> out;
    int S = 0;
    cudaEvent_t ready = nullptr;
    int rc = POLFED_OK;
    std::string msg;
    bool done = false;
  };

  // Launch while every running realization is waiting for its filter.
  void drain(std::unique_lock<std::mutex>& lk) {
    while (!launching_ && !pending_.empty() && (int)pending_.size() >= active_) {
      launching_ = true;
      std::vector<Req*> batch;
      batch.swap(pending_);
      lk.unlock();
      run(batch);
      lk.lock();
      launching_ = false;
      for (Req* r : batch) r->done = true;
      cv_.notify_all();
    }
  }

  void run(std::vector<Req*>& batch) {
    // one launch per (storage kind, J2 != 0) class
    for (int kind : {POLFED_F32, POLFED_DF64})
      for (int j2 = 0; j2 < 2; j2++) {
        std::vector<Req*> grp;
        std::vector<BatchFilterItem> items;
        for (Req* r : batch)
          if (r->kind == kind && ((r->plan->geo.J2 != 0.0) == (j2 == 1))) {
            grp.push_back(r);
            cudaStreamWaitEvent(stream_, r->ready, 0);
            for (size_t q = 0; q < r->in.size(); q++)
              items.push_back(BatchFilterItem{r->plan, r->coef, r->K, r->invD, r->in[q], r->out[q], r->S, false});
          }
        if (grp.empty()) continue;
        const Counters c0 = counters();
        int rc = buf_.ensure(batch_scratch_bytes(items, kind));
        BatchStats bs;
        if (rc == POLFED_OK) rc = filter_batched(items, kind, POLFED_F64, buf_.p, buf_.n, stream_, ctas_, &bs);
        const Counters c1 = counters();
        launches_ += c1.launches - c0.launches;
        rounds_++;
        gpu_s_ += bs.gpu_s;
        alg_ += bs.alg_bytes;
        size_t k = 0;
        for (Req* r : grp) {
          r->rc = rc;
          if (rc != POLFED_OK) r->msg = polfed_last_error();
          for (size_t q = 0; q < r->in.size(); q++, k++)
            if (rc == POLFED_OK && items[k].bounds_error) {
              r->rc = POLFED_EBOUNDS;
              r->msg = "filter output grew beyond the Chebyshev bound: spectrum outside [e_lo, e_hi]";
            }
        }
      }
  }

  std::mutex mu_;
  std::condition_variable cv_;
  std::vector<Req*> pending_;
  int active_ = 0;
  bool launching_ = false;
  int ctas_ = 0;
  cudaStream_t stream_ = nullptr;
  DeviceBuffer buf_;
  int rounds_ = 0;
  double gpu_s_ = 0.0, alg_ = 0.0;
  int64_t launches_ = 0;
};

// Rigorous bound on ||H||: each bond term has norm <= |J| (1/2 + |Delta|/4), each field term |h_i| / 2.
double norm_bound(const polfed_model& m) {
  const double nb1 = m.periodic ? m.L : m.L - 1, nb2 = m.periodic ? m.L : m.L - 2;
  double b = (nb1 * std::fabs(m.J1) + nb2 * std::fabs(m.J2)) * (0.5 + std::fabs(m.Delta) / 4.0);
  for (int i = 0; i < m.L; i++) b += 0.5 * std::fabs(m.h[i]);
  return b;
}

__global__ void k_fill_pattern(double* x, int64_t n, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
}

struct TuneResult {
  std::vector<int> S;  // per realization
  int ctas = 0;
  double seconds = 0.0;
  double t_slice[3][2] = {{0}};  // measured seconds per filter step, [S index][ctas - 1]
};

// Time the batched filter on the realizations' operators (16 steps) for each
// block width and grid, then pick per-realization widths (file comment).
int autotune(const std::vector<polfed_model>& models, const std::vector<int>& N_ev, int kind, const polfed_opts& o,
             TuneResult& tr) {
  const double t0 = wall_s();
  const int n = (int)models.size();
  const int nt = std::min(n, 16);  // a representative subset bounds the tuning cost
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
    return fail(POLFED_ECUDA, "cudaStreamCreate failed");
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  } sg{s};
  std::vector<HamPlan> plans(nt);
  size_t vec_bytes = 0;
  for (int i = 0; i < nt; i++) {
    PF_CHECK(plans[i].init(&models[i], s, false, batch_b(models[i].L)));
    const double b = norm_bound(models[i]);
    PF_CHECK(plans[i].prepare_typed(kind, -b, b));
    vec_bytes += (size_t)plans[i].geo.dim * 64 * sizeof(double);
  }
  DeviceBuffer X, Y, scr;
  PF_CHECK(X.ensure(vec_bytes));
  PF_CHECK(Y.ensure(vec_bytes));
  k_fill_pattern<<<152 * 8, 256, 0, s>>>((double*)X.p, (int64_t)(vec_bytes / 8), o.seed);
  count_launch();
  const int Kt = 16;
  std::vector<double> coef(Kt + 1);
  for (int k = 0; k <= Kt; k++) coef[k] = (k % 2 == 0) ? ((k / 2) % 2 ? -2.0 : 2.0) : 0.0;
  coef[0] = 1.0;
  const int widths[3] = {16, 32, 64};
  double best_t32 = 1e300;
  for (int wi = 0; wi < 3; wi++)
    for (int ctas = 1; ctas <= 2; ctas++) {
      std::vector<BatchFilterItem> items;
      size_t off = 0;
      for (int i = 0; i < nt; i++) {
        items.push_back(BatchFilterItem{&plans[i], coef.data(), Kt, 1.0 / Kt, (char*)X.p + off, (char*)Y.p + off,
                                        widths[wi], false});
        off += (size_t)plans[i].geo.dim * 64 * sizeof(double);
      }
      PF_CHECK(scr.ensure(batch_scratch_bytes(items, kind)));
      BatchStats bs;
      PF_CHECK(filter_batched(items, kind, POLFED_F64, scr.p, scr.n, s, ctas, &bs));  // warm-up
      PF_CHECK(filter_batched(items, kind, POLFED_F64, scr.p, scr.n, s, ctas, &bs));
      tr.t_slice[wi][ctas - 1] = bs.gpu_s / Kt;
      if (wi == 1 && bs.gpu_s < best_t32) {
        best_t32 = bs.gpu_s;
        tr.ctas = ctas;
      }
    }
  // per-realization width: time per step is shared by the subset; the cost of
  // a width for realization i scales with its share of rows
  double rows = 0.0;
  for (int i = 0; i < nt; i++) rows += (double)plans[i].geo.dim;
  tr.S.assign(n, 32);
  for (int i = 0; i < n; i++) {
    const double dim = (double)binom_host(models[i].L, models[i].L / 2);
    double best = 1e300;
    for (int wi = 0; wi < 3; wi++) {
      const int S = widths[wi];
      // steps to convergence: onset at ms ~ 2.2 (1 + k_margin) N_ev, then about 8 more
      const int m = std::max(16, (int)std::ceil(2.2 * (1.0 + o.k_margin) * N_ev[i] / S) + 8);
      const double per_step = tr.t_slice[wi][tr.ctas - 1] * dim / rows;
      const double cost = per_step * m;
      if (cost < best) {
        best = cost;
        tr.S[i] = S;
      }
    }
  }
  tr.seconds = wall_s() - t0;
  return POLFED_OK;
}

}  // namespace
}  // namespace polfed

using namespace polfed;

extern "C" {

int polfed_cheb_filter_batched(int32_t n_inst, const polfed_model* models, const double* e_lo, const double* e_hi,
                               const double* sigma, const int32_t* K, const void* const* d_X, void* const* d_Y,
                               int32_t n_b, int32_t dtype, int32_t ctas_per_sm, polfed_stream_t stream) {
  if (n_inst < 1 || !models || !e_lo || !e_hi || !sigma || !K || !d_X || !d_Y)
    return fail(POLFED_EINVAL, "NULL argument or n_inst < 1");
  if (dtype != POLFED_F32 && dtype != POLFED_DF64) return fail(POLFED_EINVAL, "batched filter: dtype F32 or DF64");
  if (n_b < 1 || n_b > 128) return fail(POLFED_EINVAL, "n_b must be in 1..128");
  if (ctas_per_sm < 0 || ctas_per_sm > 2) return fail(POLFED_EINVAL, "ctas_per_sm must be 0, 1 or 2");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<HamPlan> plans(n_inst);
  std::vector<std::vector<double>> coefs(n_inst);
  std::vector<BatchFilterItem> items;
  const bool j2 = models[0].J2 != 0.0;
  for (int i = 0; i < n_inst; i++) {
    if ((models[i].J2 != 0.0) != j2) return fail(POLFED_EINVAL, "all realizations must agree on J2 = 0 or not");
    if (!(e_lo[i] < e_hi[i])) return fail(POLFED_EINVAL, "need e_lo < e_hi");
    if (!(sigma[i] > -1.0 && sigma[i] < 1.0)) return fail(POLFED_EINVAL, "sigma must be in (-1, 1)");
    if (K[i] < 0 || K[i] > 10000000) return fail(POLFED_EINVAL, "K must be in 0..1e7");
    if (!d_X[i] || !d_Y[i] || d_X[i] == d_Y[i]) return fail(POLFED_EINVAL, "bad X / Y pointers");
    PF_CHECK(plans[i].init(&models[i], s, true, batch_b(models[i].L)));
    PF_CHECK(plans[i].prepare_typed(dtype, e_lo[i], e_hi[i]));
    double D = 1.0;
    cheb_coeffs(sigma[i], K[i], coefs[i], D);
    items.push_back(BatchFilterItem{&plans[i], coefs[i].data(), K[i], 1.0 / D, d_X[i], d_Y[i], n_b, false});
  }
  const int abi = dtype == POLFED_F32 ? POLFED_F32 : POLFED_F64;
  void* scr = nullptr;
  const size_t bytes = batch_scratch_bytes(items, dtype);
  PF_CUDA(cudaMallocAsync(&scr, bytes, s));
  BatchStats bs;
  int rc = filter_batched(items, dtype, abi, scr, bytes, s, ctas_per_sm, &bs);
  cudaFreeAsync(scr, s);
  cudaStreamSynchronize(s);
  if (rc != POLFED_OK) return rc;
  for (const auto& it : items)
    if (it.bounds_error)
      return fail(POLFED_EBOUNDS, "filter output grew beyond the Chebyshev bound: spectrum outside [e_lo, e_hi]");
  return POLFED_OK;
}

int polfed_eigs_batched(int32_t device, int32_t n_inst, const polfed_model* models, const double* eps_target,
                        const int32_t* N_ev, const int32_t* K, int32_t n_b, const polfed_opts* opts,
                        int32_t max_workers, double* evals, double* resid, double* const* d_evecs,
                        polfed_stats* stats, int32_t* status, polfed_batch_info* info) {
  if (n_inst < 1 || !models || !eps_target || !N_ev || !evals || !status)
    return fail(POLFED_EINVAL, "NULL argument or n_inst < 1");
  if (n_b != 0 && (n_b < 1 || n_b > 128)) return fail(POLFED_EINVAL, "n_b must be 0 (autotune) or in 1..128");
  polfed_opts o;
  if (opts)
    o = *opts;
  else
    polfed_opts_default(&o);
  if (o.precision != POLFED_F32 && o.precision != POLFED_DF64)
    return fail(POLFED_EINVAL, "batched runner: precision POLFED_F32 or POLFED_DF64");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return fail(POLFED_EINVAL, "invalid CUDA device");
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  const double t0 = wall_s();
  std::vector<polfed_model> ms(models, models + n_inst);
  std::vector<int> nev(N_ev, N_ev + n_inst);
  std::vector<int64_t> off(n_inst + 1, 0);
  for (int i = 0; i < n_inst; i++) {
    if (nev[i] < 1) return fail(POLFED_EINVAL, "N_ev must be >= 1");
    off[i + 1] = off[i] + nev[i];
    status[i] = POLFED_ECUDA;  // until a worker has run the realization
  }
  // 1. autotuning of the block widths and the grid
  TuneResult tr;
  if (n_b == 0) {
    PF_CHECK(autotune(ms, nev, o.precision, o, tr));
  } else {
    tr.S.assign(n_inst, n_b);
    tr.ctas = 0;
  }
  // 2. workers
  Rendezvous rv(tr.ctas);
  PF_CHECK(rv.init());
  const int nw = std::max(1, std::min<int>(n_inst, max_workers > 0 ? max_workers : 64));
  std::atomic<int> next{0};
  std::vector<int> wrc(nw, POLFED_OK);
  std::vector<std::string> wmsg(nw);
  std::vector<int64_t> wlaunch(nw, 0);
  auto worker = [&](int w) {
    cudaSetDevice(device);
    polfed_ctx* ctx = nullptr;
    int rc = polfed_ctx_create(device, 0, &ctx);
    if (rc != POLFED_OK) {
      wrc[w] = rc;
      wmsg[w] = polfed_last_error();
      return;
    }
    const Counters c0 = counters();
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= n_inst) break;
      polfed_stats st;
      memset(&st, 0, sizeof(st));
      rv.enter();
      const int r = eigs_impl(ctx, &ms[i], eps_target[i], nev[i], K ? K[i] : 0, tr.S[i], &o, evals + off[i],
                              d_evecs ? d_evecs[i] : nullptr, resid ? resid + off[i] : nullptr, &st, &rv);
      rv.leave();
      status[i] = r;
      if (r != POLFED_OK && wrc[w] == POLFED_OK) {
        wrc[w] = r;
        wmsg[w] = polfed_last_error();
      }
      if (stats) stats[i] = st;
    }
    wlaunch[w] = counters().launches - c0.launches;
    polfed_ctx_destroy(ctx);
  };
  std::vector<std::thread> th;
  for (int w = 0; w < nw; w++) th.emplace_back(worker, w);
  for (auto& t : th) t.join();
  int rc = POLFED_OK;
  std::string msg;
  for (int w = 0; w < nw; w++)
    if (wrc[w] != POLFED_OK && rc == POLFED_OK) {
      rc = wrc[w];
      msg = wmsg[w];
    }
  if (info) {
    memset(info, 0, sizeof(*info));
    info->n_b = tr.S.empty() ? n_b : tr.S[0];
    info->ctas_per_sm = tr.ctas;
    info->rounds = rv.rounds();
    info->workers = nw;
    info->t_total = wall_s() - t0;
    info->t_tune = tr.seconds;
    info->filter_gpu_s = rv.gpu_s();
    info->filter_alg_bytes = rv.alg_bytes();
    int64_t nl = 0;
    for (int64_t v : wlaunch) nl += v;
    info->n_launches = nl;
    for (int wi = 0; wi < 3; wi++)
      for (int c = 0; c < 2; c++) info->tune_step_s[wi][c] = tr.t_slice[wi][c];
    for (int i = 0; i < n_inst; i++) {
      const int S = tr.S[i];
      if (S == 16) info->n_width16++;
      else if (S == 32) info->n_width32++;
      else info->n_width64++;
    }
  }
  if (rc != POLFED_OK) return fail(rc, "batched runner: " + msg);
  return POLFED_OK;
}

}  // extern "C"
