// Internal declarations of the POLFED GB300 library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/polfed.h"

namespace polfed {

// ----------------------------------------------------------------- errors
struct Error {
  int code;
  std::string msg;
};
void set_error(int code, const std::string& msg);
int fail(int code, const std::string& msg);  // set_error + return code
void clear_error();                          // an entry point starts with an empty message

#define PF_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return ::polfed::fail(POLFED_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define PF_CHECK(call)          \
  do {                          \
    int rc_ = (call);           \
    if (rc_ != POLFED_OK) return rc_; \
  } while (0)

// ------------------------------------------------------------- counters
// Process-wide counters of kernel launches and of the step kernel's device
// time (CUDA events on the launching stream); calls report their deltas.
struct Counters {
  int64_t launches = 0;
  // step-kernel launches inside CUDA-event-timed runs (see StepTimer), in all
  // and by storage kind (index POLFED_F64 / POLFED_F32 / POLFED_DF64)
  int64_t step_launches = 0;
  double step_gpu_s = 0.0;
  double step_alg_bytes = 0.0;
  int64_t kind_launches[3] = {0, 0, 0};
  double kind_gpu_s[3] = {0.0, 0.0, 0.0};
  double kind_alg_bytes[3] = {0.0, 0.0, 0.0};
  // every step-kernel launch, timed or not (the timer reads its share from these)
  int64_t all_launches[3] = {0, 0, 0};
  double all_alg_bytes[3] = {0.0, 0.0, 0.0};
};
Counters& counters();
inline void count_launch(int64_t n = 1) { counters().launches += n; }
// count one step-kernel launch of storage kind `kind` moving `alg_bytes` algorithmic bytes
inline void count_step(int kind, double alg_bytes) {
  Counters& c = counters();
  c.launches++;
  c.all_launches[kind]++;
  c.all_alg_bytes[kind] += alg_bytes;
}

// -------------------------------------------------------------- binomials
// C(n, k) for 0 <= n, k <= 32 (C(32,16) < 2^31).
uint32_t binom_host(int n, int k);
void upload_binomials();  // __constant__ table, once per device

// ------------------------------------------------- Hamiltonian operator plan
// A term of Eq. (1) between sites i < j with coupling class l (1: J1, 2: J2).
struct Bond {
  int i, j, cls;
};

constexpr int kMaxBonds = 64;
constexpr int kMaxCross = 16;

// Split of the L bits into a low part (bits 0..b-1) and a high part (bits
// b..L-1).  Rows whose states share the high part s_hi form one contiguous
// "group"; rank(s) = T_hi[s_hi] + T_lo[s_lo] (combinatorial number system).
struct HamGeometry {
  int L, b, nh, n_up, periodic;
  int64_t dim;
  double J1, J2, Delta;
  double h[32];
  // literal terms of Eq. (1), classified by where their two sites lie
  int n_low1, n_low2;    // low bonds, class 1 first then class 2
  uint32_t low_mask[kMaxBonds];
  int n_high1, n_high2;  // high bonds (masks relative to bit b)
  uint32_t high_mask[kMaxBonds];
  int n_cross;           // one site in each part
  int cross_lo[kMaxCross], cross_hi[kMaxCross], cross_cls[kMaxCross];
  int cls_off[34];       // offset of popcount class c in the U_lo table
  int max_group;         // largest group (rows)
  int n_groups;          // valid groups
  int rec_stride;        // uint16 entries per neighbour record (16 or 32)
};

// Device tables of a geometry (owned by HamPlan).
struct HamTables {
  uint16_t* T_lo;   // [2^b] rank of s_lo among b-bit strings of equal popcount
  uint16_t* U_lo;   // [2^b] inverse: U_lo[cls_off[c] + k] = k-th b-bit string with popcount c
  int32_t* T_hi;    // [2^nh] first row of group s_hi, -1 if the group is empty
  int32_t* order;   // [n_groups] groups, largest first
  double* F_lo;     // [2^b] diagonal part from low bonds and low fields (H units)
  double* F_hi;     // [2^nh] diagonal part from high bonds and high fields
  double* C_x;      // [2^n_cross] diagonal part from cross bonds by "differ" pattern
  // [2^b * rec_stride] per-row neighbour record, indexed by cls_off[c] + local index:
  //   entry 0: s_lo; entry 1: n1 | n2 << 8 (active low bonds of class 1 and 2);
  //   entries 2..: local indices of the active low-bond neighbours, class 1 first;
  //   last entries (from the end): local index, in the neighbouring popcount
  //   class, of s_lo with the low site of cross bond k flipped
  uint16_t* rec;
  // [2^b * rec_stride] bytes: the same records with one-byte entries (local
  // indices are < 256), for the shared-memory copy of the bulk-copy kernel:
  //   bytes 0-1: s_lo; byte 2: n1; byte 3: n2; bytes 4..: active low-bond
  //   neighbours (class 1 first); last bytes (from the end): cross neighbours
  uint8_t* rec8;
  // [n_groups] per-group constants in schedule order (see GroupRec)
  struct GroupRec* grec;
};

constexpr int kMaxHigh = 32;  // high bonds: L = 24 J1-J2 with b = 10 has 13 + 12 = 25
// Per-group constants (one group = rows sharing s_hi), precomputed per plan.
struct alignas(16) GroupRec {
  int r0, n_g, cls_base, n_hn1, n_hn, need_mask, pad0, pad1;
  int hn_base[kMaxHigh];  // first row of each neighbouring group through an antiparallel high bond
  int cr_base[8];         // first row of the group reached through cross bond k
  int cr_n[8];            // rows of that group (0 if no row of this group has the bond antiparallel)
};

int build_geometry(const polfed_model* m, int b_override, HamGeometry* g);

// A captured run of Clenshaw step launches (see filter_block).
struct StepGraph {
  int kind = 0, K = 0, lpr = 0;
  double invD = 0.0, lo = 0.0, hi = 0.0;
  uint64_t coef_hash = 0;
  uint32_t wait_cap = 0;
  const void *xs = nullptr, *ba = nullptr, *bb = nullptr;
  cudaGraphExec_t exec = nullptr;  // null: key seen once, not captured yet
  int64_t launches = 0;             // step launches of one replay
  double alg_bytes = 0.0;           // their algorithmic bytes
  int uses = 0;
};

class HamPlan {
 public:
  HamGeometry geo;
  HamTables tab{};
  void* dev = nullptr;       // one allocation for all tables
  int* err_flag = nullptr;   // set by a kernel whose bounded wait expired
  // per-precision alpha/beta-scaled tables (F_lo, F_hi, C_x), indexed by dtype
  void* typed[3] = {nullptr, nullptr, nullptr};
  size_t typed_bytes[3] = {0, 0, 0};
  bool typed_ok[3] = {false, false, false};
  double typed_lo[3] = {0, 0, 0}, typed_hi[3] = {0, 0, 0};
  cudaStream_t stream = nullptr;
  bool stream_alloc = false;  // tables from cudaMallocAsync
  std::vector<StepGraph> graphs;  // captured Clenshaw runs on this plan's tables (destroyed with it)

  int init(const polfed_model* m, cudaStream_t s, bool stream_ordered, int b_override = -1);
  int prepare_typed(int kind, double e_lo, double e_hi);  // alpha/beta-scaled tables
  void release();
  ~HamPlan() { release(); }
};

// Arguments of one H~-slice kernel launch: out = cX*X + cH*(H~ b1) + cB*b2, all
// operands slice-major (ld = W elements, W = VEC * LPR).
struct StepArgs {
  const void* b1;
  const void* b2;  // may be null when cB == 0
  const void* x;   // may be null when cX == 0
  void* out;
  double cX, cH, cB;
  int lpr;         // lanes per row: slice = 16 * lpr bytes
  const float* cxcol = nullptr;  // F32 only: per-column cX (device, W floats) in place of cX
};

// Launch one step (kind = POLFED_F32 / F64 / DF64 storage type).
int launch_ham_step(const HamPlan& plan, int kind, const StepArgs& a, cudaStream_t s);

// Elements per slice for a precision and lanes-per-row.
int slice_width(int kind, int lpr);
size_t elem_bytes(int kind);  // internal storage element size (DF64: 8 = two floats)

// Filter engine over an arbitrary-width ABI block.  in/out are row-major
// dim x n_b of "abi_kind" (POLFED_F32: float, else double).
struct FilterScratch {
  void* xs = nullptr;  // slice buffers (dim x W each)
  void* ba = nullptr;
  void* bb = nullptr;
  float* flag = nullptr;  // [4] max |x|, max |y| (as float bits)
  size_t bytes = 0;
};
int filter_block(HamPlan& plan, int kind, const double* coeffs, int K, double invD, const void* in, void* out,
                 int n_b, int abi_kind, FilterScratch& scr, cudaStream_t s, int lpr_hint = 0);
// FP32 filter with its own coefficients per column: out[:, j] = sum_n coef_j[n] T_n(H~) in[:, j].
// The block is filtered in slices of W = slice_width(POLFED_F32, choose_lpr(POLFED_F32, n_b)) columns;
// d_coef (device) holds, per slice q, (K + 1) rows of W floats:
// d_coef[(q (K + 1) + n) W + j - q W] = coefficient of column j at order n.  in/out as filter_block.
int filter_block_cols(HamPlan& plan, const float* d_coef, int K, const void* in, void* out, int n_b, int abi_kind,
                      FilterScratch& scr, cudaStream_t s);
int apply_block(HamPlan& plan, int kind, const void* in, void* out, int n_b, int abi_kind, FilterScratch& scr,
                cudaStream_t s, int lpr_hint = 0);
size_t filter_scratch_bytes(const HamPlan& plan, int kind, int lpr);
int choose_lpr(int kind, int n_b);

// Batched filter: one cooperative launch runs the Clenshaw recurrences of
// many (realization, 128-byte column slice) jobs, each with its own plan,
// order and coefficients (F32 or DF64 storage; all jobs J2 == 0 or all not).
struct BatchFilterItem {
  HamPlan* plan;          // prepare_typed(kind, ...) done
  const double* coef;     // host, K + 1 coefficients: Y = invD * sum_n coef[n] T_n(H~) X
  int K;
  double invD;
  const void* in;         // device, row-major dim x n_b (abi kind)
  void* out;              // device, row-major dim x n_b
  int n_b;
  bool bounds_error;      // out: output grew beyond the Chebyshev bound
};
struct BatchStats {
  int n_jobs = 0, n_steps = 0, grid = 0;
  double gpu_s = 0.0, alg_bytes = 0.0;
};
size_t batch_scratch_bytes(const std::vector<BatchFilterItem>& items, int kind);
int filter_batched(std::vector<BatchFilterItem>& items, int kind, int abi_kind, void* scratch, size_t bytes,
                   cudaStream_t s, int ctas_per_sm, BatchStats* st);

// Filter calls of the block-Lanczos driver can be routed through a hook (the
// batched runner's rendezvous).  Panels q = 0..npan-1: out[q] = invD sum_n
// coef[n] T_n(H~) in[q], each dim x S row-major FP64 on `s`.
struct FilterHook {
  virtual int filter(HamPlan& plan, int kind, const double* coef, int K, double invD, const double* const* in,
                     double* const* out, int npan, int S, cudaStream_t s) = 0;
  virtual int plan_b(int L) { return -1; }  // low/high split for the plans (-1 = default)
  // the caller launches its own kernels until resume() and sends no filter() meanwhile
  virtual void suspend() {}
  virtual void resume() {}
  virtual ~FilterHook() {}
};
// Context internals for the other translation units.
cudaStream_t ctx_stream(polfed_ctx* c);
void* ctx_solver(polfed_ctx* c);  // cusolverDnHandle_t
int ctx_device(polfed_ctx* c);

// polfed_eigs with an optional hook (nullptr = direct filter launches).
int eigs_impl(polfed_ctx* c, const polfed_model* model, double eps_target, int32_t N_ev, int32_t K, int32_t n_b,
              const polfed_opts* opts, double* evals, double* d_evecs, double* resid, polfed_stats* stats,
              FilterHook* hook);

// Chebyshev coefficients of Eq. (2) in FP64: c_n, n = 0..K, and D.
void cheb_coeffs(double sigma, int K, std::vector<double>& c, double& D);

// Kernel polynomial method: stochastic Chebyshev moments of H~ and the
// Jackson-damped fraction of the spectrum inside an interval.
constexpr int kMaxKpmMoments = 65536;
struct KpmBuffers {
  void* t0;
  void* t1;
  void* y;       // three dim x R blocks of the ABI element type
  double* part;  // per-block partial sums
  double* mu;    // raw moment pairs
};
void jackson_coeffs(int N, std::vector<double>& g);
size_t kpm_buffer_bytes(int64_t dim, int R, int abi_kind);
KpmBuffers kpm_carve(void* base, int64_t dim, int R, int abi_kind);
// mu[n] = (1/R) sum_r r^T T_n(H~) r, n < n_mom (host out); r is row-major dim x R
// of float (kind POLFED_F32) or double.  Needs plan.prepare_typed(kind, ...).
int kpm_moments(HamPlan& plan, int kind, const void* r, int R, int n_mom, double* mu, const KpmBuffers& b,
                FilterScratch& scr, cudaStream_t s);
double kpm_count_fraction(const double* mu, int n_mom, double x_a, double x_b);

// Basis kernel (polfed_basis_build).
int launch_basis(int L, int n_up, uint32_t* d_states, int64_t dim, cudaStream_t s);

}  // namespace polfed
