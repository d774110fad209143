/*
 * polfed.h -- C ABI of the GB300 POLFED hot path.
 *
 * POLFED (Sierant, Lewenstein, Zakrzewski, arXiv:2005.09534) finds the
 * eigenpairs of the disordered spin-1/2 chain of Eq. (1) whose energies are
 * nearest a target, by block Lanczos (Eqs. (3)-(4)) on the polynomial
 * spectral transform P^K_sigma(H~) of Eq. (2), with full
 * re-orthogonalization and Rayleigh quotients of the Ritz vectors.
 *
 * Conventions shared by every call:
 *   - Site i (0-based) of the chain is bit i of a basis state; bit = 1 is
 *     spin up (S^z = +1/2).  The S^z = 0 sector has L/2 up spins and
 *     dimension N = C(L, L/2).  States are listed in ascending integer order
 *     and a vector's row r belongs to the r-th state.
 *   - A "block" of n_b vectors is row-major N x n_b: the n_b values of one
 *     basis state are contiguous.  Device pointers are plain CUDA device
 *     addresses (any allocator); the caller owns every buffer it passes.
 *   - Energies (e_lo, e_hi, eigenvalues, residuals) are in units of J1 = 1
 *     unless stated otherwise.  The rescaled operator is
 *     H~ = [2H - (e_lo + e_hi)] / (e_hi - e_lo) (text before Eq. (3)).
 *   - Every call returns POLFED_OK (0) or a negative status; the thread-local
 *     message of the last failure is returned by polfed_last_error().  No
 *     C++ exception crosses this boundary.  Calls that take a stream enqueue
 *     their kernels on it; they may return before the GPU work completes
 *     unless stated otherwise.
 */
#ifndef POLFED_H
#define POLFED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* polfed_stream_t; /* same type as cudaStream_t; NULL = legacy default stream */

enum {
  POLFED_OK = 0,
  POLFED_EINVAL = -1,   /* invalid argument (odd L, L > 32, n_b out of range, e_lo >= e_hi, ...) */
  POLFED_ENOMEM = -2,   /* device or host allocation failed */
  POLFED_ECUDA = -3,    /* a CUDA or cuSOLVER call failed */
  POLFED_EBOUNDS = -4,  /* the spectrum is not inside [e_lo, e_hi]: the Chebyshev recurrence grew */
  POLFED_ENOCONV = -5,  /* block Lanczos hit its step limit; partial results and n_conv are set */
  POLFED_ETIMEOUT = -6  /* a bounded device-side wait expired */
};

enum {
  POLFED_F64 = 0,  /* FP64 storage and FP64 arithmetic */
  POLFED_F32 = 1,  /* FP32 storage and FP32 arithmetic */
  POLFED_DF64 = 2  /* FP64 input/output, internal float-float (two FP32) storage and arithmetic */
};

/* Parameters of Eq. (1):
 *   H = sum_{l=1,2} sum_{i=1..L} J_l (S^x_i S^x_{i+l} + S^y_i S^y_{i+l} + Delta S^z_i S^z_{i+l})
 *       + sum_i h_i S^z_i.
 * periodic = 1 wraps i + l modulo L (the paper's boundary condition); 0 drops
 * the wrapping terms (open chain, used by tests).  h is a HOST array of L
 * doubles (h[i] is the field on site i), read during the call only. */
typedef struct polfed_model {
  int32_t L;
  int32_t periodic;
  double J1, J2, Delta;
  const double* h;
} polfed_model;

/* Options of polfed_eigs.  polfed_opts_default() fills every field. */
typedef struct polfed_opts {
  double p;              /* accessible-eigenvalue threshold of the transform, paper: 0.17 */
  double k_margin;       /* choose K so that about (1 + k_margin) N_ev eigenvalues have P >= p */
  double tol_conv;       /* block-Lanczos convergence: ||B_{j+1} t~_i|| <= tol_conv (units of P) */
  double tol_resid;      /* acceptance: ||H u - E u|| <= tol_resid * ||H||, ||H|| = max(|E_min|, |E_max|) */
  double cols_factor;    /* Lanczos column budget = cols_factor * (1 + k_margin) * N_ev (paper: 2.8) */
  int32_t precision;     /* filter arithmetic: POLFED_F64, POLFED_DF64, or POLFED_F32 for the Lanczos stage
                            followed by float-float refinement sweeps (Jackson-damped filter + Rayleigh-Ritz) */
  int32_t bounds_steps;  /* max single-vector Lanczos steps for E_min / E_max */
  int32_t verbose;       /* 1 = progress lines on stderr */
  int32_t reserved;
  uint64_t seed;         /* seed of the random starting block Q_1 */
} polfed_opts;

/* Counters and timers of one polfed_eigs / polfed_block_lanczos call. */
typedef struct polfed_stats {
  int32_t K;             /* filter order used */
  int32_t m;             /* block Lanczos steps taken */
  int32_t n_b;           /* block size s */
  int32_t n_conv;        /* converged Ritz pairs with theta >= p */
  int32_t n_ritz_checks; /* eigen-solves of T_j */
  int32_t status;        /* final status */
  int32_t n_refine;      /* refinement sweeps (POLFED_F32 precision) */
  int32_t refine_K;      /* order of the last refinement filter */
  int64_t dim;           /* N */
  int64_t matvec_cols;   /* column matrix-vector products with H~ (filter + bounds + checks) */
  double E_min, E_max;   /* spectral bounds (Lanczos) */
  double e_lo, e_hi;     /* padded rescaling interval */
  double sigma;          /* target in H~ units */
  double target;         /* target energy E* in H units */
  double rho_sigma;      /* density of states per unit of H~ used to set K */
  double max_resid;      /* max ||H u - E u|| over the returned pairs (H units) */
  double t_bounds, t_filter, t_reorth, t_qr, t_teig, t_ritz, t_total; /* seconds */
  int64_t n_launches;      /* kernels this library launched during the call */
  int64_t n_step_launches; /* launches of the Chebyshev / H~ step kernel */
  double step_gpu_s;       /* device time of those launches (CUDA events on the launching stream) */
  double step_alg_bytes;   /* algorithmic bytes of those launches: N * cols * w * (3 + [c_k != 0]) each */
} polfed_stats;

typedef struct polfed_ctx polfed_ctx;

/* Default options: p = 0.17, k_margin = 0.2, tol_conv = 1e-7 (tightened until the residuals pass), tol_resid = 1e-8,
 * cols_factor = 2.8, precision = POLFED_DF64, bounds_steps = 600, seed = 1234. */
void polfed_opts_default(polfed_opts* opts);

/* Basis of the S^z sector with n_up up spins ("Benchmark models": N = C(L, L/2)
 * for n_up = L/2).
 *   L        : chain length, 2 <= L <= 32.
 *   n_up     : number of up spins, 0 <= n_up <= L (L/2 for the S^z = 0 sector).
 *   d_states : device array of *dim uint32 receiving the states in ascending
 *              order, or NULL to only query the dimension.
 *   dim      : host out, the sector dimension.
 * Enqueues one kernel on `stream` when d_states != NULL. */
int polfed_basis_build(int32_t L, int32_t n_up, uint32_t* d_states, int64_t* dim, polfed_stream_t stream);

/* Y = H~ X (matrix-free; the text before Eq. (3) and the Supplement's
 * "Technical details").  With e_lo == e_hi == 0 the raw H of Eq. (1) is applied.
 *   model    : Eq. (1) parameters (host struct, host h).
 *   d_states : device basis from polfed_basis_build for n_up = L/2 (used to
 *              check dim; the kernels rank states with integer tables).
 *   dim      : C(L, L/2).
 *   d_X, d_Y : device, row-major dim x n_b, element type by dtype
 *              (POLFED_F32: float; POLFED_F64 / POLFED_DF64: double).  X and Y must not overlap.
 *   n_b      : 1 <= n_b <= 128.
 * Synchronizes the stream before returning (it owns stream-ordered scratch). */
int polfed_h_apply(const polfed_model* model, const uint32_t* d_states, int64_t dim, double e_lo, double e_hi,
                   const void* d_X, void* d_Y, int32_t n_b, int32_t dtype, polfed_stream_t stream);

/* Y = P^K_sigma(H~) X, Eq. (2), by the Clenshaw recurrence (text after
 * Eq. (4)); columns are filtered independently (paper: one core per column;
 * here 128-byte column slices).
 *   sigma  : target in H~ units, -1 < sigma < 1.
 *   K      : order, 0 <= K <= 10^7.
 *   coeffs : NULL for the paper's c_n / D (c_n = sqrt(4 - 3 delta_{0n}) cos(n arccos sigma),
 *            D = sum_n c_n T_n(sigma)); else a HOST array of K + 1 doubles used as
 *            Y = sum_n coeffs[n] T_n(H~) X.
 *   other arguments as in polfed_h_apply.
 * Enqueues about K + 3 kernels per 128-byte column slice; synchronizes the
 * stream before returning (it owns stream-ordered scratch).  Returns
 * POLFED_EBOUNDS if the output is not finite (spectrum outside [e_lo, e_hi]). */
int polfed_cheb_filter(const polfed_model* model, const uint32_t* d_states, int64_t dim, double e_lo, double e_hi,
                       double sigma, int32_t K, const double* coeffs, const void* d_X, void* d_Y, int32_t n_b,
                       int32_t dtype, polfed_stream_t stream);

/* Allocation-free variant of polfed_cheb_filter (the paper has no
 * counterpart; this is a service for callers).  Some callers cannot allocate
 * device memory while they run: code executing inside an allocator or memory
 * pool callback, a host application that owns every device allocation
 * itself, or a latency-critical loop that must never enter the allocator.
 * This call takes the same arguments and computes the same Y as
 * polfed_cheb_filter, but it allocates and frees no device memory (and no
 * host memory on its normal path): its operator tables and Clenshaw buffers
 * are carved out of one fixed 32 MiB device array that every GPU using this
 * library holds from the moment the library's device code is loaded until
 * the process exits.
 *   Limit: the tables plus three dim x 128-byte slice buffers must fit in
 *          32 MiB, i.e. L <= 18 (dim <= 48620) for any n_b; larger problems
 *          return POLFED_ENOMEM with a message naming the bytes needed.
 *   First call on a device: looks up the array's device address
 *          (cudaGetSymbolAddress) with that device current; make this first
 *          call before any stream capture.
 *   Sharing: every call uses the same array and leaves its last contents in
 *          it; each call rewrites everything it reads (tables, recurrence
 *          buffers, flags), so nothing carries over.  Calls that overlap on
 *          the GPU (other streams, other host threads) race on the array and
 *          must be serialized by the caller.
 * Synchronizes the stream before returning. */
int polfed_cheb_filter_static(const polfed_model* model, const uint32_t* d_states, int64_t dim, double e_lo,
                              double e_hi, double sigma, int32_t K, const double* coeffs, const void* d_X, void* d_Y,
                              int32_t n_b, int32_t dtype, polfed_stream_t stream);

/* Context: device, stream, cuSOLVER handle and reusable device workspace.
 *   device          : CUDA device ordinal (the context makes it current in its calls).
 *   workspace_bytes : advisory upper bound for the context's device workspace
 *                     (0 = no limit); exceeding it returns POLFED_ENOMEM.
 *   out             : host out, the new context.  Destroy with polfed_ctx_destroy. */
int polfed_ctx_create(int32_t device, size_t workspace_bytes, polfed_ctx** out);
void polfed_ctx_destroy(polfed_ctx* ctx);
/* Stream used by the context's calls (NULL before any call = its own stream). */
int polfed_ctx_set_stream(polfed_ctx* ctx, polfed_stream_t stream);

/* Block Lanczos on P^K_sigma(H~), Eqs. (3)-(4), with full
 * re-orthogonalization of U_j against Q_1..Q_j, QR by Cholesky QR (twice),
 * convergence by ||B_{j+1} t~_i|| for theta_i >= p, Ritz vectors
 * u_i = Q_m t_i, and eigenvalues u_i^T H~ u_i after a Rayleigh-Ritz step
 * with H~ on the converged Ritz vectors.
 *   e_lo, e_hi : rescaling interval (must contain the spectrum).
 *   sigma, K   : transform target (H~ units) and order.
 *   n_b        : block size s, 1 <= n_b <= 128.
 *   N_ev       : number of eigenpairs requested (nearest sigma).
 *   d_evecs    : device out, dim x N_ev column-major FP64, or NULL.
 *   evals      : host out, N_ev eigenvalues in H units, ascending.
 *   resid      : host out, N_ev residual norms ||H u - E u|| in H units.
 *   n_conv     : host out, number of pairs returned (< N_ev on POLFED_ENOCONV).
 * Uses opts/precision from the last polfed_eigs call on ctx, or defaults.
 * Blocking. */
int polfed_block_lanczos(polfed_ctx* ctx, const polfed_model* model, double e_lo, double e_hi, double sigma,
                         int32_t K, int32_t n_b, int32_t N_ev, double* d_evecs, double* evals, double* resid,
                         int32_t* n_conv);

/* The whole method ("POLFED algorithm" section): spectral bounds by Lanczos,
 * rescaling, K from the density of states and p, block Lanczos, Ritz
 * vectors, Rayleigh quotients and residual check.
 *   eps_target : rescaled target energy in [0, 1]: E* = E_min + eps_target (E_max - E_min)
 *                (0.5 is the middle of the spectrum, sigma = 0).
 *   N_ev       : number of eigenpairs nearest E*.
 *   K          : filter order, 0 = choose from the density of states.
 *   n_b        : block size s.
 *   opts       : options or NULL for defaults.
 *   evals      : host out, N_ev ascending (H units).
 *   d_evecs    : device out, dim x N_ev column-major FP64, or NULL.
 *   resid      : host out, N_ev residual norms (H units), or NULL.
 *   stats      : host out or NULL.
 * Blocking.  Returns POLFED_ENOCONV with partial results if the column
 * budget ran out. */
int polfed_eigs(polfed_ctx* ctx, const polfed_model* model, double eps_target, int32_t N_ev, int32_t K, int32_t n_b,
                const polfed_opts* opts, double* evals, double* d_evecs, double* resid, polfed_stats* stats);

/* Message of the last failing call on this thread ("" if none). */
const char* polfed_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* POLFED_H */
