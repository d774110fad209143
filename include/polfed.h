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
                            followed by refinement sweeps by defect correction (per-column FP32 filters of the
                            residuals against the Jackson-damped transform, FP64 Rayleigh-Ritz) */
  int32_t bounds_steps;  /* max single-vector Lanczos steps for E_min / E_max */
  int32_t verbose;       /* 1 = progress lines on stderr */
  int32_t dos_rule;      /* how K gets the density of states at the target: POLFED_DOS_* */
  uint64_t seed;         /* seed of the random starting block Q_1 (and of the KPM vectors) */
  double rho_hint;       /* POLFED_DOS_HINT: (E_max - E_min) rho(E*) / N, the density of states at the target per
                            unit of rescaled energy eps, per state (e.g. from polfed_mlp_predict) */
  double emin_hint, emax_hint; /* POLFED_DOS_HINT: predicted, padded spectral bounds; used as [e_lo, e_hi] when the
                            Lanczos probe confirms that they contain the spectrum, else ignored (0, 0 = none) */
  int32_t kpm_moments;   /* POLFED_DOS_KPM: Chebyshev moments (default 256) */
  int32_t kpm_vectors;   /* POLFED_DOS_KPM: random vectors of the stochastic trace (default 16) */
  double tol_refine;     /* POLFED_F32: refinement sweeps continue (at most 24; 40 when tol_refine < tol_resid)
                            until every residual is <= tol_refine * ||H||; 0 = tol_resid.  Eigenvector-derived quantities such as the
                            entanglement entropy move with the eigenvector error ~ residual / level spacing, so
                            a smaller value buys them accuracy; acceptance still uses tol_resid */
} polfed_opts;

/* Density-of-states rules for the choice of K (polfed_opts.dos_rule). */
enum {
  POLFED_DOS_MOMENTS = 0, /* Gaussian with the exact sector mean and variance of H (Tr H / N, Tr H^2 / N) */
  POLFED_DOS_GAMMA = 1,   /* the paper's analytic width: Gamma^2 = L [(J1^2 + J2^2)/8 + Delta^2 (J1^2 + J2^2)/16
                             + sum_i h_i^2 / (4L)], centred at the sector mean */
  POLFED_DOS_KPM = 2,     /* stochastic kernel-polynomial estimate at the target (polfed_kpm_moments) */
  POLFED_DOS_HINT = 3     /* the caller's rho_hint (and bounds hints), e.g. from the learned predictor */
};

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
  int64_t n_step_launches; /* launches of the Chebyshev step kernels inside event-timed filter runs */
  double step_gpu_s;       /* device time of those launches (CUDA events on the launching stream) */
  double step_alg_bytes;   /* algorithmic bytes of those launches: N * cols * w * (3 + [c_k != 0]) each */
  int32_t dos_rule;        /* rule that set K */
  int32_t bounds_from_hint;/* 1 if [e_lo, e_hi] came from the caller's (probe-confirmed) bounds hints */
  int32_t n_restarts;      /* restarts with a smaller K because fewer than N_ev eigenvalues had P >= p */
  int32_t fallback_df64;   /* POLFED_F32: 1 if the refinement stalled and a float-float run replaced it */
  int64_t kind_launches[3];  /* the three step counters above by storage kind, */
  double kind_gpu_s[3];      /* indexed POLFED_F64, POLFED_F32, POLFED_DF64 */
  double kind_alg_bytes[3];
} polfed_stats;

typedef struct polfed_ctx polfed_ctx;

/* Default options: p = 0.17, k_margin = 0.2, tol_conv = 1e-7 (tightened until the residuals pass), tol_resid = 1e-8,
 * cols_factor = 2.8, precision = POLFED_DF64, bounds_steps = 600, dos_rule = POLFED_DOS_MOMENTS, seed = 1234,
 * no hints, kpm_moments = 256, kpm_vectors = 16, tol_refine = 0. */
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

/* Y[:, j] = sum_n coeffs[j (K + 1) + n] T_n(H~) X[:, j]: every column through
 * its own order-K Chebyshev series (the Clenshaw recurrence of the text after
 * Eq. (4) with per-column coefficients).  POLFED's mixed-precision refinement
 * uses it for the divided differences g_j(x) = (P(x) - P(lam_j)) / (x - lam_j)
 * of Eq. (2)'s transform at each Ritz value lam_j, applied to the residuals.
 *   K      : 1 <= K <= 10^7.
 *   coeffs : HOST array of n_b (K + 1) doubles, column j's series at coeffs + j (K + 1).
 *   d_X, d_Y : device, row-major dim x n_b FP32 (dtype is FP32 only).
 *   other arguments as in polfed_h_apply.
 * Synchronizes the stream before returning.  POLFED_EBOUNDS if the output is
 * not finite. */
int polfed_cheb_filter_cols(const polfed_model* model, const uint32_t* d_states, int64_t dim, double e_lo,
                            double e_hi, int32_t K, const double* coeffs, const void* d_X, void* d_Y, int32_t n_b,
                            polfed_stream_t stream);

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

/* Phase boundaries of a polfed_eigs run, reported to the progress hook.  The
 * paper's run is a sequence of block-Lanczos steps (Eqs. (3)-(4): one
 * Chebyshev filter of the block, re-orthogonalization, QR and, from some
 * step on, the T_j eigenproblem with the convergence test and the Ritz
 * vectors); the mixed-precision form appends refinement sweeps. */
enum {
  POLFED_PHASE_START = 0,  /* bounds and K chosen; index = K */
  POLFED_PHASE_BLOCK = 1,  /* block-Lanczos step finished; index = j (0-based), counted over restarts */
  POLFED_PHASE_REFINE = 2, /* refinement sweep finished; index = sweep (0-based) */
  POLFED_PHASE_END = 3     /* results written; index = final status */
};

/* Progress hook: fn(user, phase, index) is called on the calling host thread
 * of polfed_eigs / polfed_block_lanczos at every phase boundary above, after
 * the context's stream has been synchronized, so a caller can time whole
 * steps of the method (CUDA events on that stream, wall clocks) or log
 * progress.  fn must not call into this library with the same context.
 * fn = NULL removes the hook.  Not used by the batched runner. */
typedef void (*polfed_progress_fn)(void* user, int32_t phase, int32_t index);
int polfed_ctx_set_progress(polfed_ctx* ctx, polfed_progress_fn fn, void* user);

/* One convergence check of block Lanczos (the eigen-solve of T_j and the test
 * ||B_{j+1} t~_i|| after Eq. (4); the Supplement's "Convergence of POLFED"
 * follows the converged count against the number of Lanczos columns). */
typedef struct polfed_conv_point {
  int32_t step;        /* block-Lanczos step j (1-based) of the attempt */
  int32_t cols;        /* Lanczos columns m s at the check */
  int32_t n_conv;      /* Ritz values theta >= p whose ||B t~|| <= the current tolerance */
  int32_t n_acc;       /* Ritz values theta >= p */
  int32_t attempt;     /* 0 = first run; restarts with a smaller K and the float-float rerun count up */
  int32_t reserved;
  double theta_nev;    /* N_ev-th largest Ritz value (-1 if fewer columns) */
  double max_res_top;  /* largest ||B t~|| among the N_ev largest Ritz values */
} polfed_conv_point;

/* Convergence history of the last polfed_eigs / polfed_block_lanczos call on
 * ctx: copies min(max, available) checks to out (host) and sets *n to the
 * number available. */
int polfed_ctx_history(polfed_ctx* ctx, polfed_conv_point* out, int32_t max, int32_t* n);

/* Process counters of this library's device work issued by the calling host
 * thread since it first called the library (monotone; take differences):
 * kernel launches, and the Chebyshev step kernels' launches, device time
 * (CUDA events around each run of step launches, on the launching stream) and
 * algorithmic bytes N * cols * w * (3 + [c_k != 0]), in all and by storage
 * kind (index POLFED_F64 / POLFED_F32 / POLFED_DF64). */
typedef struct polfed_counters {
  int64_t launches;
  int64_t step_launches;
  double step_gpu_s;
  double step_alg_bytes;
  int64_t kind_launches[3];
  double kind_gpu_s[3];
  double kind_alg_bytes[3];
} polfed_counters;
int polfed_get_counters(polfed_counters* out);

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
 * With K = 0, a run that finds fewer than N_ev Ritz values with P >= p (the
 * density of states was overestimated) restarts, at most twice, with a
 * smaller K.  With precision POLFED_F32 the FP32-stage pairs are refined by
 * defect-correction sweeps (FP32 per-column filters of the residuals, FP64
 * Rayleigh-Ritz; columns already at half the target are locked); if the
 * sweeps stagnate, or would cost more than a float-float run at their
 * observed rate, a float-float (POLFED_DF64) run replaces the result.
 * Blocking.  Returns POLFED_ENOCONV with partial results if the column
 * budget ran out. */
int polfed_eigs(polfed_ctx* ctx, const polfed_model* model, double eps_target, int32_t N_ev, int32_t K, int32_t n_b,
                const polfed_opts* opts, double* evals, double* d_evecs, double* resid, polfed_stats* stats);

/* Spectral bounds E_min, E_max of H by single-vector Lanczos (the first step
 * of the "POLFED algorithm" section): stops when both extreme Ritz values have
 * residual bounds |beta_m t_m| <= 1e-12 max(|E_min|, |E_max|) or after
 * opts.bounds_steps steps (opts of the last polfed_eigs call on ctx, else
 * defaults).
 *   bounds : host out, {E_min, E_max, err} with err the larger residual bound.
 * Blocking. */
int polfed_spectral_bounds(polfed_ctx* ctx, const polfed_model* model, double* bounds);

/* Stochastic Chebyshev moments of H~ (kernel polynomial method; the paper
 * cites such estimators for the density of states that fixes K):
 *   mu[n] = (1/R) sum_{r<R} x_r^T T_n(H~) x_r,  n = 0..n_mom-1,
 * with x_r the columns of d_R.  E[mu_n] = Tr T_n(H~) when the entries of x_r
 * are independent with zero mean and unit variance.
 *   e_lo, e_hi : rescaling interval (must contain the spectrum).
 *   n_mom      : 2 <= n_mom <= 65536; takes ceil(n_mom / 2) applications of H~
 *                (T_{2k} = 2 T_k^2 - T_0, T_{2k+1} = 2 T_{k+1} T_k - T_1).
 *   d_R        : device, row-major dim x R (float for POLFED_F32, else double), read only.
 *   R          : 1..128.
 *   dtype      : arithmetic of the H~ applications (POLFED_F64 / DF64 / F32).
 *   mu         : host out, n_mom doubles.
 * Synchronizes the stream.  POLFED_EBOUNDS if some |mu_n| > 1.01 mu_0
 * (spectrum outside [e_lo, e_hi]). */
int polfed_kpm_moments(const polfed_model* model, const uint32_t* d_states, int64_t dim, double e_lo, double e_hi,
                       int32_t n_mom, const void* d_R, int32_t R, int32_t dtype, double* mu, polfed_stream_t stream);

/* Fraction of the spectrum of H~ inside [x_a, x_b] (-1 <= x_a <= x_b <= 1)
 * from KPM moments: sum_n g_n c_n mu_n / mu_0 with Jackson factors g_n (Weisse
 * et al., Rev. Mod. Phys. 78, 275, Eq. (71), N = n_mom) and the indicator's
 * Chebyshev coefficients c_0 = (th_a - th_b)/pi, c_n = 2 (sin n th_a - sin n th_b)/(n pi),
 * th = arccos x.  Host only. */
int polfed_kpm_count(const double* mu, int32_t n_mom, double x_a, double x_b, double* fraction);

/* Labels for the learned predictor, produced by the method's own machinery:
 * out[0] = E_min, out[1] = E_max (polfed_spectral_bounds), out[2] = the
 * density of states at E* = E_min + eps_target (E_max - E_min) per unit of
 * eps and per state, (E_max - E_min) rho(E*) / N, from the KPM eigenvalue
 * count of a window around E* (n_mom moments, R random vectors seeded by
 * opts.seed).  Blocking. */
int polfed_spectral_labels(polfed_ctx* ctx, const polfed_model* model, double eps_target, int32_t n_mom, int32_t R,
                           double* out);

/* ------------------------------------------------------------------------
 * Learned predictor of the spectral bounds and of the density of states
 * (the paper has no counterpart: it takes E_min / E_max from Lanczos and
 * rho from a Gaussian estimate).  A fully connected FP32 network
 * x -> tanh(W1 x + b1) -> tanh(W2 . + b2) -> W3 . + b3, trained and evaluated
 * by this library's kernels.  Parameters are one float array:
 * W1 [H x d_in] row-major, b1 [H], W2 [H x H], b2 [H], W3 [d_out x H], b3 [d_out].
 * Inputs and targets are standardized inside the network with the affine
 * maps set by polfed_mlp_set_scaling (identity by default):
 * x' = (x - x_mean) / x_std, and the network's outputs are in units of
 * (y - y_mean) / y_std.  All device arrays are row-major B x d.
 * ------------------------------------------------------------------------ */
typedef struct polfed_mlp polfed_mlp;

/* d_in 1..1024, hidden d_out..4096, d_out 1..64; weights uniform in
 * +-sqrt(6 / (fan_in + fan_out)) from a splitmix64 stream of seed, biases 0.
 * The network lives on the current device. */
int polfed_mlp_create(int32_t d_in, int32_t hidden, int32_t d_out, uint64_t seed, polfed_mlp** out);
void polfed_mlp_destroy(polfed_mlp* net);
int32_t polfed_mlp_num_params(const polfed_mlp* net);
/* Host copies of the parameters (set also resets the Adam state). */
int polfed_mlp_set_params(polfed_mlp* net, const float* host);
int polfed_mlp_get_params(const polfed_mlp* net, float* host);
/* Host arrays of d_in (x) and d_out (y) floats; std entries must be > 0. */
int polfed_mlp_set_scaling(polfed_mlp* net, const float* x_mean, const float* x_std, const float* y_mean,
                           const float* y_std);
/* d_y = network(d_x) in target units (de-standardized); B >= 1.  Synchronizes the stream. */
int polfed_mlp_forward(polfed_mlp* net, const float* d_x, int32_t B, float* d_y, polfed_stream_t stream);
/* Gradient of the loss 0.5/B sum_b |f(x_b) - t'_b|^2 (t' = standardized targets)
 * with respect to the parameters; d_grad (device, num_params floats) may be
 * NULL; loss (host) may be NULL.  Synchronizes the stream. */
int polfed_mlp_grad(polfed_mlp* net, const float* d_x, const float* d_t, int32_t B, float* d_grad, float* loss,
                    polfed_stream_t stream);
/* One Adam step (Kingma & Ba; beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected)
 * on the gradient above with learning rate lr.  Synchronizes the stream. */
int polfed_mlp_train_step(polfed_mlp* net, const float* d_x, const float* d_t, int32_t B, float lr, float* loss,
                          polfed_stream_t stream);
/* Feature and target conventions of the spectral predictor (d_in = L + 1, d_out = 3):
 *   x = (h_0, ..., h_{L-1}, W)   (W: the disorder strength the fields were drawn with)
 *   y = (E_min / L, E_max / L, log rho_eps), rho_eps = (E_max - E_min) rho(E*) / N.
 * polfed_mlp_features writes x (host, L + 1 floats); polfed_mlp_targets maps
 * labels {E_min, E_max, rho_eps} (host) of a chain of length L to y (host, 3 floats). */
int polfed_mlp_features(const polfed_model* model, double W, float* x);
int polfed_mlp_targets(int32_t L, const double* labels, float* y);
/* Prediction for one realization: out = {E_min, E_max, rho_eps} (host), i.e.
 * the inverse of polfed_mlp_targets applied to the network's output for
 * polfed_mlp_features(model, W).  Needs d_in == L + 1 and d_out == 3.  Blocking. */
int polfed_mlp_predict(polfed_mlp* net, const polfed_model* model, double W, double* out);

/* ------------------------------------------------------------------------
 * Batched runner (the paper runs disorder realizations independently, one
 * per compute node; this is the single-GPU form of that parallelism).
 * ------------------------------------------------------------------------ */

/* Eq. (2) filter of many realizations in ONE cooperative kernel launch: every
 * (realization, 128-byte column slice) job runs its own Clenshaw recurrence of
 * order K[i] with the paper's coefficients for sigma[i], on its own H~ (plans
 * with the low/high split b = min(10, L - 4)).  Launch step t performs step t
 * of every job with t < K[i]; CTAs meet at a grid barrier between steps
 * (bounded wait: POLFED_ETIMEOUT, never a hang).
 *   n_inst       : number of realizations (>= 1); all with J2 == 0 or all with J2 != 0.
 *   models       : host array of n_inst models (any mix of L).
 *   e_lo, e_hi, sigma, K : host arrays of n_inst (as in polfed_cheb_filter, K <= 1e7).
 *   d_X, d_Y     : host arrays of n_inst device pointers, row-major dim_i x n_b
 *                  (float for POLFED_F32, double for POLFED_DF64); X_i, Y_i must not overlap.
 *   n_b          : 1..128 (the same for all).
 *   dtype        : POLFED_F32 or POLFED_DF64.
 *   ctas_per_sm  : 0 = as many as fit (1 or 2), else 1 or 2.
 * Synchronizes the stream.  POLFED_EBOUNDS if an output grew beyond the
 * Chebyshev bound. */
int polfed_cheb_filter_batched(int32_t n_inst, const polfed_model* models, const double* e_lo, const double* e_hi,
                               const double* sigma, const int32_t* K, const void* const* d_X, void* const* d_Y,
                               int32_t n_b, int32_t dtype, int32_t ctas_per_sm, polfed_stream_t stream);

/* What polfed_eigs_batched did. */
typedef struct polfed_batch_info {
  int32_t n_b;              /* block width of realization 0 */
  int32_t ctas_per_sm;      /* grid of the batched filter (0 = all that fit) */
  int32_t rounds;           /* batched filter launches */
  int32_t workers;          /* host threads */
  int32_t n_width16, n_width32, n_width64; /* realizations per block width */
  int32_t reserved;
  double t_total;           /* seconds, whole call */
  double t_tune;            /* seconds spent autotuning */
  double filter_gpu_s;      /* device time of the batched filter launches (CUDA events) */
  double filter_alg_bytes;  /* their algorithmic bytes (Clenshaw minimum) */
  double tune_step_s[3][2]; /* autotuner: seconds per filter step for widths 16/32/64 x 1/2 CTAs per SM */
  int64_t n_launches;       /* kernels launched by the call */
} polfed_batch_info;

/* polfed_eigs for n_inst realizations at once.  Each realization runs the
 * polfed_eigs driver on its own host thread, context and stream (at most
 * max_workers at a time, 0 = 64); their filter calls meet and run as one
 * polfed_cheb_filter_batched-style launch per round, while the dense block
 * work of all realizations proceeds concurrently.
 *   device     : CUDA device ordinal.
 *   eps_target, N_ev, K : host arrays of n_inst (K may be NULL = all automatic).
 *   n_b        : block width for all, or 0 = autotune: the batched filter is timed on the
 *                realizations' operators for widths 16/32/64 and 1/2 CTAs per SM, and each
 *                realization takes the width with the least predicted filter time.
 *   opts       : options (precision POLFED_F32 or POLFED_DF64), or NULL.
 *   evals      : host out, sum(N_ev) values: realization i at offset sum_{j<i} N_ev[j].
 *   resid      : host out like evals, or NULL.
 *   d_evecs    : host array of n_inst device pointers (dim_i x N_ev[i] column-major FP64,
 *                each may be NULL), or NULL.
 *   stats      : host out, n_inst, or NULL (launch and time counters of a realization
 *                include the batched launches its thread issued for the whole round).
 *   status     : host out, n_inst statuses.
 *   info       : host out or NULL.
 * Blocking.  Returns the first failing realization's status (the others still run). */
int polfed_eigs_batched(int32_t device, int32_t n_inst, const polfed_model* models, const double* eps_target,
                        const int32_t* N_ev, const int32_t* K, int32_t n_b, const polfed_opts* opts,
                        int32_t max_workers, double* evals, double* resid, double* const* d_evecs,
                        polfed_stats* stats, int32_t* status, polfed_batch_info* info);

/* Test support for the failure path (the paper has no counterpart).  Every
 * device-side wait of this library is bounded: the bulk-copy pipeline of the
 * step kernel polls its mbarriers at most 2^22 times, the grid barrier of the
 * batched filter at most 2^24 times (about a second); a wait that runs out
 * makes the kernel stop, wait with the full cap for the copies it already
 * issued, and the call returns POLFED_ETIMEOUT with its output discarded.
 * polfed_set_wait_limit(polls) lowers both caps to `polls` for the calls that
 * follow in this process (0 restores the defaults), so a test can make the
 * waits run out without stalling anything.  Not for production use. */
int polfed_set_wait_limit(uint32_t polls);

/* ------------------------------------------------------------------------
 * Observables of the eigenpairs (section "Entanglement entropy and level
 * statistics").
 * ------------------------------------------------------------------------ */

/* Mean gap ratio r = (1 / (n - 2)) sum_i min(g_i, g_{i+1}) / max(g_i, g_{i+1}),
 * g_i = E_{i+1} - E_i (the level-statistics indicator of that section).
 *   d_evals : device, n eigenvalues in ascending order (e.g. polfed_eigs' evals copied over).
 *   n       : >= 3.
 *   r_mean  : host out.
 *   d_r     : device out, the n - 2 ratios r_i, or NULL.
 * Synchronizes the stream.  POLFED_EINVAL if the values are not ascending or
 * two consecutive gaps are both zero (the ratio is undefined). */
int polfed_gap_ratio(const double* d_evals, int32_t n, double* r_mean, double* d_r, polfed_stream_t stream);

/* Half-chain entanglement entropy S_E = -sum alpha^2 ln alpha^2 of S^z = 0
 * sector vectors for the cuts A = [x, x + L/2) (sites mod L) of that section,
 * from the Schmidt coefficients alpha (per block of fixed magnetization of A,
 * the eigenvalues of M_k M_k^T, natural logarithm).
 *   ctx      : context (device, stream, cuSOLVER handle).
 *   L        : even, 4 <= L <= 32.
 *   d_states : device basis from polfed_basis_build(L, L/2).
 *   d_vecs   : device, column-major dim x n_vec FP64 (vector v at d_vecs + v * ld), normalized
 *              (e.g. polfed_eigs' d_evecs).
 *   per_cut  : 0 = S[v] is the average over the L cut positions x = 0..L-1;
 *              1 = S[v * L + x] is the entropy of cut x.
 *   S        : host out.
 * Uses stream-ordered device scratch of about 2 GiB at most.  Blocking. */
int polfed_entanglement_entropy(polfed_ctx* ctx, int32_t L, const uint32_t* d_states, const double* d_vecs,
                                int64_t ld, int32_t n_vec, int32_t per_cut, double* S);

/* Message of the last failing call on this thread ("" if none). */
const char* polfed_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* POLFED_H */
