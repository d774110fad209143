// Dense block operations of block Lanczos (Eqs. (3)-(4)), FP64 in and out
// (the two contractions compute in float-float, see below):
//   Gram:   C_j = Q_j^T R for a set of N x S panels (re-orthogonalization, A_j, Rayleigh-Ritz)
//   update: Out = beta Out + alpha sum_j Q_j C_j (re-orthogonalization, Ritz vectors u_i = Q t_i)
//   Cholesky QR of an N x S panel (Q_{j+1} B_{j+1} = R_{j+1}), random start block,
//   reductions for single-vector Lanczos, residual column norms, layout transposes.
// Panels are row-major N x S (ld = S) and a basis is panel-major (panel j at j * N * S).
#include <algorithm>
#include <cmath>
#include <mutex>

#include "dense.h"

namespace polfed {

// ------------------------------------------------- float-float arithmetic
// GB300 runs FP64 FMAs at about 1/58 of its FP32 rate, and its FP64 tensor
// path is no faster, so the block contractions below compute in float-float
// on the FP32 pipes: an FP64 operand x is split into hi = fl32(x) and
// lo = fl32(x - hi) (x = hi + lo to about 2^-48 relative), a product is
// hi*hi with its exact rounding error (an FMA) plus the two cross terms, and
// a sum is kept as an unevaluated pair (h, l) grown by Knuth's two-sum and
// renormalized by Dekker's fast two-sum after every tile of rows.  The lo*lo
// term (2^-48 relative) is dropped.  Results go back to FP64 as h + l.
__device__ __forceinline__ float2 ff_split(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(__dsub_rn(v, (double)h)));
}
// (h, l) += x * y
// (the _rn intrinsics keep the compiler from contracting these into FMAs,
// which would break the error terms)
__device__ __forceinline__ void ff_fma(float& h, float& l, float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = fmaf(x.x, y.x, -p);
  e = fmaf(x.x, y.y, e);
  e = fmaf(x.y, y.x, e);
  const float s = __fadd_rn(h, p);
  const float bv = __fsub_rn(s, h);
  const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bv)), __fsub_rn(p, bv));
  h = s;
  l = __fadd_rn(l, __fadd_rn(err, e));
}
__device__ __forceinline__ void ff_norm(float& h, float& l) {
  const float s = __fadd_rn(h, l);
  l = __fsub_rn(l, __fsub_rn(s, h));
  h = s;
}

// ------------------------------------------------------------------ Gram
// partial[(chunk * J + j) * S * S + a * S + b] = sum_{rows in chunk} Q_j[r][a] R[r][b]
// (float-float accumulation over the chunk, FP64 partials)
template <int S>
__global__ void __launch_bounds__(256) k_gram(const double* __restrict__ Q, int64_t pstride,
                                               const double* __restrict__ R, int64_t dim, int64_t rows_per_chunk,
                                               int J, double* __restrict__ partial) {
  constexpr int T = S / 16;  // thread tile T x T
  constexpr int RT = S >= 128 ? 16 : 32;
  extern __shared__ __align__(16) double sh[];
  float2* sQ = reinterpret_cast<float2*>(sh);  // RT x S (hi, lo)
  float2* sR = sQ + RT * S;                    // RT x S
  const int j = blockIdx.y;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk;
  const int64_t r1 = min(dim, r0 + rows_per_chunk);
  const double* Qj = Q + (int64_t)j * pstride;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float ah[T][T], al[T][T];
#pragma unroll
  for (int a = 0; a < T; a++)
#pragma unroll
    for (int b = 0; b < T; b++) ah[a][b] = al[a][b] = 0.f;
  for (int64_t rb = r0; rb < r1; rb += RT) {
    const int nr = (int)min((int64_t)RT, r1 - rb);
    for (int e = threadIdx.x; e < RT * S; e += 256) {
      const int rr = e / S;
      sQ[e] = ff_split(rr < nr ? Qj[(rb + rr) * S + (e - rr * S)] : 0.0);
      sR[e] = ff_split(rr < nr ? R[(rb + rr) * S + (e - rr * S)] : 0.0);
    }
    __syncthreads();
    for (int rr = 0; rr < nr; rr++) {
      float2 q[T], r[T];
#pragma unroll
      for (int a = 0; a < T; a++) q[a] = sQ[rr * S + ty + 16 * a];
#pragma unroll
      for (int b = 0; b < T; b++) r[b] = sR[rr * S + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < T; a++)
#pragma unroll
        for (int b = 0; b < T; b++) ff_fma(ah[a][b], al[a][b], q[a], r[b]);
    }
#pragma unroll
    for (int a = 0; a < T; a++)
#pragma unroll
      for (int b = 0; b < T; b++) ff_norm(ah[a][b], al[a][b]);
    __syncthreads();
  }
  double* P = partial + ((int64_t)blockIdx.x * J + j) * S * S;
#pragma unroll
  for (int a = 0; a < T; a++)
#pragma unroll
    for (int b = 0; b < T; b++) P[(ty + 16 * a) * S + tx + 16 * b] = (double)ah[a][b] + (double)al[a][b];
}

// C[(j*S + a) * ldc + col0 + b] = sum_chunk partial[chunk][j][a][b]
__global__ void k_gram_reduce(const double* __restrict__ partial, int nchunk, int J, int S, double* C, int ldc,
                              int col0) {
  const int64_t n = (int64_t)J * S * S;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nchunk; c++) s += partial[(int64_t)c * n + e];
    const int64_t jb = e / (S * S);
    const int a = (int)((e / S) % S), b = (int)(e % S);
    C[(jb * S + a) * ldc + col0 + b] = s;
  }
}

// ---------------------------------------------------------------- update
// Out[r][b] = beta Out[r][b] + alpha sum_j sum_a Q_j[r][a] C[(j*S + a)*crs + (col0 + b)*ccs]
// One output panel per blockIdx.y: columns col0 = blockIdx.y * S, Out panel at Out + blockIdx.y * ostride.
template <int S>
__global__ void __launch_bounds__(256) k_update(const double* __restrict__ Q, int64_t pstride, int J,
                                                 const double* __restrict__ C, int64_t crs, int64_t ccs,
                                                 int ncols_valid, double* Out, int64_t ostride, int64_t dim,
                                                 double alpha, double beta) {
  constexpr int RT = 32;                 // rows per tile
  constexpr int TR = RT / 16;            // rows per thread
  constexpr int TC = S / 16;             // columns per thread
  extern __shared__ __align__(16) double sh[];
  float2* sC = reinterpret_cast<float2*>(sh);  // S x S (hi, lo)
  float2* sQ = sC + S * S;                     // RT x S
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int col0 = blockIdx.y * S;
  double* O = Out + (int64_t)blockIdx.y * ostride;
  for (int64_t rb = (int64_t)blockIdx.x * RT; rb < dim; rb += (int64_t)gridDim.x * RT) {
    const int nr = (int)min((int64_t)RT, dim - rb);
    float ah[TR][TC], al[TR][TC];  // float-float accumulators
#pragma unroll
    for (int a = 0; a < TR; a++)
#pragma unroll
      for (int b = 0; b < TC; b++) ah[a][b] = al[a][b] = 0.f;
    for (int j = 0; j < J; j++) {
      __syncthreads();
      for (int e = threadIdx.x; e < S * S; e += 256) {
        const int a = e / S, b = e - a * S;
        sC[e] = ff_split((col0 + b < ncols_valid) ? C[((int64_t)j * S + a) * crs + (int64_t)(col0 + b) * ccs] : 0.0);
      }
      const double* Qj = Q + (int64_t)j * pstride;
      for (int e = threadIdx.x; e < RT * S; e += 256) {
        const int rr = e / S;
        sQ[e] = ff_split(rr < nr ? Qj[(rb + rr) * S + (e - rr * S)] : 0.0);
      }
      __syncthreads();
      for (int a = 0; a < S; a++) {
        float2 q[TR], c[TC];
#pragma unroll
        for (int i = 0; i < TR; i++) q[i] = sQ[(ty + 16 * i) * S + a];
#pragma unroll
        for (int k = 0; k < TC; k++) c[k] = sC[a * S + tx + 16 * k];
#pragma unroll
        for (int i = 0; i < TR; i++)
#pragma unroll
          for (int k = 0; k < TC; k++) ff_fma(ah[i][k], al[i][k], q[i], c[k]);
      }
#pragma unroll
      for (int i = 0; i < TR; i++)
#pragma unroll
        for (int k = 0; k < TC; k++) ff_norm(ah[i][k], al[i][k]);
    }
#pragma unroll
    for (int i = 0; i < TR; i++) {
      const int rr = ty + 16 * i;
      if (rr < nr) {
#pragma unroll
        for (int k = 0; k < TC; k++) {
          const int64_t o = (rb + rr) * S + tx + 16 * k;
          const double v = (double)ah[i][k] + (double)al[i][k];
          O[o] = (beta == 0.0 ? 0.0 : beta * O[o]) + alpha * v;
        }
      }
    }
  }
}

// ------------------------------------------------------- small Cholesky
// G (S x S, symmetric positive definite) = L L^T.  Writes Minv = L^{-T}
// (so that Q = R Minv has orthonormal columns) and B = L^T (R = Q B).
// flag[0] |= 1 if a pivot is not positive (rank-deficient block).
__global__ void k_chol_small(const double* __restrict__ G, int S, double* Minv, double* B, int* flag) {
  extern __shared__ double sm[];
  double* A = sm;  // S x S, becomes L (lower)
  for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
    const int i = e / S, j = e % S;
    A[e] = 0.5 * (G[i * S + j] + G[j * S + i]);
  }
  __syncthreads();
  __shared__ double dmax;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < S; i++) m = fmax(m, A[i * S + i]);
    dmax = m;
  }
  __syncthreads();
  for (int k = 0; k < S; k++) {
    if (threadIdx.x == 0) {
      double d = A[k * S + k];
      if (!(d > 1e-28 * dmax)) {
        atomicOr(flag, 1);
        d = fmax(1e-28 * dmax, 1e-300);
      }
      A[k * S + k] = sqrt(d);
    }
    __syncthreads();
    const double piv = A[k * S + k];
    for (int i = k + 1 + threadIdx.x; i < S; i += blockDim.x) A[i * S + k] /= piv;
    __syncthreads();
    const int m = S - k - 1;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j <= i) A[i * S + j] -= A[i * S + k] * A[j * S + k];
    }
    __syncthreads();
  }
  // column c of L^{-1} by forward substitution (one thread per column),
  // stored transposed: Minv[c * S + i] = (L^{-1})[i][c], i.e. Minv = L^{-T}.
  for (int c = threadIdx.x; c < S; c += blockDim.x) {
    double* col = Minv + (size_t)c * S;
    for (int i = 0; i < c; i++) col[i] = 0.0;
    for (int i = c; i < S; i++) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; k++) s -= A[i * S + k] * col[k];
      col[i] = s / A[i * S + i];
    }
  }
  for (int e = threadIdx.x; e < S * S; e += blockDim.x) {
    const int i = e / S, j = e % S;
    B[e] = (j >= i) ? A[j * S + i] : 0.0;  // L^T
  }
}

// ------------------------------------------------------------ small kernels
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void k_random(double* X, int64_t n, uint64_t seed) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t z = splitmix64(seed ^ splitmix64((uint64_t)e));
    X[e] = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
  }
}

// out[0..S) += partial dot products of columns: out[c] = sum_r A[r][c] * B[r][c]
__global__ void k_coldot(const double* __restrict__ A, const double* __restrict__ B, int64_t dim, int S,
                         double* partial) {
  extern __shared__ double red[];
  const int c = threadIdx.x % S;
  const int lane_rows = blockDim.x / S;
  double s = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)lane_rows + threadIdx.x / S; r < dim; r += (int64_t)gridDim.x * lane_rows)
    s = fma(A[r * S + c], B[r * S + c], s);
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < S) {
    double t = 0.0;
    for (int k = threadIdx.x; k < blockDim.x; k += S) t += red[k];
    partial[(int64_t)blockIdx.x * S + threadIdx.x] = t;
  }
}

__global__ void k_reduce_rows(const double* partial, int nblk, int S, double* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= S) return;
  double t = 0.0;
  for (int b = 0; b < nblk; b++) t += partial[(int64_t)b * S + c];
  out[c] = t;
}

// y = a*x + b*y + c*z (vectors of length n)
__global__ void k_axpbypcz(int64_t n, double a, const double* x, double b, double* y, double c, const double* z) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double v = a * x[e] + b * y[e];
    if (z) v += c * z[e];
    y[e] = v;
  }
}

// R[r][c] = W[r][c] - lam[c] * U[r][c]   (residual block, in place into W allowed)
__global__ void k_resid(const double* __restrict__ U, double* W, const double* lam, int64_t dim, int S) {
  const int64_t n = dim * S;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % S);
    W[e] = W[e] - lam[c] * U[e];
  }
}

// panel-major (N x S panels) -> column-major N x n (columns >= n dropped)
__global__ void k_panels_to_colmajor(const double* __restrict__ P, int64_t dim, int S, int n, double* out) {
  const int64_t tot = dim * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / dim, r = e - col * dim;
    const int64_t p = col / S, c = col - p * S;
    out[e] = P[p * dim * S + r * S + c];
  }
}

// Compact column gather on panel-major blocks (N x S panels): column j of
// out (j < nc_pad) is column idx[j] of in for j < nc, zero for j >= nc.
__global__ void k_gather_panel_cols(const double* __restrict__ in, int64_t dim, int S, const int* __restrict__ idx,
                                    int nc, int nc_pad, double* __restrict__ out) {
  const int64_t tot = dim * nc_pad;
  const int64_t pst = dim * S;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / pst, rem = e - p * pst;
    const int64_t r = rem / S;
    const int c = (int)(rem - r * S);
    const int j = (int)(p * S + c);
    double v = 0.0;
    if (j < nc) {
      const int src = idx[j];
      v = in[(int64_t)(src / S) * pst + r * S + (src % S)];
    }
    out[e] = v;
  }
}

// F_i <- pl_i F_i + G_{pos_i} for every column i of npan panels (pos_i < 0: no
// G term); G is a compact panel-major block.
__global__ void k_scale_add_cols(double* F, const double* __restrict__ G, const int* __restrict__ pos,
                                 const double* __restrict__ pl, int64_t dim, int S, int npan) {
  const int64_t pst = dim * S;
  const int64_t tot = pst * npan;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / pst, rem = e - p * pst;
    const int64_t r = rem / S;
    const int c = (int)(rem - r * S);
    const int i = (int)(p * S + c);
    double v = pl[i] * F[e];
    const int j = pos[i];
    if (j >= 0) v += G[(int64_t)(j / S) * pst + r * S + (j % S)];
    F[e] = v;
  }
}

// ------------------------------------------------------------------- host
static int grid_for(int64_t n, int per = 256) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + per - 1) / per, 152 * 8)); }

int Dense::gram(const double* Q, int64_t pstride, int J, const double* R, double* C, int ldc, int col0,
                cudaStream_t s) {
  if (J <= 0) return POLFED_OK;
  int64_t nchunk = std::max<int64_t>(1, std::min<int64_t>((4 * 152 + J - 1) / J, (dim + 2047) / 2048));
  const int64_t rpc = (dim + nchunk - 1) / nchunk;
  nchunk = (dim + rpc - 1) / rpc;
  const size_t need = (size_t)nchunk * J * S * S * sizeof(double);
  PF_CHECK(ensure(partial, partial_bytes, need));
  dim3 grid((unsigned)nchunk, (unsigned)J);
  const int RT = S >= 128 ? 16 : 32;
  const size_t smem = 2 * (size_t)RT * S * sizeof(double);
  switch (S) {
    case 16: k_gram<16><<<grid, 256, smem, s>>>(Q, pstride, R, dim, rpc, J, (double*)partial); break;
    case 32: k_gram<32><<<grid, 256, smem, s>>>(Q, pstride, R, dim, rpc, J, (double*)partial); break;
    case 64: k_gram<64><<<grid, 256, smem, s>>>(Q, pstride, R, dim, rpc, J, (double*)partial); break;
    case 128: k_gram<128><<<grid, 256, smem, s>>>(Q, pstride, R, dim, rpc, J, (double*)partial); break;
    default: return fail(POLFED_EINVAL, "block size must be 16, 32, 64 or 128");
  }
  PF_CUDA(cudaGetLastError());
  k_gram_reduce<<<grid_for((int64_t)J * S * S), 256, 0, s>>>((const double*)partial, (int)nchunk, J, S, C, ldc, col0);
  PF_CUDA(cudaGetLastError());
  count_launch(2);
  return POLFED_OK;
}

int Dense::update(const double* Q, int64_t pstride, int J, const double* C, int64_t crs, int64_t ccs, int ncols,
                  double* Out, int64_t ostride, double alpha, double beta, cudaStream_t s) {
  const int npan = (ncols + S - 1) / S;
  if (npan == 0) return POLFED_OK;
  if (J == 0) {
    if (beta == 1.0) return POLFED_OK;
  }
  const size_t smem = ((size_t)S * S + 32 * (size_t)S) * sizeof(double);
  const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((dim + 31) / 32, (int64_t)(2 * 152 + npan - 1) / npan * 4));
  dim3 grid(gx, npan);
  switch (S) {
    case 16: k_update<16><<<grid, 256, smem, s>>>(Q, pstride, J, C, crs, ccs, ncols, Out, ostride, dim, alpha, beta); break;
    case 32: k_update<32><<<grid, 256, smem, s>>>(Q, pstride, J, C, crs, ccs, ncols, Out, ostride, dim, alpha, beta); break;
    case 64: k_update<64><<<grid, 256, smem, s>>>(Q, pstride, J, C, crs, ccs, ncols, Out, ostride, dim, alpha, beta); break;
    case 128: k_update<128><<<grid, 256, smem, s>>>(Q, pstride, J, C, crs, ccs, ncols, Out, ostride, dim, alpha, beta); break;
    default: return fail(POLFED_EINVAL, "block size must be 16, 32, 64 or 128");
  }
  PF_CUDA(cudaGetLastError());
  count_launch();
  return POLFED_OK;
}

int Dense::cholqr(double* R, double* Qout, double* B_host, int passes, cudaStream_t s, bool* breakdown) {
  // R (N x S) -> Qout (N x S) with Qout B = R; B accumulated over passes (B = B2 B1)
  PF_CHECK(ensure(small, small_bytes, (size_t)(4 * S * S + 8) * sizeof(double)));
  double* G = (double*)small;
  double* Minv = G + S * S;
  double* B = Minv + S * S;
  int* flag = (int*)(B + S * S);
  std::vector<double> Bacc((size_t)S * S, 0.0), Bp((size_t)S * S), tmp((size_t)S * S);
  for (int i = 0; i < S; i++) Bacc[(size_t)i * S + i] = 1.0;
  PF_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
  const double* src = R;
  for (int p = 0; p < passes; p++) {
    PF_CHECK(gram(src, 0, 1, src, G, S, 0, s));
    const size_t smem = (size_t)S * S * sizeof(double);
    k_chol_small<<<1, 256, smem, s>>>(G, S, Minv, B, flag);
    PF_CUDA(cudaGetLastError());
    count_launch();
    // Qout = src * Minv (one panel; in place is safe: each row tile is read before it is written)
    PF_CHECK(update(src, 0, 1, Minv, S, 1, S, Qout, 0, 1.0, 0.0, s));
    PF_CUDA(cudaMemcpyAsync(Bp.data(), B, (size_t)S * S * sizeof(double), cudaMemcpyDeviceToHost, s));
    PF_CUDA(cudaStreamSynchronize(s));
    // Bacc = Bp * Bacc
    for (int i = 0; i < S; i++)
      for (int j = 0; j < S; j++) {
        double t = 0.0;
        for (int k = 0; k < S; k++) t += Bp[(size_t)i * S + k] * Bacc[(size_t)k * S + j];
        tmp[(size_t)i * S + j] = t;
      }
    Bacc.swap(tmp);
    src = Qout;
  }
  int hflag = 0;
  PF_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  if (breakdown) *breakdown = hflag != 0;
  if (B_host) std::copy(Bacc.begin(), Bacc.end(), B_host);
  return POLFED_OK;
}

int Dense::random_fill(double* X, int64_t n, uint64_t seed, cudaStream_t s) {
  k_random<<<grid_for(n), 256, 0, s>>>(X, n, seed);
  PF_CUDA(cudaGetLastError());
  count_launch();
  return POLFED_OK;
}

int Dense::coldot(const double* A, const double* B, int ncol, double* out_host, cudaStream_t s) {
  // column dot products of two N x ncol row-major blocks
  const int threads = std::max(ncol, (256 / ncol) * ncol);
  const int nblk = 152 * 2;
  PF_CHECK(ensure(partial, partial_bytes, (size_t)nblk * ncol * sizeof(double) + (size_t)ncol * sizeof(double)));
  double* part = (double*)partial;
  double* res = part + (size_t)nblk * ncol;
  k_coldot<<<nblk, threads, threads * sizeof(double), s>>>(A, B, dim, ncol, part);
  PF_CUDA(cudaGetLastError());
  k_reduce_rows<<<(ncol + 127) / 128, 128, 0, s>>>(part, nblk, ncol, res);
  PF_CUDA(cudaGetLastError());
  count_launch(2);
  PF_CUDA(cudaMemcpyAsync(out_host, res, (size_t)ncol * sizeof(double), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  return POLFED_OK;
}

int Dense::axpbypcz(int64_t n, double a, const double* x, double b, double* y, double c, const double* z,
                    cudaStream_t s) {
  k_axpbypcz<<<grid_for(n), 256, 0, s>>>(n, a, x, b, y, c, z);
  PF_CUDA(cudaGetLastError());
  count_launch();
  return POLFED_OK;
}

int Dense::resid(const double* U, double* W, const double* lam_dev, cudaStream_t s) {
  k_resid<<<grid_for(dim * S), 256, 0, s>>>(U, W, lam_dev, dim, S);
  PF_CUDA(cudaGetLastError());
  count_launch();
  return POLFED_OK;
}

int Dense::panels_to_colmajor(const double* P, int n, double* out, cudaStream_t s) {
  k_panels_to_colmajor<<<grid_for(dim * n), 256, 0, s>>>(P, dim, S, n, out);
  PF_CUDA(cudaGetLastError());
  count_launch();
  return POLFED_OK;
}

int Dense::gather_cols(const double* in, const int* idx_dev, int nc, int nc_pad, double* out, cudaStream_t s) {
  if (nc_pad <= 0) return POLFED_OK;
  k_gather_panel_cols<<<grid_for(dim * nc_pad), 256, 0, s>>>(in, dim, S, idx_dev, nc, nc_pad, out);
  PF_CUDA(cudaGetLastError());
  count_launch();
  return POLFED_OK;
}

int Dense::scale_add_cols(double* F, const double* G, const int* pos_dev, const double* pl_dev, int npan,
                          cudaStream_t s) {
  k_scale_add_cols<<<grid_for(dim * S * npan), 256, 0, s>>>(F, G, pos_dev, pl_dev, dim, S, npan);
  PF_CUDA(cudaGetLastError());
  count_launch();
  return POLFED_OK;
}

int Dense::ensure(void*& p, size_t& have, size_t need) {
  if (p && have >= need) return POLFED_OK;
  if (p) cudaFree(p);
  p = nullptr;
  have = 0;
  PF_CUDA(cudaMalloc(&p, need));
  have = need;
  return POLFED_OK;
}

void Dense::release() {
  if (partial) cudaFree(partial);
  if (small) cudaFree(small);
  if (tmpbuf) cudaFree(tmpbuf);
  partial = small = tmpbuf = nullptr;
  partial_bytes = small_bytes = tmpbuf_bytes = 0;
}

int Dense::configure() {
  // allow the large dynamic shared memory of the S = 128 kernels
  static std::mutex mu;  // worker threads of the batched runner configure concurrently
  static bool done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && done[dev]) return POLFED_OK;
  const int big = 200 * 1024;
  PF_CUDA(cudaFuncSetAttribute(k_update<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  PF_CUDA(cudaFuncSetAttribute(k_update<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  PF_CUDA(cudaFuncSetAttribute(k_gram<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  PF_CUDA(cudaFuncSetAttribute(k_chol_small, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  if (dev < 64) done[dev] = true;
  return POLFED_OK;
}

}  // namespace polfed
