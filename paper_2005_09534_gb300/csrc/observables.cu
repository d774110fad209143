// Observables of the eigenpairs (section "Entanglement entropy and level
// statistics"): the mean gap ratio of a sorted spectrum and the half-chain
// entanglement entropy of sector eigenvectors.
//
// Gap ratio: r_i = min(g_i, g_{i+1}) / max(g_i, g_{i+1}), g_i = E_{i+1} - E_i,
// averaged over i.
//
// Entanglement entropy of the bipartition A = sites [x, x + L/2) (mod L), B =
// the rest: S = -sum alpha^2 ln alpha^2 over the Schmidt coefficients alpha.
// In the S^z = 0 sector the amplitude matrix psi[a][b] (a: configuration of A,
// b: configuration of B) is block diagonal in the number k of up spins in A:
// block k is C(L/2, k) x C(L/2, L/2 - k), rows and columns ranked within their
// popcount class by the combinatorial number system.  The alpha^2 of block k
// are the eigenvalues of its Gram matrix G_k = M_k M_k^T, a small symmetric
// projected eigenproblem (the reduced density matrix rho_A restricted to k up
// spins) solved with cuSOLVER's batched symmetric eigensolver.  The blocks of
// one vector hold sum_k C(L/2, k)^2 = C(L, L/2) = N entries, so a vector's
// blocks and Gram matrices each take N doubles.
// A and its complement have the same entropy, so cut x + L/2 repeats cut x:
// L/2 cuts are computed and the average over the L positions x is their mean.
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "polfed_internal.h"

namespace polfed {

namespace {

// C(n, k) for n, k <= 16 from a per-CTA Pascal triangle
struct SmallBinom {
  uint32_t c[17][17];
};

__device__ void fill_binom(SmallBinom& b) {
  if (threadIdx.x == 0) {
    for (int n = 0; n <= 16; n++)
      for (int k = 0; k <= 16; k++) b.c[n][k] = 0;
    for (int n = 0; n <= 16; n++) {
      b.c[n][0] = 1;
      for (int k = 1; k <= n; k++) b.c[n][k] = b.c[n - 1][k - 1] + (k <= n - 1 ? b.c[n - 1][k] : 0);
    }
  }
  __syncthreads();
}

// colex rank of an h-bit string among those of equal popcount: sum_j C(p_j, j + 1)
__device__ __forceinline__ uint32_t colex_rank(uint32_t a, const SmallBinom& b) {
  uint32_t r = 0;
  int j = 0;
  while (a) {
    const int p = __ffs(a) - 1;
    r += b.c[p][++j];
    a &= a - 1;
  }
  return r;
}

// Scatter the amplitudes of nv vectors into the Schmidt blocks of cut x:
// M[v * N + boff[k] + ra * C_k + rb] = psi_v[r] with s = states[r] rotated so
// that site x is bit 0, a = its low h bits (subsystem A), b = its high h bits.
__global__ void k_schmidt_scatter(const uint32_t* __restrict__ states, int64_t dim, int L, int x,
                                  const double* __restrict__ vecs, int64_t ld, int nv, const int64_t* boff,
                                  double* __restrict__ M) {
  __shared__ SmallBinom sb;
  fill_binom(sb);
  const int h = L / 2;
  const uint32_t full = (L == 32) ? 0xFFFFFFFFu : ((1u << L) - 1u);
  const uint32_t hmask = (1u << h) - 1u;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < dim; r += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t s = states[r];
    const uint32_t rot = x == 0 ? s : (((s >> x) | (s << (L - x))) & full);
    const uint32_t a = rot & hmask, b = rot >> h;
    const int k = __popc(a);
    const uint32_t Ck = sb.c[h][k];
    const int64_t off = boff[k] + (int64_t)colex_rank(a, sb) * Ck + colex_rank(b, sb);
    for (int v = 0; v < nv; v++) M[(int64_t)v * dim + off] = vecs[(int64_t)v * ld + r];
  }
}

// G_k = M_k M_k^T for every (vector, block): 32 x 32 output tiles, 256 threads,
// FP64.  Block k of vector v: M at v * N + boff[k], G at goff[k] + v * C_k^2
// (the Gram matrices of one block index are contiguous over the vectors, the
// layout the batched eigensolver takes).
struct GramJob {
  int k, n, tiles;      // block index, C_k, tiles per side
  int64_t boff, goff;   // offsets of M_k in a vector's blocks, of G_k's region
  int64_t tile0;        // first global tile of this block index (over vectors)
};

__global__ void __launch_bounds__(256) k_schmidt_gram(const double* __restrict__ M, int64_t dim, const GramJob* jobs,
                                                      int n_jobs, int nv, double* __restrict__ G) {
  __shared__ double As[32][33], Bs[32][33];
  // find the job of this CTA (jobs in tile0 order)
  const int64_t t = blockIdx.x;
  int j = 0;
  while (j + 1 < n_jobs && jobs[j + 1].tile0 <= t) j++;
  const GramJob J = jobs[j];
  const int64_t local = t - J.tile0;
  const int per_vec = J.tiles * J.tiles;
  const int v = (int)(local / per_vec);
  if (v >= nv) return;
  const int ti = (int)(local % per_vec) / J.tiles, tj = (int)(local % per_vec) % J.tiles;
  const int n = J.n;
  const double* Mk = M + (int64_t)v * dim + J.boff;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 8 rows of 32
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int c0 = 0; c0 < n; c0 += 32) {
    for (int q = 0; q < 4; q++) {
      const int row = ty + 8 * q;
      const int gi = ti * 32 + row, gj = tj * 32 + row, gc = c0 + tx;
      As[row][tx] = (gi < n && gc < n) ? Mk[(int64_t)gi * n + gc] : 0.0;
      Bs[row][tx] = (gj < n && gc < n) ? Mk[(int64_t)gj * n + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int c = 0; c < 32; c++) {
      const double bv = Bs[tx][c];
#pragma unroll
      for (int q = 0; q < 4; q++) acc[q] = fma(As[ty + 8 * q][c], bv, acc[q]);
    }
    __syncthreads();
  }
  double* Gk = G + J.goff + (int64_t)v * n * n;
  for (int q = 0; q < 4; q++) {
    const int gi = ti * 32 + ty + 8 * q, gj = tj * 32 + tx;
    if (gi < n && gj < n) Gk[(int64_t)gj * n + gi] = acc[q];  // symmetric: either order
  }
}

// -sum lambda ln lambda over the eigenvalues of every block of vector v
// (lambda <= 0 from rounding contributes nothing); one CTA per vector, fixed
// summation order.  W holds the eigenvalues at the Gram layout's offsets
// divided by C_k (woff[k] + v * C_k).
__global__ void k_schmidt_entropy(const double* __restrict__ W, const int64_t* woff, const int* sizes, int nblk,
                                  int nv, double* out, int64_t out_stride) {
  __shared__ double red[256];
  const int v = blockIdx.x;
  if (v >= nv) return;
  double s = 0.0;
  for (int k = 0; k < nblk; k++) {
    const int n = sizes[k];
    const double* w = W + woff[k] + (int64_t)v * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double l = w[i];
      if (l > 0.0) s -= l * log(l);
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(int64_t)v * out_stride] = red[0];
}

// r_i for i = 0..n-3 and their sum, one CTA (fixed order); flag[0] = 1 if the
// values are not ascending, flag[1] = 1 if two consecutive gaps are both zero.
__global__ void k_gap_ratio(const double* __restrict__ e, int n, double* r_out, double* sum_out, int* flag) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i + 2 < n; i += blockDim.x) {
    const double g0 = e[i + 1] - e[i], g1 = e[i + 2] - e[i + 1];
    if (g0 < 0.0 || g1 < 0.0) flag[0] = 1;
    const double mx = fmax(g0, g1), mn = fmin(g0, g1);
    double r = 0.0;
    if (mx > 0.0)
      r = mn / mx;
    else
      flag[1] = 1;
    if (r_out) r_out[i] = r;
    s += r;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *sum_out = red[0];
}

struct StreamMem {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  ~StreamMem() {
    if (p) cudaFreeAsync(p, s);
  }
};

uint64_t binom64(int n, int k) {
  if (k < 0 || k > n) return 0;
  uint64_t r = 1;
  for (int i = 1; i <= k; i++) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
  return r;
}

}  // namespace

}  // namespace polfed

using namespace polfed;

extern "C" {

int polfed_gap_ratio(const double* d_evals, int32_t n, double* r_mean, double* d_r, polfed_stream_t stream) {
  clear_error();
  if (!d_evals || !r_mean) return fail(POLFED_EINVAL, "d_evals or r_mean is NULL");
  if (n < 3) return fail(POLFED_EINVAL, "need at least 3 eigenvalues");
  cudaStream_t s = (cudaStream_t)stream;
  StreamMem mem;
  mem.s = s;
  PF_CUDA(cudaMallocAsync(&mem.p, 64, s));
  double* sum = (double*)mem.p;
  int* flag = (int*)((char*)mem.p + 32);
  PF_CUDA(cudaMemsetAsync(mem.p, 0, 64, s));
  k_gap_ratio<<<1, 1024, 0, s>>>(d_evals, n, d_r, sum, flag);
  PF_CUDA(cudaGetLastError());
  count_launch();
  double hs = 0.0;
  int hf[2] = {0, 0};
  PF_CUDA(cudaMemcpyAsync(&hs, sum, sizeof(double), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaMemcpyAsync(hf, flag, sizeof(hf), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  if (hf[0]) return fail(POLFED_EINVAL, "eigenvalues are not in ascending order");
  if (hf[1]) return fail(POLFED_EINVAL, "two consecutive zero gaps: the gap ratio is undefined");
  *r_mean = hs / (double)(n - 2);
  return POLFED_OK;
}

int polfed_entanglement_entropy(polfed_ctx* ctx, int32_t L, const uint32_t* d_states, const double* d_vecs,
                                int64_t ld, int32_t n_vec, int32_t per_cut, double* S) {
  clear_error();
  if (!ctx) return fail(POLFED_EINVAL, "ctx is NULL");
  if (L < 4 || L > 32 || (L & 1)) return fail(POLFED_EINVAL, "L must be even, 4 <= L <= 32");
  if (!d_states || !d_vecs || !S) return fail(POLFED_EINVAL, "NULL pointer");
  const int h = L / 2;
  if (h > 16) return fail(POLFED_EINVAL, "L must be <= 32");
  const int64_t dim = (int64_t)binom64(L, h);
  if (ld < dim) return fail(POLFED_EINVAL, "ld must be >= C(L, L/2)");
  if (n_vec < 1) return fail(POLFED_EINVAL, "n_vec must be >= 1");
  const int dev = ctx_device(ctx);
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(dev);
  struct Restore {
    int d;
    ~Restore() { cudaSetDevice(d); }
  } restore{prev};
  cudaStream_t s = ctx_stream(ctx);
  cusolverDnHandle_t solver = (cusolverDnHandle_t)ctx_solver(ctx);
  // blocks k = 0..h (C_k = C(h, k)); Gram regions ordered k = 0, h, 1, h-1, ... so that the two
  // blocks of equal size sit next to each other (one batched eigen-solve per size)
  std::vector<int> sizes(h + 1);
  std::vector<int64_t> boff(h + 2, 0);
  for (int k = 0; k <= h; k++) {
    sizes[k] = (int)binom64(h, k);
    boff[k + 1] = boff[k] + (int64_t)sizes[k] * sizes[k];
  }
  // batch of vectors per pass: blocks + Gram matrices (2 N doubles each) within ~1 GiB
  const int nv_max = (int)std::max<int64_t>(1, std::min<int64_t>(n_vec, (int64_t)(1 << 30) / (16 * dim)));
  std::vector<int> order;  // block order of the Gram regions
  for (int k = 0; k <= h / 2; k++) {
    order.push_back(k);
    if (h - k != k) order.push_back(h - k);
  }
  std::vector<int64_t> goff(h + 1), woff(h + 1);
  {
    int64_t g = 0, w = 0;
    for (int k : order) {
      goff[k] = g;
      woff[k] = w;
      g += (int64_t)nv_max * sizes[k] * sizes[k];
      w += (int64_t)nv_max * sizes[k];
    }
  }
  // Gram jobs (tiles) in block order
  std::vector<GramJob> jobs;
  int64_t tiles_total = 0;
  for (int k = 0; k <= h; k++) {
    GramJob J;
    J.k = k;
    J.n = sizes[k];
    J.tiles = (sizes[k] + 31) / 32;
    J.boff = boff[k];
    J.goff = goff[k];
    J.tile0 = tiles_total;
    tiles_total += (int64_t)nv_max * J.tiles * J.tiles;
    jobs.push_back(J);
  }
  // batched eigensolver workspace per size class
  cusolverDnParams_t params = nullptr;
  if (cusolverDnCreateParams(&params) != CUSOLVER_STATUS_SUCCESS) return fail(POLFED_ECUDA, "cusolverDnCreateParams");
  struct Params {
    cusolverDnParams_t p;
    ~Params() { cusolverDnDestroyParams(p); }
  } pguard{params};
  size_t ws_dev = 0, ws_host = 0;
  for (size_t q = 0; q < order.size();) {
    const int k = order[q];
    const int n = sizes[k];
    const int cnt = (q + 1 < order.size() && sizes[order[q + 1]] == n) ? 2 : 1;
    size_t d = 0, hh = 0;
    if (cusolverDnXsyevBatched_bufferSize(solver, params, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                          CUDA_R_64F, nullptr, n, CUDA_R_64F, nullptr, CUDA_R_64F, &d, &hh,
                                          (int64_t)cnt * nv_max) != CUSOLVER_STATUS_SUCCESS)
      return fail(POLFED_ECUDA, "cusolverDnXsyevBatched_bufferSize failed");
    ws_dev = std::max(ws_dev, d);
    ws_host = std::max(ws_host, hh);
    q += cnt;
  }
  const size_t a256 = 255;
  auto up = [&](size_t b) { return (b + a256) & ~a256; };
  const size_t bM = up((size_t)nv_max * dim * 8), bG = up((size_t)nv_max * dim * 8), bW = up((size_t)nv_max * dim * 8);
  const size_t bOff = up((h + 2) * 8 * 3), bJobs = up(jobs.size() * sizeof(GramJob)), bSz = up((h + 1) * 4);
  const size_t bInfo = up((size_t)2 * nv_max * 4), bS = up((size_t)n_vec * h * 8), bWs = up(ws_dev + 16);
  StreamMem mem;
  mem.s = s;
  if (cudaMallocAsync(&mem.p, bM + bG + bW + bOff + bJobs + bSz + bInfo + bS + bWs, s) != cudaSuccess) {
    cudaGetLastError();
    return fail(POLFED_ENOMEM, "device workspace for the Schmidt blocks");
  }
  char* base = (char*)mem.p;
  double* M = (double*)base;
  double* G = (double*)(base + bM);
  double* Wd = (double*)(base + bM + bG);
  int64_t* d_boff = (int64_t*)(base + bM + bG + bW);
  int64_t* d_woff = d_boff + (h + 2);
  GramJob* d_jobs = (GramJob*)(base + bM + bG + bW + bOff);
  int* d_sizes = (int*)(base + bM + bG + bW + bOff + bJobs);
  int* d_info = (int*)(base + bM + bG + bW + bOff + bJobs + bSz);
  double* d_S = (double*)(base + bM + bG + bW + bOff + bJobs + bSz + bInfo);
  void* d_ws = base + bM + bG + bW + bOff + bJobs + bSz + bInfo + bS;
  std::vector<char> h_ws(ws_host + 16);
  std::vector<int64_t> offs(2 * (h + 2), 0);
  for (int k = 0; k <= h + 1; k++) offs[k] = boff[k];
  for (int k = 0; k <= h; k++) offs[h + 2 + k] = woff[k];
  PF_CUDA(cudaMemcpyAsync(d_boff, offs.data(), offs.size() * 8, cudaMemcpyHostToDevice, s));
  PF_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(GramJob), cudaMemcpyHostToDevice, s));
  PF_CUDA(cudaMemcpyAsync(d_sizes, sizes.data(), sizes.size() * 4, cudaMemcpyHostToDevice, s));
  std::vector<int> hinfo(2 * nv_max);
  for (int v0 = 0; v0 < n_vec; v0 += nv_max) {
    const int nv = std::min(nv_max, n_vec - v0);
    for (int x = 0; x < h; x++) {
      const int grid = (int)std::min<int64_t>((dim + 255) / 256, 152 * 8);
      k_schmidt_scatter<<<grid, 256, 0, s>>>(d_states, dim, L, x, d_vecs + (int64_t)v0 * ld, ld, nv, d_boff, M);
      PF_CUDA(cudaGetLastError());
      count_launch();
      // tiles of the vectors present (the job table is laid out for nv_max vectors; CTAs of absent
      // vectors return at once)
      k_schmidt_gram<<<(unsigned)tiles_total, 256, 0, s>>>(M, dim, d_jobs, (int)jobs.size(), nv, G);
      PF_CUDA(cudaGetLastError());
      count_launch();
      for (size_t q = 0; q < order.size();) {
        const int k = order[q];
        const int n = sizes[k];
        const int cnt = (q + 1 < order.size() && sizes[order[q + 1]] == n) ? 2 : 1;
        // the regions of the cnt blocks are adjacent; with nv < nv_max the second one starts
        // nv_max matrices after the first, so solve each block's nv matrices separately then
        for (int c = 0; c < cnt; c++) {
          const int kk = order[q + c];
          if (n == 1) {  // a 1 x 1 block is its own eigenvalue
            PF_CUDA(cudaMemcpyAsync(Wd + woff[kk], G + goff[kk], (size_t)nv * 8, cudaMemcpyDeviceToDevice, s));
            continue;
          }
          if (cusolverDnXsyevBatched(solver, params, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                     CUDA_R_64F, G + goff[kk], n, CUDA_R_64F, Wd + woff[kk], CUDA_R_64F, d_ws,
                                     ws_dev, h_ws.data(), ws_host, d_info, (int64_t)nv) != CUSOLVER_STATUS_SUCCESS)
            return fail(POLFED_ECUDA, "cusolverDnXsyevBatched failed");
          PF_CUDA(cudaMemcpyAsync(hinfo.data(), d_info, (size_t)nv * 4, cudaMemcpyDeviceToHost, s));
          PF_CUDA(cudaStreamSynchronize(s));
          for (int i = 0; i < nv; i++)
            if (hinfo[i] != 0) return fail(POLFED_ECUDA, "batched eigen-solve info = " + std::to_string(hinfo[i]));
        }
        q += cnt;
      }
      k_schmidt_entropy<<<nv, 256, 0, s>>>(Wd, d_woff, d_sizes, h + 1, nv, d_S + (int64_t)v0 * h + x, h);
      PF_CUDA(cudaGetLastError());
      count_launch();
    }
  }
  std::vector<double> Sh((size_t)n_vec * h);
  PF_CUDA(cudaMemcpyAsync(Sh.data(), d_S, Sh.size() * 8, cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  for (int v = 0; v < n_vec; v++) {
    if (per_cut) {
      for (int x = 0; x < L; x++) S[(size_t)v * L + x] = Sh[(size_t)v * h + (x % h)];
    } else {
      double a = 0.0;
      for (int x = 0; x < h; x++) a += Sh[(size_t)v * h + x];
      S[v] = a / h;
    }
  }
  return POLFED_OK;
}

}  // extern "C"
