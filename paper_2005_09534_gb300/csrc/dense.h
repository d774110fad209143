// FP64 dense block operations (see dense.cu).
#pragma once

#include <vector>

#include "polfed_internal.h"

namespace polfed {

struct Dense {
  int64_t dim = 0;
  int S = 0;  // block size: 16, 32, 64 or 128
  void* partial = nullptr;
  size_t partial_bytes = 0;
  void* small = nullptr;
  size_t small_bytes = 0;
  void* tmpbuf = nullptr;
  size_t tmpbuf_bytes = 0;

  int configure();
  // C[(j*S + a) * ldc + col0 + b] = (Q_j^T R)[a][b] for panels j < J (panel stride pstride)
  int gram(const double* Q, int64_t pstride, int J, const double* R, double* C, int ldc, int col0, cudaStream_t s);
  // Out_p = beta Out_p + alpha sum_j Q_j C_j[:, pS:(p+1)S] for output panels p (ncols columns),
  // C element (row k, col c) at C[k * crs + c * ccs]
  int update(const double* Q, int64_t pstride, int J, const double* C, int64_t crs, int64_t ccs, int ncols,
             double* Out, int64_t ostride, double alpha, double beta, cudaStream_t s);
  // Cholesky QR (passes times): Qout B = R, B (upper, S x S row-major) to host
  int cholqr(double* R, double* Qout, double* B_host, int passes, cudaStream_t s, bool* breakdown);
  int random_fill(double* X, int64_t n, uint64_t seed, cudaStream_t s);
  int coldot(const double* A, const double* B, int ncol, double* out_host, cudaStream_t s);
  int axpbypcz(int64_t n, double a, const double* x, double b, double* y, double c, const double* z, cudaStream_t s);
  int resid(const double* U, double* W, const double* lam_dev, cudaStream_t s);
  int panels_to_colmajor(const double* P, int n, double* out, cudaStream_t s);
  // out (nc_pad / S panels) = columns idx[0..nc) of the panel-major block in, zero padded
  int gather_cols(const double* in, const int* idx_dev, int nc, int nc_pad, double* out, cudaStream_t s);
  // F_i = pl_i F_i + G_{pos_i} (pos_i >= 0) or pl_i F_i (pos_i < 0), npan panels of F, G compact
  int scale_add_cols(double* F, const double* G, const int* pos_dev, const double* pl_dev, int npan, cudaStream_t s);
  int ensure(void*& p, size_t& have, size_t need);
  void release();
  ~Dense() { release(); }
};

}  // namespace polfed
