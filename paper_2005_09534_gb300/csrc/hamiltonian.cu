// Matrix-free H~ application and the Clenshaw evaluation of P^K_sigma(H~) X.
//
// Eq. (1) in the S^z = 0 basis: the diagonal is sum_{bonds} J_l Delta z_i z_j
// + sum_i h_i z_i (z = +-1/2) and every antiparallel pair (i, i+l) connects s
// to s ^ (2^i | 2^(i+l)) with amplitude J_l / 2 (Supplement, "Technical
// details": the off-diagonal elements are constants and are never loaded).
// Rescaling (text before Eq. (3)): H~ = alpha (H - beta), alpha = 2/(e_hi - e_lo),
// beta = (e_hi + e_lo)/2.
//
// Ranking.  Split a state into its low b bits s_lo and high L-b bits s_hi.
// With the combinatorial number system, rank(s) = sum_k C(p_k, k+1) over the
// set bits p_0 < p_1 < ...  The low bits contribute T_lo[s_lo] (the rank of
// s_lo among b-bit strings of its popcount) and the high bits T_hi[s_hi]
// (their indices are shifted by popc(s_lo) = L/2 - popc(s_hi)), so
// rank(s) = T_hi[s_hi] + T_lo[s_lo].  All rows with one s_hi form a contiguous
// "group" of C(b, L/2 - popc(s_hi)) rows starting at T_hi[s_hi].
//
// Kernel layout.  A CTA owns one group at a time and stages the group's rows
// of the gather source b1 in shared memory.  A row's neighbours are then
//   - low bonds (both sites in the low part): rows of the same group -> shared memory;
//   - high bonds (both sites high): row T_hi[s_hi'] + local index, i.e. the
//     same local row of another group -> coalesced global reads;
//   - cross bonds (one site in each part): a gather inside a neighbour group.
// Vectors are processed in column slices of 16*LPR bytes (LPR lanes per row,
// 16 bytes per lane), stored slice-major (row stride = slice width).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <type_traits>

#include "polfed_internal.h"

namespace polfed {

// ------------------------------------------------------------- binomials
__constant__ uint32_t c_binom[33][33];
static uint32_t h_binom[33][33];
static std::once_flag h_binom_once;

static void init_binom() {
  std::call_once(h_binom_once, [] {
    memset(h_binom, 0, sizeof(h_binom));
    for (int n = 0; n <= 32; n++) {
      h_binom[n][0] = 1;
      for (int k = 1; k <= n; k++) h_binom[n][k] = h_binom[n - 1][k - 1] + (k <= n - 1 ? h_binom[n - 1][k] : 0);
    }
  });
}

uint32_t binom_host(int n, int k) {
  init_binom();
  if (n < 0 || n > 32 || k < 0 || k > n) return 0;
  return h_binom[n][k];
}

void upload_binomials() {
  init_binom();
  static std::mutex mu;
  static uint64_t done = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && (done >> dev) & 1) return;
  cudaMemcpyToSymbol(c_binom, h_binom, sizeof(h_binom));
  if (dev < 64) done |= (1ull << dev);
}

// -------------------------------------------------------------- geometry
static int choose_b(int L) {
  // >= 2^10 groups at large L (load balance over 152 SMs) and a 128-byte-row
  // group block of at most C(10,5) * 128 B = 32 KB
  int b = L - 10;
  if (const char* e = getenv("POLFED_LOWBITS")) b = atoi(e);
  if (b > 10) b = 10;
  if (b < 2) b = 2;
  if (L - b < 2) b = L - 2;
  return b;
}

int build_geometry(const polfed_model* m, int b_override, HamGeometry* g) {
  if (!m) return fail(POLFED_EINVAL, "model is NULL");
  if (m->L < 4 || m->L > 32 || (m->L & 1)) return fail(POLFED_EINVAL, "L must be even, 4 <= L <= 32");
  if (!m->h) return fail(POLFED_EINVAL, "model.h is NULL");
  memset(g, 0, sizeof(*g));
  const int L = m->L;
  g->L = L;
  g->n_up = L / 2;
  g->periodic = m->periodic ? 1 : 0;
  g->J1 = m->J1;
  g->J2 = m->J2;
  g->Delta = m->Delta;
  for (int i = 0; i < L; i++) {
    if (!std::isfinite(m->h[i])) return fail(POLFED_EINVAL, "non-finite field h_i");
    g->h[i] = m->h[i];
  }
  if (!std::isfinite(m->J1) || !std::isfinite(m->J2) || !std::isfinite(m->Delta))
    return fail(POLFED_EINVAL, "non-finite coupling");
  g->dim = (int64_t)binom_host(L, L / 2);
  int b = b_override > 0 ? b_override : choose_b(L);
  if (b < 2 || L - b < 2) return fail(POLFED_EINVAL, "bad low/high split");
  g->b = b;
  g->nh = L - b;
  // literal terms of Eq. (1): l = 1, 2 and i = 0..L-1 (j = i + l, wrapped if periodic)
  std::vector<Bond> low, high, cross;
  for (int l = 1; l <= 2; l++) {
    double J = (l == 1) ? m->J1 : m->J2;
    if (J == 0.0) continue;
    for (int i = 0; i < L; i++) {
      int j = i + l;
      if (j >= L) {
        if (!g->periodic) continue;
        j -= L;
      }
      Bond bd{std::min(i, j), std::max(i, j), l};
      if (bd.j < b)
        low.push_back(bd);
      else if (bd.i >= b)
        high.push_back(bd);
      else
        cross.push_back(bd);
    }
  }
  auto by_cls = [](const Bond& x, const Bond& y) { return x.cls < y.cls; };
  std::stable_sort(low.begin(), low.end(), by_cls);
  std::stable_sort(high.begin(), high.end(), by_cls);
  if ((int)low.size() > kMaxBonds || (int)high.size() > kMaxBonds || (int)cross.size() > 8)
    return fail(POLFED_EINVAL, "too many bonds for the table layout");
  for (auto& x : low) {
    g->low_mask[g->n_low1 + g->n_low2] = (1u << x.i) | (1u << x.j);
    (x.cls == 1 ? g->n_low1 : g->n_low2)++;
  }
  for (auto& x : high) {
    g->high_mask[g->n_high1 + g->n_high2] = (1u << (x.i - b)) | (1u << (x.j - b));
    (x.cls == 1 ? g->n_high1 : g->n_high2)++;
  }
  for (auto& x : cross) {
    g->cross_lo[g->n_cross] = x.i;
    g->cross_hi[g->n_cross] = x.j - b;
    g->cross_cls[g->n_cross] = x.cls;
    g->n_cross++;
  }
  int off = 0;
  for (int c = 0; c <= b + 1; c++) {
    g->cls_off[c] = off;
    if (c <= b) off += (int)binom_host(b, c);
  }
  {
    const bool j2 = g->n_low2 + g->n_high2 > 0 || m->J2 != 0.0;
    const int maxcr = j2 ? 6 : 2;
    g->rec_stride = j2 ? 32 : 16;
    if (2 + g->n_low1 + g->n_low2 + maxcr > g->rec_stride) return fail(POLFED_EINVAL, "too many low bonds for the record");
    if (g->n_high1 + g->n_high2 > kMaxHigh) return fail(POLFED_EINVAL, "too many high bonds for the group table");
  }
  g->max_group = 0;
  g->n_groups = 0;
  for (int pc = 0; pc <= g->nh; pc++) {
    int n_lo = g->n_up - pc;
    if (n_lo < 0 || n_lo > b) continue;
    g->max_group = std::max(g->max_group, (int)binom_host(b, n_lo));
    g->n_groups += (int)binom_host(g->nh, pc);
  }
  return POLFED_OK;
}

// ------------------------------------------------------------ table kernels
__global__ void k_tables_lo(const HamGeometry g, uint16_t* T_lo, uint16_t* U_lo, double* F_lo) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= (1 << g.b)) return;
  uint32_t r = 0;
  int k = 0;
  for (int p = 0; p < g.b; p++)
    if ((a >> p) & 1) r += c_binom[p][++k];
  T_lo[a] = (uint16_t)r;
  U_lo[g.cls_off[k] + r] = (uint16_t)a;
  double d = 0.0;
  const int nl = g.n_low1 + g.n_low2;
  for (int q = 0; q < nl; q++) {
    const double J = q < g.n_low1 ? g.J1 : g.J2;
    d += J * g.Delta * (__popc(a & g.low_mask[q]) == 1 ? -0.25 : 0.25);
  }
  for (int i = 0; i < g.b; i++) d += g.h[i] * (((a >> i) & 1) ? 0.5 : -0.5);
  F_lo[a] = d;
}

__global__ void k_tables_rec(const HamGeometry g, const uint16_t* T_lo, uint16_t* rec) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= (1 << g.b)) return;
  const int RS = g.rec_stride;
  uint16_t* r = rec + (size_t)(g.cls_off[__popc(a)] + T_lo[a]) * RS;
  for (int e = 0; e < RS; e++) r[e] = 0;
  r[0] = (uint16_t)a;
  int n1 = 0, n2 = 0;
  for (int k = 0; k < g.n_low1; k++) {
    const uint32_t m = g.low_mask[k];
    if (__popc((uint32_t)a & m) == 1) r[2 + n1++] = T_lo[a ^ m];
  }
  for (int k = g.n_low1; k < g.n_low1 + g.n_low2; k++) {
    const uint32_t m = g.low_mask[k];
    if (__popc((uint32_t)a & m) == 1) r[2 + n1 + n2++] = T_lo[a ^ m];
  }
  r[1] = (uint16_t)(n1 | (n2 << 8));
  for (int k = 0; k < g.n_cross; k++) r[RS - 1 - k] = T_lo[a ^ (1 << g.cross_lo[k])];
}

// One-byte copy of the neighbour records (layout in HamTables::rec8).
__global__ void k_tables_rec8(const HamGeometry g, const uint16_t* rec, uint8_t* rec8) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= (1 << g.b)) return;
  const int RS = g.rec_stride;
  const uint16_t* r = rec + (size_t)a * RS;
  uint8_t* o = rec8 + (size_t)a * RS;
  for (int e = 0; e < RS; e++) o[e] = 0;
  const int n1 = r[1] & 0xFF, n2 = r[1] >> 8;
  o[0] = (uint8_t)(r[0] & 0xFF);
  o[1] = (uint8_t)(r[0] >> 8);
  o[2] = (uint8_t)n1;
  o[3] = (uint8_t)n2;
  for (int k = 0; k < n1 + n2; k++) o[4 + k] = (uint8_t)r[2 + k];
  for (int k = 0; k < g.n_cross; k++) o[RS - 1 - k] = (uint8_t)r[RS - 1 - k];
}

// Per-group constants in schedule order.
__global__ void k_tables_groups(const HamGeometry g, const int32_t* T_hi, const int32_t* order, GroupRec* gr) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.n_groups) return;
  const int grp = order[idx];
  GroupRec r;
  const int n_lo = g.n_up - __popc(grp);
  r.r0 = T_hi[grp];
  r.n_g = (int)c_binom[g.b][n_lo];
  r.cls_base = g.cls_off[n_lo];
  int cnt = 0, cnt1 = 0;
  for (int k = 0; k < g.n_high1 + g.n_high2; k++) {
    const uint32_t m = g.high_mask[k];
    if (__popc((uint32_t)grp & m) == 1 && cnt < kMaxHigh) {
      r.hn_base[cnt++] = T_hi[grp ^ m];
      if (k < g.n_high1) cnt1++;
    }
  }
  for (int k = cnt; k < kMaxHigh; k++) r.hn_base[k] = 0;
  r.n_hn = cnt;
  r.n_hn1 = cnt1;
  int need = 0;
  for (int k = 0; k < 8; k++) {
    r.cr_base[k] = 0;
    r.cr_n[k] = 0;
    if (k < g.n_cross) {
      const int hb = (grp >> g.cross_hi[k]) & 1;
      if (!hb) need |= 1 << k;  // the low bit must differ from the high bit
      const int g2 = grp ^ (1 << g.cross_hi[k]);
      const int n_lo2 = g.n_up - __popc(g2);
      // rows with the bond antiparallel exist only if the neighbouring class is valid
      if (T_hi[g2] >= 0 && n_lo2 >= 0 && n_lo2 <= g.b) {
        r.cr_base[k] = T_hi[g2];
        r.cr_n[k] = (int)c_binom[g.b][n_lo2];
      }
    }
  }
  r.need_mask = need;
  r.pad0 = r.pad1 = 0;
  gr[idx] = r;
}

__global__ void k_tables_hi(const HamGeometry g, int32_t* T_hi, double* F_hi) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= (1 << g.nh)) return;
  const int n_lo = g.n_up - __popc(c);
  if (n_lo < 0 || n_lo > g.b) {
    T_hi[c] = -1;
    F_hi[c] = 0.0;
    return;
  }
  uint32_t r = 0;
  int k = 0;
  for (int q = 0; q < g.nh; q++)
    if ((c >> q) & 1) r += c_binom[g.b + q][n_lo + (++k)];
  T_hi[c] = (int32_t)r;
  double d = 0.0;
  const int nhb = g.n_high1 + g.n_high2;
  for (int q = 0; q < nhb; q++) {
    const double J = q < g.n_high1 ? g.J1 : g.J2;
    d += J * g.Delta * (__popc(c & g.high_mask[q]) == 1 ? -0.25 : 0.25);
  }
  for (int i = 0; i < g.nh; i++) d += g.h[g.b + i] * (((c >> i) & 1) ? 0.5 : -0.5);
  F_hi[c] = d;
}

__global__ void k_tables_cx(const HamGeometry g, double* C_x) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (1 << g.n_cross)) return;
  double d = 0.0;
  for (int k = 0; k < g.n_cross; k++) {
    const double J = g.cross_cls[k] == 1 ? g.J1 : g.J2;
    d += J * g.Delta * (((p >> k) & 1) ? -0.25 : 0.25);
  }
  C_x[p] = d;
}

// --------------------------------------------------------- number policies
struct KCf {
  float cX, cH, cB, o1, o2;
};
struct KCd {
  double cX, cH, cB, o1, o2;
};
struct KCdf {
  float2 cX, cH, cB, o1, o2;
  int exact;  // cX, cH, cB are 0 or +-2^k: multiply hi and lo separately (exact)
};

// Float-float arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2.
// two_sum: Knuth (TAOCP vol. 2, 4.2.2); fast_two_sum: Dekker (1971);
// products use the FMA-based exact product error.
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
  float s = a + b;
  float e = b - (s - a);
  return make_float2(s, e);
}
__device__ __forceinline__ float2 two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return make_float2(s, e);
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float2 s = two_sum(a.x, b.x);
  s.y += a.y + b.y;
  return fast_two_sum(s.x, s.y);
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  return fast_two_sum(p, e);
}

struct NF32 {
  using S = float;
  using C = float;
  using A = float;
  using KC = KCf;
  static __device__ __forceinline__ A zero() { return 0.f; }
  static __device__ __forceinline__ void acc(A& a, S v) { a += v; }
  static __device__ __forceinline__ C add3(C a, C b, C c) { return a + b + c; }
  static __device__ __forceinline__ S combine(S xv, S x1, S b2v, A a1, A a2, C ad, const KC& k, bool hx, bool hb,
                                              bool j2, C cx) {
    float y = ad * x1 + k.o1 * a1;
    if (j2) y = fmaf(k.o2, a2, y);
    float r = k.cH * y;
    if (hx) r = fmaf(cx, xv, r);
    if (hb) r = fmaf(k.cB, b2v, r);
    return r;
  }
  // the same combination in two parts: e = cX x + cB b2 when x and b2 arrive,
  // then cH (d x1 + o1 a1 + o2 a2) + e
  static __device__ __forceinline__ S pre(S xv, S b2v, const KC& k, bool hx, bool hb, C cx) {
    float e = hx ? cx * xv : 0.f;
    if (hb) e = fmaf(k.cB, b2v, e);
    return e;
  }
  static __device__ __forceinline__ S fin(S x1, A a1, A a2, C ad, const KC& k, bool j2, S e) {
    float y = ad * x1 + k.o1 * a1;
    if (j2) y = fmaf(k.o2, a2, y);
    return fmaf(k.cH, y, e);
  }
  static __device__ __forceinline__ float mag(S v) { return fabsf(v); }
};

struct NF64 {
  using S = double;
  using C = double;
  using A = double;
  using KC = KCd;
  static __device__ __forceinline__ A zero() { return 0.0; }
  static __device__ __forceinline__ void acc(A& a, S v) { a += v; }
  static __device__ __forceinline__ C add3(C a, C b, C c) { return a + b + c; }
  static __device__ __forceinline__ S combine(S xv, S x1, S b2v, A a1, A a2, C ad, const KC& k, bool hx, bool hb,
                                              bool j2, C cx) {
    double y = ad * x1 + k.o1 * a1;
    if (j2) y = fma(k.o2, a2, y);
    double r = k.cH * y;
    if (hx) r = fma(cx, xv, r);
    if (hb) r = fma(k.cB, b2v, r);
    return r;
  }
  static __device__ __forceinline__ S pre(S xv, S b2v, const KC& k, bool hx, bool hb, C cx) {
    double e = hx ? cx * xv : 0.0;
    if (hb) e = fma(k.cB, b2v, e);
    return e;
  }
  static __device__ __forceinline__ S fin(S x1, A a1, A a2, C ad, const KC& k, bool j2, S e) {
    double y = ad * x1 + k.o1 * a1;
    if (j2) y = fma(k.o2, a2, y);
    return fma(k.cH, y, e);
  }
  static __device__ __forceinline__ float mag(S v) { return (float)fabs(v); }
};

struct NDF {
  using S = float2;  // (hi, lo)
  using C = float2;
  using A = float2;  // (running hi sum, accumulated low parts and rounding errors)
  using KC = KCdf;
  static __device__ __forceinline__ A zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ void acc(A& a, S v) {
    float2 s = two_sum(a.x, v.x);
    a.x = s.x;
    a.y += s.y + v.y;
  }
  static __device__ __forceinline__ C add3(C a, C b, C c) { return df_add(df_add(a, b), c); }
  static __device__ __forceinline__ S combine(S xv, S x1, S b2v, A a1, A a2, C ad, const KC& k, bool hx, bool hb,
                                              bool j2, C cx) {
    float2 y = df_add(df_mul(ad, x1), df_mul(k.o1, fast_two_sum(a1.x, a1.y)));
    if (j2) y = df_add(y, df_mul(k.o2, fast_two_sum(a2.x, a2.y)));
    if (k.exact) {
      float2 r = make_float2(k.cH.x * y.x, k.cH.x * y.y);
      if (hx) r = df_add(r, make_float2(cx.x * xv.x, cx.x * xv.y));
      if (hb) r = df_add(r, make_float2(k.cB.x * b2v.x, k.cB.x * b2v.y));
      return r;
    }
    float2 r = df_mul(k.cH, y);
    if (hx) r = df_add(r, df_mul(cx, xv));
    if (hb) r = df_add(r, df_mul(k.cB, b2v));
    return r;
  }
  static __device__ __forceinline__ S pre(S xv, S b2v, const KC& k, bool hx, bool hb, C cx) {
    float2 e = make_float2(0.f, 0.f);
    if (k.exact) {
      if (hx) e = make_float2(cx.x * xv.x, cx.x * xv.y);
      if (hb) e = df_add(e, make_float2(k.cB.x * b2v.x, k.cB.x * b2v.y));
      return e;
    }
    if (hx) e = df_mul(cx, xv);
    if (hb) e = df_add(e, df_mul(k.cB, b2v));
    return e;
  }
  static __device__ __forceinline__ S fin(S x1, A a1, A a2, C ad, const KC& k, bool j2, S e) {
    float2 y = df_add(df_mul(ad, x1), df_mul(k.o1, fast_two_sum(a1.x, a1.y)));
    if (j2) y = df_add(y, df_mul(k.o2, fast_two_sum(a2.x, a2.y)));
    const float2 r = k.exact ? make_float2(k.cH.x * y.x, k.cH.x * y.y) : df_mul(k.cH, y);
    return df_add(r, e);
  }
  static __device__ __forceinline__ float mag(S v) { return fabsf(v.x); }
};

// cX of the lane's element e: the per-column array (FP32 storage only) or the step's scalar
template <class NT>
__device__ __forceinline__ typename NT::C col_cx(const float* cxcol, int col, const typename NT::KC& kc) {
  if constexpr (std::is_same<NT, NF32>::value) {
    if (cxcol) return __ldg(cxcol + col);
  }
  return kc.cX;
}

template <class S>
union V16 {
  int4 i;
  S s[16 / sizeof(S)];
};

// acc[0..VEC) += the elements of one 16-byte chunk; FP32 uses the packed
// two-wide add of sm_100+ (two additions per instruction, same rounding)
template <class NT>
__device__ __forceinline__ void acc_chunk(typename NT::A* acc, const V16<typename NT::S>& u) {
  if constexpr (std::is_same<NT, NF32>::value) {
    float2 p0 = __fadd2_rn(make_float2(acc[0], acc[1]), make_float2(u.s[0], u.s[1]));
    float2 p1 = __fadd2_rn(make_float2(acc[2], acc[3]), make_float2(u.s[2], u.s[3]));
    acc[0] = p0.x;
    acc[1] = p0.y;
    acc[2] = p1.x;
    acc[3] = p1.y;
  } else {
#pragma unroll
    for (int v = 0; v < (int)(16 / sizeof(typename NT::S)); v++) NT::acc(acc[v], u.s[v]);
  }
}

// ---------------------------------------------------------- the step kernel
struct StepTables {
  const uint16_t* rec;
  const uint8_t* rec8;
  const GroupRec* grec;
  const void* F_lo;  // typed, alpha-scaled
  const void* F_hi;  // typed, alpha-scaled, includes -alpha*beta (indexed by s_hi)
  const void* C_x;   // typed, alpha-scaled
  const int32_t* order;
};

template <bool COH>
__device__ __forceinline__ int4 ld_vec(const int4* p) {
  if constexpr (COH)
    return __ldcg(p);  // L2 only: data written earlier in the same (persistent) launch
  else
    return __ldg(p);
}
template <bool COH>
__device__ __forceinline__ int4 ld_stream(const int4* p) {
  if constexpr (COH)
    return __ldcg(p);
  else
    return __ldcs(p);
}

// One group (rows sharing s_hi) of one Clenshaw / H~ step on a 16*LPR-byte
// column slice, by the CTA's 256 threads (see k_ham_step).  COH selects loads
// that bypass L1, for a persistent kernel whose earlier steps wrote b1 and b2.
template <class NT, int LPR, bool J2, bool COH>
__device__ __forceinline__ void step_group(const int gidx, const int n_cross, const int* cr_lb, const int* cr_c2,
                                           const StepTables& t, const typename NT::S* __restrict__ b1,
                                           const typename NT::S* b2, const typename NT::S* __restrict__ x,
                                           typename NT::S* out, const typename NT::KC& kc, const int has_x,
                                           const int has_b2, typename NT::S* tile, const typename NT::C* sFlo,
                                           const typename NT::C* sCx, const float* cxcol) {
  using S = typename NT::S;
  using C = typename NT::C;
  using A = typename NT::A;
  constexpr int VEC = 16 / sizeof(S);
  constexpr int W = VEC * LPR;
  constexpr int MAXCR = J2 ? 6 : 2;  // cross bonds: (b-1,b), (L-1,0) and, with J2, four more
  constexpr int RS = J2 ? 32 : 16;   // record entries
  constexpr int LOWMAX = RS - 2 - MAXCR;
  constexpr int PCH = J2 ? 2 : 4;    // rows per thread per pass
  constexpr int NT_ = 256;
  constexpr int RSTEP = NT_ / LPR;   // rows between a thread's consecutive rows in a pass
  const int tr = threadIdx.x / LPR, lane = threadIdx.x % LPR;
  const typename NT::C* gFhi = reinterpret_cast<const typename NT::C*>(t.F_hi);
  const GroupRec* G = t.grec + gidx;
  const int r0 = __ldg(&G->r0), n_g = __ldg(&G->n_g), cls_base = __ldg(&G->cls_base);
  const int n_hn = __ldg(&G->n_hn), n_hn1 = __ldg(&G->n_hn1), need = __ldg(&G->need_mask);
  int cr_bs[MAXCR];
#pragma unroll
  for (int k = 0; k < MAXCR; k++) cr_bs[k] = __ldg(&G->cr_base[k]);
  const C fhi = gFhi[t.order[gidx]];
  __syncthreads();  // tables loaded / previous tile fully consumed
  {
    const int4* src = reinterpret_cast<const int4*>(b1 + (size_t)r0 * W);
    int4* dst = reinterpret_cast<int4*>(tile);
    const int nchunk = n_g * LPR;
    for (int c = threadIdx.x; c < nchunk; c += NT_) dst[c] = ld_vec<COH>(src + c);
  }
  __syncthreads();
  for (int p0 = 0; p0 < n_g; p0 += RSTEP * PCH) {
    A a1[PCH][VEC], a2[PCH][VEC];
#pragma unroll
    for (int i = 0; i < PCH; i++)
#pragma unroll
      for (int v = 0; v < VEC; v++) {
        a1[i][v] = NT::zero();
        a2[i][v] = NT::zero();
      }
    // ---- H: high-bond neighbours: the same local rows of another group;
    //      loads of HU neighbours x PCH rows are issued before any is consumed
    constexpr int HU = 2;
    for (int k0 = 0; k0 < n_hn; k0 += HU) {
      V16<S> u[HU][PCH];
#pragma unroll
      for (int j = 0; j < HU; j++) {
        if (k0 + j < n_hn) {
          const int base = __ldg(&G->hn_base[k0 + j]);
#pragma unroll
          for (int i = 0; i < PCH; i++) {
            const int row = p0 + tr + RSTEP * i;
            if (row < n_g)
              u[j][i].i = ld_vec<COH>(reinterpret_cast<const int4*>(b1 + (size_t)(base + row) * W + lane * VEC));
          }
        }
      }
#pragma unroll
      for (int j = 0; j < HU; j++) {
        if (k0 + j < n_hn) {
          const bool c1 = !J2 || k0 + j < n_hn1;
#pragma unroll
          for (int i = 0; i < PCH; i++) {
            const int row = p0 + tr + RSTEP * i;
            if (row < n_g) {
              if (c1) {
#pragma unroll
                for (int v = 0; v < VEC; v++) NT::acc(a1[i][v], u[j][i].s[v]);
              } else {
#pragma unroll
                for (int v = 0; v < VEC; v++) NT::acc(a2[i][v], u[j][i].s[v]);
              }
            }
          }
        }
      }
    }
    // ---- L + C: low bonds (shared memory) and cross bonds (global), LR rows at a time:
    //      records of all LR rows first, then their cross-bond loads, then the gathers
    constexpr int LR = J2 ? 1 : 2;
    uint32_t key[PCH];  // s_lo | cross pattern << 16
#pragma unroll
    for (int i0 = 0; i0 < PCH; i0 += LR) {
      uint32_t rw[LR][RS / 2];
#pragma unroll
      for (int j = 0; j < LR; j++) {
        const int row = p0 + tr + RSTEP * (i0 + j);
        const uint4* rp = reinterpret_cast<const uint4*>(t.rec + (size_t)(cls_base + (row < n_g ? row : 0)) * RS);
#pragma unroll
        for (int q = 0; q < RS / 8; q++) {
          const uint4 v = __ldg(rp + q);
          rw[j][4 * q] = v.x;
          rw[j][4 * q + 1] = v.y;
          rw[j][4 * q + 2] = v.z;
          rw[j][4 * q + 3] = v.w;
        }
      }
#define PF_ENTRY(j, e) ((rw[j][(e) >> 1] >> (((e)&1) * 16)) & 0xFFFFu)
      V16<S> cv[LR][MAXCR];
      uint32_t pat[LR];
#pragma unroll
      for (int j = 0; j < LR; j++) {
        const int row = p0 + tr + RSTEP * (i0 + j);
        const uint32_t s_lo = PF_ENTRY(j, 0);
        pat[j] = 0;
#pragma unroll
        for (int k = 0; k < MAXCR; k++) {
          if (row < n_g && k < n_cross && ((s_lo >> cr_lb[k]) & 1u) == ((need >> k) & 1)) {
            pat[j] |= 1u << k;
            cv[j][k].i = ld_vec<COH>(
                reinterpret_cast<const int4*>(b1 + (size_t)(cr_bs[k] + PF_ENTRY(j, RS - 1 - k)) * W + lane * VEC));
          }
        }
        key[i0 + j] = s_lo | (pat[j] << 16);
      }
#pragma unroll
      for (int j = 0; j < LR; j++) {
        const int i = i0 + j;
        const int row = p0 + tr + RSTEP * i;
        const uint32_t cnt = PF_ENTRY(j, 1);
        const int n1 = row < n_g ? (int)(cnt & 0xFF) : 0;
        const int nl = row < n_g ? n1 + (J2 ? (int)(cnt >> 8) : 0) : 0;
        const int nmax = __reduce_max_sync(0xffffffffu, nl);
#pragma unroll
        for (int k0 = 0; k0 < LOWMAX; k0 += 4) {
          if (k0 >= nmax) break;
          V16<S> u[4];
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const int k = k0 + q;
            if (k < LOWMAX && k < nl)
              u[q].i = *reinterpret_cast<const int4*>(tile + (size_t)PF_ENTRY(j, 2 + k) * W + lane * VEC);
          }
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const int k = k0 + q;
            if (k < LOWMAX && k < nl) {
              if (!J2 || k < n1) {
#pragma unroll
                for (int v = 0; v < VEC; v++) NT::acc(a1[i][v], u[q].s[v]);
              } else {
#pragma unroll
                for (int v = 0; v < VEC; v++) NT::acc(a2[i][v], u[q].s[v]);
              }
            }
          }
        }
#pragma unroll
        for (int k = 0; k < MAXCR; k++) {
          if ((pat[j] >> k) & 1u) {
            if (!J2 || !cr_c2[k]) {
#pragma unroll
              for (int v = 0; v < VEC; v++) NT::acc(a1[i][v], cv[j][k].s[v]);
            } else {
#pragma unroll
              for (int v = 0; v < VEC; v++) NT::acc(a2[i][v], cv[j][k].s[v]);
            }
          }
        }
      }
#undef PF_ENTRY
    }
    // ---- F: diagonal, combination, store (x and b2 loads issued per chunk of rows)
    constexpr int FCH = 2;
#pragma unroll
    for (int i0 = 0; i0 < PCH; i0 += FCH) {
      V16<S> xv[FCH], bv[FCH];
#pragma unroll
      for (int j = 0; j < FCH; j++) {
        const int row = p0 + tr + RSTEP * (i0 + j);
        if (row < n_g) {
          const size_t off = (size_t)(r0 + row) * W + lane * VEC;
          if (has_x) xv[j].i = ld_stream<COH>(reinterpret_cast<const int4*>(x + off));
          if (has_b2) bv[j].i = ld_stream<COH>(reinterpret_cast<const int4*>(b2 + off));
        }
      }
#pragma unroll
      for (int j = 0; j < FCH; j++) {
        const int i = i0 + j;
        const int row = p0 + tr + RSTEP * i;
        if (row < n_g) {
          const size_t off = (size_t)(r0 + row) * W + lane * VEC;
          const uint32_t s_lo = key[i] & 0xFFFFu, pattern = key[i] >> 16;
          const C ad = NT::add3(sFlo[s_lo], fhi, sCx[pattern]);
          V16<S> xo, res;
          xo.i = *reinterpret_cast<const int4*>(tile + (size_t)row * W + lane * VEC);
#pragma unroll
          for (int v = 0; v < VEC; v++)
            res.s[v] = NT::combine(has_x ? xv[j].s[v] : S(), xo.s[v], has_b2 ? bv[j].s[v] : S(), a1[i][v],
                                   a2[i][v], ad, kc, has_x, has_b2, J2, col_cx<NT>(cxcol, lane * VEC + v, kc));
          __stcg(reinterpret_cast<int4*>(out + off), res.i);
        }
      }
    }
  }
}

// One Clenshaw / H~ step on a 16*LPR-byte column slice:
//   out = cX * x + cH * (H~ b1) + cB * b2     (row-major slice buffers, ld = W)
// A CTA takes groups in schedule order; a group's rows of b1 are staged in
// shared memory, then rows are processed in passes of PCH rows per thread:
//   H: whole neighbouring-group blocks (high bonds) streamed with coalesced loads,
//   L: low-bond neighbours gathered from the staged rows (compact per-row record),
//   C: cross-bond neighbours gathered from global memory,
//   F: diagonal, combination with x and b2, store.
template <class NT, int LPR, bool J2>
__global__ void __launch_bounds__(256, 2) k_ham_step(const HamGeometry g, const StepTables t,
                                                      const typename NT::S* __restrict__ b1,
                                                      const typename NT::S* b2, const typename NT::S* __restrict__ x,
                                                      typename NT::S* out, const typename NT::KC kc, int has_x,
                                                      int has_b2, const float* cxcol) {
  using S = typename NT::S;
  using C = typename NT::C;
  using A = typename NT::A;
  constexpr int VEC = 16 / sizeof(S);
  constexpr int W = VEC * LPR;
  constexpr int MAXCR = J2 ? 6 : 2;  // cross bonds: (b-1,b), (L-1,0) and, with J2, four more
  constexpr int RS = J2 ? 32 : 16;   // record entries
  constexpr int LOWMAX = RS - 2 - MAXCR;
  constexpr int PCH = J2 ? 2 : 4;    // rows per thread per pass
  constexpr int NT_ = 256;
  constexpr int RSTEP = NT_ / LPR;   // rows between a thread's consecutive rows in a pass

  extern __shared__ __align__(16) unsigned char smem[];
  const int nlo_tab = 1 << g.b;
  S* tile = reinterpret_cast<S*>(smem);
  C* sFlo = reinterpret_cast<C*>(smem + (size_t)g.max_group * W * sizeof(S));
  C* sCx = sFlo + nlo_tab;

  const C* gFlo = reinterpret_cast<const C*>(t.F_lo);
  const C* gCx = reinterpret_cast<const C*>(t.C_x);
  for (int i = threadIdx.x; i < nlo_tab; i += NT_) sFlo[i] = gFlo[i];
  for (int i = threadIdx.x; i < (1 << g.n_cross); i += NT_) sCx[i] = gCx[i];

  int cr_lb[MAXCR], cr_c2[MAXCR];
#pragma unroll
  for (int k = 0; k < MAXCR; k++) {
    cr_lb[k] = k < g.n_cross ? g.cross_lo[k] : 0;
    cr_c2[k] = k < g.n_cross && g.cross_cls[k] == 2;
  }

  for (int gidx = blockIdx.x; gidx < g.n_groups; gidx += gridDim.x)
    step_group<NT, LPR, J2, false>(gidx, g.n_cross, cr_lb, cr_c2, t, b1, b2, x, out, kc, has_x, has_b2, tile, sFlo,
                                   sCx, cxcol);
}

// -------------------------------------------------------- bounded waits
// Iteration caps of the device-side waits: the TMA pipeline's mbarrier waits
// and the batched kernel's grid barrier.  A wait that runs out makes the
// kernel stop, drain the copies it issued (always with the full cap) and
// report POLFED_ETIMEOUT.  polfed_set_wait_limit lowers the caps for tests.
constexpr uint32_t kMbarWaitPolls = 1u << 22;
constexpr uint32_t kBarrierWaitPolls = 1u << 24;
static std::atomic<uint32_t> g_wait_limit{0};
static uint32_t wait_cap(uint32_t dflt) {
  const uint32_t v = g_wait_limit.load();
  return v == 0 ? dflt : std::min(v, dflt);
}

// ------------------------------------------------ batched persistent filter
// Many independent filter jobs -- one 128-byte column slice of one disorder
// realization each, with its own operator tables, order K and coefficients --
// advance through their Clenshaw steps inside ONE cooperative launch.  Launch
// step st performs step st of every job with st < K_j (Clenshaw index
// k = K_j - 1 - st): the CTAs share out the groups of all active jobs in a
// fixed order, then meet at a grid barrier.  The barrier's waits are bounded;
// a wait that runs out sets *err and every CTA leaves at its next barrier.
struct BatchJob {
  StepTables t;
  const double* coef;  // c_0..c_K of the job (device, FP64)
  void* xs;            // slice buffers (dim x W, storage type of the kernel)
  void* ba;
  void* bb;
  double invD, o1, o2;
  int K, n_groups, n_cross, nlo_tab;
  int cross_lo[6], cross_cls[6];
};

__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, int* err, uint32_t cap) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    const unsigned g0 = *(volatile unsigned*)gen;
    __threadfence();
    const unsigned arrived = atomicAdd(count, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      uint32_t it = 0;
      while (*(volatile unsigned*)gen == g0) {
        if (*(volatile int*)err) {
          ok = 0;
          break;
        }
        if (++it > cap) {  // default 2^24: about a second of 32-64 ns naps
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  return __syncthreads_and(ok) != 0;
}

template <class NT>
__device__ __forceinline__ void make_kc(double cX, double cH, double cB, double o1, double o2, typename NT::KC& kc) {
  if constexpr (std::is_same<NT, NDF>::value) {
    auto split = [](double v) {
      const float hi = (float)v;
      return make_float2(hi, (float)(v - (double)hi));
    };
    auto p2 = [](double v) {
      if (v == 0.0) return true;
      int e = 0;
      const double m = frexp(fabs(v), &e);
      return m == 0.5 && e > -120 && e < 120;
    };
    kc.cX = split(cX);
    kc.cH = split(cH);
    kc.cB = split(cB);
    kc.o1 = split(o1);
    kc.o2 = split(o2);
    kc.exact = p2(cX) && p2(cH) && p2(cB);
  } else {
    using C = typename NT::C;
    kc.cX = (C)cX;
    kc.cH = (C)cH;
    kc.cB = (C)cB;
    kc.o1 = (C)o1;
    kc.o2 = (C)o2;
  }
}

template <class NT, bool J2>
__global__ void __launch_bounds__(256, 2)
    k_filter_batched(const BatchJob* __restrict__ jobs, int n_jobs, int n_steps, int tile_elems, int nlo_max,
                     unsigned* bar_count, unsigned* bar_gen, int* err, uint32_t wait_cap) {
  using S = typename NT::S;
  using C = typename NT::C;
  constexpr int LPR = 8;
  constexpr int MAXCR = J2 ? 6 : 2;
  extern __shared__ __align__(16) unsigned char smem[];
  S* tile = reinterpret_cast<S*>(smem);
  C* sFlo = reinterpret_cast<C*>(smem + (size_t)tile_elems * sizeof(S));
  C* sCx = sFlo + nlo_max;
  int loaded = -1, n_cross = 0;
  int cr_lb[MAXCR], cr_c2[MAXCR];
  const int G = gridDim.x;
  for (int st = 0; st < n_steps; st++) {
    int base = 0;
    for (int j = 0; j < n_jobs; j++) {
      const int K = jobs[j].K;
      if (st >= K) continue;
      const int ng = jobs[j].n_groups;
      for (int w = base + (int)((blockIdx.x + G - (unsigned)base % G) % G); w < base + ng; w += G) {
        const BatchJob& J = jobs[j];
        if (loaded != j) {
          __syncthreads();  // the previous job's tables and tile are no longer read
          const C* gFlo = reinterpret_cast<const C*>(J.t.F_lo);
          const C* gCx = reinterpret_cast<const C*>(J.t.C_x);
          for (int i = threadIdx.x; i < J.nlo_tab; i += 256) sFlo[i] = gFlo[i];
          for (int i = threadIdx.x; i < (1 << J.n_cross); i += 256) sCx[i] = gCx[i];
          n_cross = J.n_cross;
#pragma unroll
          for (int k = 0; k < MAXCR; k++) {
            cr_lb[k] = k < n_cross ? J.cross_lo[k] : 0;
            cr_c2[k] = k < n_cross && J.cross_cls[k] == 2;
          }
          loaded = j;
        }
        const int kk = K - 1 - st;
        S* cur = reinterpret_cast<S*>((st & 1) ? J.bb : J.ba);  // b_{k+1}
        S* oth = reinterpret_cast<S*>((st & 1) ? J.ba : J.bb);  // b_{k+2}, overwritten by b_k
        typename NT::KC kc;
        double cX, cH, cB;
        if (kk >= 1) {
          cX = J.coef[kk];
          cH = 2.0;
          cB = (kk == K - 1) ? 0.0 : -1.0;
        } else {  // Y = (c_0 X + H~ b_1 - b_2) / D
          cX = J.coef[0] * J.invD;
          cH = J.invD;
          cB = (K == 1) ? 0.0 : -J.invD;
        }
        make_kc<NT>(cX, cH, cB, J.o1, J.o2, kc);
        step_group<NT, LPR, J2, true>(w - base, n_cross, cr_lb, cr_c2, J.t, cur, oth,
                                      reinterpret_cast<const S*>(J.xs), oth, kc, cX != 0.0, cB != 0.0, tile, sFlo,
                                      sCx, nullptr);
      }
      base += ng;
    }
    if (!grid_barrier(bar_count, bar_gen, err, wait_cap)) return;
  }
}

// ------------------------------------------------- TMA-pipelined step kernel
// The same step for 128-byte slices with whole groups moved by the bulk-copy
// (TMA) engine: a persistent CTA per SM takes groups in schedule order; the
// group's own rows of b1 are fetched into a double-buffered shared tile, and
// the neighbouring groups' blocks reached through high bonds stream through a
// NSTAGE-deep shared ring (mbarrier completion, bounded waits).  Each thread
// owns up to RPT rows (8 lanes of 16 bytes per row); x and b2 rows are loaded
// into registers when the group starts and consumed at the end.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false if the phase did not complete within the iteration cap
// or another thread already gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, uint32_t cap) {
  for (uint32_t it = 0; it < cap; ++it) {
    if (mbar_try_wait(b, parity)) return true;
    if (*abort_flag) return false;
  }
  return false;
}

// Shapes of the kernel: CW consumer warps (plus the producer warp), LPR lanes
// per 128-byte row (4: two 16-byte chunks per lane; 8: one chunk per lane),
// RPT rows per lane, RPT * 32 CW / LPR >= C(10, 5) = 252 rows (the largest group).
template <int CW_, int LPR_>
struct TmaShape {
  static constexpr int CW = CW_;
  static constexpr int LPR = LPR_;
  static constexpr int THREADS = 32 * (CW + 1);  // warp 0 issues the copies
  static constexpr int UNITS = 32 * CW / LPR;
  static constexpr int RPT = (252 + UNITS - 1) / UNITS;
};
// 544 threads, 2 rows of 2 chunks per lane.  Measured on GB300 (L = 22 XXZ and
// L = 20 J1-J2 slices, FP32 and float-float): 24 consumer warps with one chunk
// per lane (800 threads) and 16 warps with four chunks per lane (one row each)
// were 4-25% slower.
using TmaShapeA = TmaShape<16, 4>;
__host__ __device__ constexpr int tma_stages(bool j2) { return j2 ? 3 : 4; }
// int4 words of GroupRec::hn_base the producer reads: up to 16 (XXZ) or 28 (J1-J2) high neighbours
__host__ __device__ constexpr int tma_high_words(bool j2) { return j2 ? 7 : 4; }

template <class NT, bool J2, class SH>
__global__ void __launch_bounds__(SH::THREADS, 1)
    k_ham_step_tma(const HamGeometry g, const StepTables t, const typename NT::S* __restrict__ b1,
                   const typename NT::S* b2, const typename NT::S* __restrict__ x, typename NT::S* out,
                   const typename NT::KC kc, int has_x, int has_b2, int* err, uint32_t wait_cap,
                   const float* cxcol) {
  using S = typename NT::S;
  using C = typename NT::C;
  using A = typename NT::A;
  constexpr int LPR = SH::LPR;          // lanes per 128-byte row
  constexpr int VEC = 16 / sizeof(S);   // elements per 16-byte chunk
  constexpr int NCH = 8 / LPR;          // 16-byte chunks per lane
  constexpr int W = 8 * VEC;            // elements per 128-byte row
  constexpr int VL = NCH * VEC;         // elements per lane
  constexpr int MAXCR = J2 ? 6 : 2;
  constexpr int RS = J2 ? 32 : 16;  // bytes per record
  constexpr int LOWMAX = RS - 4 - MAXCR;
  constexpr int NS = tma_stages(J2);
  constexpr int RPT = SH::RPT;
  constexpr int UNITS = SH::UNITS;
  constexpr int kThreads = SH::THREADS;
  constexpr int kConsumerWarps = SH::CW;

  extern __shared__ __align__(128) unsigned char smem[];
  const size_t stg = (size_t)g.max_group * W;  // elements per stage
  S* own = reinterpret_cast<S*>(smem);         // [2][stg]
  S* ring = own + 2 * stg;                     // [NS][stg]
  uint8_t* sRec = reinterpret_cast<uint8_t*>(ring + NS * stg);  // [2^b][RS] one-byte neighbour records
  C* sFlo = reinterpret_cast<C*>(sRec + ((size_t)RS << g.b));
  C* sCx = sFlo + (1 << g.b);
  __shared__ __align__(8) uint64_t own_full[2], own_empty[2], full[NS], empty[NS];
  __shared__ __align__(16) GroupRec s_grp[2];  // constants of the group in each own buffer
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane32 = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < 2; i++) {
      mbar_init(&own_full[i], 1);
      mbar_init(&own_empty[i], kConsumerWarps);
    }
    for (int i = 0; i < NS; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kConsumerWarps);
    }
    s_abort = 0;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  {
    const uint4* src = reinterpret_cast<const uint4*>(t.rec8);
    uint4* dst = reinterpret_cast<uint4*>(sRec);
    const int n16 = (RS << g.b) / 16;
    for (int i = tid; i < n16; i += kThreads) dst[i] = __ldg(src + i);
    const C* gFlo = reinterpret_cast<const C*>(t.F_lo);
    const C* gCx = reinterpret_cast<const C*>(t.C_x);
    for (int i = tid; i < (1 << g.b); i += kThreads) sFlo[i] = gFlo[i];
    for (int i = tid; i < (1 << g.n_cross); i += kThreads) sCx[i] = gCx[i];
  }
  __syncthreads();
  const int n_my = (g.n_groups - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const size_t esz = sizeof(S);

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane32 == 0) {
      // The producer is one thread and its issue rate bounds the kernel: the
      // group's fields come in a few vector loads (the next record is
      // prefetched into L1 a group ahead), the item loops are unrolled over
      // the static bond counts, and ring slots and phases are tracked with
      // counters instead of divisions.
      int q = 0;        // ring items issued
      int slot = 0;     // q % NS
      uint32_t ph = 0;  // bit s: parity of the next empty-phase wait on slot s
      int n_own = 0;    // own tiles issued
      bool ok = true;
      constexpr int HN4 = tma_high_words(J2);  // int4 words of hn_base read
      auto issue = [&](const S* src, int rows) -> bool {
        if (q >= NS) {
          const uint32_t par = (ph >> slot) & 1u;
          if (!mbar_try_wait(&empty[slot], par) && !mbar_wait(&empty[slot], par, &s_abort, wait_cap)) return false;
          ph ^= 1u << slot;
        }
        const uint32_t bytes = (uint32_t)rows * (uint32_t)(W * esz);
        mbar_expect_tx(&full[slot], bytes);
        bulk_load(ring + (size_t)slot * stg, src, bytes, &full[slot]);
        q++;
        slot = (slot + 1 == NS) ? 0 : slot + 1;
        return true;
      };
      for (int ord = 0; ord < n_my && ok; ord++) {
        const GroupRec* G = t.grec + (int)blockIdx.x + ord * (int)gridDim.x;
        if (ord + 1 < n_my) {
          const char* nx = reinterpret_cast<const char*>(G + gridDim.x);
          asm volatile("prefetch.global.L1 [%0];" ::"l"(nx));
          asm volatile("prefetch.global.L1 [%0];" ::"l"(nx + 128));
        }
        const int4* G4 = reinterpret_cast<const int4*>(G);
        const int4 w0 = __ldg(G4), w1 = __ldg(G4 + 1);
        int4 hw[HN4];
#pragma unroll
        for (int j = 0; j < HN4; j++) hw[j] = __ldg(G4 + 2 + j);
        const int4 cb0 = __ldg(G4 + 10), cn0 = __ldg(G4 + 12);
        int4 cb1 = make_int4(0, 0, 0, 0), cn1 = make_int4(0, 0, 0, 0);
        if constexpr (J2) {
          cb1 = __ldg(G4 + 11);
          cn1 = __ldg(G4 + 13);
        }
        const int r0 = w0.x, n_g = w0.y, n_hn = w1.x;
        if (ord >= 2 && !mbar_wait(&own_empty[ord & 1], (uint32_t)(((ord >> 1) - 1) & 1), &s_abort, wait_cap)) {
          ok = false;
          break;
        }
        {
          const uint32_t bytes = (uint32_t)((size_t)n_g * W * esz);
          mbar_expect_tx(&own_full[ord & 1], bytes + (uint32_t)sizeof(GroupRec));
          bulk_load(&s_grp[ord & 1], G, (uint32_t)sizeof(GroupRec), &own_full[ord & 1]);
          bulk_load(own + (size_t)(ord & 1) * stg, b1 + (size_t)r0 * W, bytes, &own_full[ord & 1]);
          n_own++;
        }
        // items: x, b2 (consumed first and released at once), cross blocks, high blocks
        if (has_x && !issue(x + (size_t)r0 * W, n_g)) {
          ok = false;
          break;
        }
        if (has_b2 && !issue(b2 + (size_t)r0 * W, n_g)) {
          ok = false;
          break;
        }
        const int cbase[8] = {cb0.x, cb0.y, cb0.z, cb0.w, cb1.x, cb1.y, cb1.z, cb1.w};
        const int cnum[8] = {cn0.x, cn0.y, cn0.z, cn0.w, cn1.x, cn1.y, cn1.z, cn1.w};
#pragma unroll
        for (int k = 0; k < MAXCR; k++)
          if (ok && k < g.n_cross && cnum[k] > 0 && !issue(b1 + (size_t)cbase[k] * W, cnum[k])) ok = false;
        if (!ok) break;
#pragma unroll
        for (int j = 0; j < HN4; j++) {
          const int hb[4] = {hw[j].x, hw[j].y, hw[j].z, hw[j].w};
#pragma unroll
          for (int u = 0; u < 4; u++)
            if (ok && 4 * j + u < n_hn && !issue(b1 + (size_t)hb[u] * W, n_g)) ok = false;
        }
        if (!ok) break;
      }
      if (!ok) {
        s_abort = 1;
        atomicExch(err, 1);
      }
      // every copy already issued must land before the CTA may exit: wait for
      // the last phase of each buffer that received one (bounded; a drain that
      // runs out of polls is reported as a timeout, so the output is discarded)
      bool drained = true;
      for (int sl = 0; sl < NS; sl++) {
        const int uses = q > sl ? (q - 1 - sl) / NS + 1 : 0;
        if (uses > 0) {
          bool landed = false;
          for (uint32_t i = 0; i < kMbarWaitPolls && !landed; ++i) landed = mbar_try_wait(&full[sl], (uint32_t)((uses - 1) & 1));
          drained = drained && landed;
        }
      }
      for (int b = 0; b < 2; b++) {
        const int uses = n_own > b ? (n_own - 1 - b) / 2 + 1 : 0;
        if (uses > 0) {
          bool landed = false;
          for (uint32_t i = 0; i < kMbarWaitPolls && !landed; ++i)
            landed = mbar_try_wait(&own_full[b], (uint32_t)((uses - 1) & 1));
          drained = drained && landed;
        }
      }
      if (!drained) {
        s_abort = 1;
        atomicExch(err, 1);
      }
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  const int ctid = tid - 32;
  const int unit = ctid / LPR, lane = ctid % LPR;
  // the 16-byte chunks of a lane (element offsets in the row); with two chunks
  // they are ordered so that the two rows read by a quarter-warp fall on
  // disjoint shared-memory banks
  int chk[NCH];
  if constexpr (NCH == 2) {
    chk[0] = (lane + 4 * (unit & 1)) * VEC;
    chk[1] = (lane + 4 * (1 - (unit & 1))) * VEC;
  } else {
    // a lane's NCH chunks are adjacent; their order rotates with the row unit,
    // so the NCH-row phases of a warp read NCH different bank groups
#pragma unroll
    for (int h = 0; h < NCH; h++) chk[h] = (lane * NCH + ((h + unit) % NCH)) * VEC;
  }

  const C* gFhi = reinterpret_cast<const C*>(t.F_hi);
  int cr_lb[MAXCR], cr_c2[MAXCR];
#pragma unroll
  for (int k = 0; k < MAXCR; k++) {
    cr_lb[k] = k < g.n_cross ? g.cross_lo[k] : 0;
    cr_c2[k] = k < g.n_cross && g.cross_cls[k] == 2;
  }
  // accumulate the lane's chunks of row `row` of buffer `p` into acc
  auto acc2 = [&](A* acc, const S* p, size_t row) {
    V16<S> u[NCH];
#pragma unroll
    for (int h = 0; h < NCH; h++) u[h].i = *reinterpret_cast<const int4*>(p + row * W + chk[h]);
#pragma unroll
    for (int h = 0; h < NCH; h++) acc_chunk<NT>(acc + h * VEC, u[h]);
  };
  int q = 0;  // ring items consumed
  C fhi_next = gFhi[blockIdx.x];  // diagonal constant of the group, schedule order (prefetched)
  for (int ord = 0; ord < n_my; ord++) {
    const int gidx = (int)blockIdx.x + ord * (int)gridDim.x;
    const C fhi = fhi_next;
    if (ord + 1 < n_my) fhi_next = gFhi[gidx + (int)gridDim.x];
    if (!mbar_wait(&own_full[ord & 1], (uint32_t)((ord >> 1) & 1), &s_abort, wait_cap)) s_abort = 1;
    if (s_abort) break;
    const GroupRec* G = &s_grp[ord & 1];
    const int r0 = G->r0, n_g = G->n_g, cls_base = G->cls_base;
    const int n_hn = G->n_hn, n_hn1 = G->n_hn1, need = G->need_mask;
    const S* tile = own + (size_t)(ord & 1) * stg;
    // ---- x and b2 (the group's first ring items): e = cX x + cB b2, then both slots are free
    S e[RPT][VL];
    {
      int x_slot = -1, b2_slot = -1;
      if (has_x) {
        x_slot = q % NS;
        if (!mbar_wait(&full[x_slot], (uint32_t)((q / NS) & 1), &s_abort, wait_cap)) s_abort = 1;
        q++;
      }
      if (has_b2 && !s_abort) {
        b2_slot = q % NS;
        if (!mbar_wait(&full[b2_slot], (uint32_t)((q / NS) & 1), &s_abort, wait_cap)) s_abort = 1;
        q++;
      }
      if (s_abort) break;
#pragma unroll
      for (int i = 0; i < RPT; i++) {
        const int row = unit + UNITS * i;
#pragma unroll
        for (int h = 0; h < NCH; h++) {
          V16<S> xv, bv;
          const size_t lo = (size_t)(row < n_g ? row : 0) * W + chk[h];
          if (has_x) xv.i = *reinterpret_cast<const int4*>(ring + (size_t)x_slot * stg + lo);
          if (has_b2) bv.i = *reinterpret_cast<const int4*>(ring + (size_t)b2_slot * stg + lo);
#pragma unroll
          for (int v = 0; v < VEC; v++)
            e[i][h * VEC + v] = NT::pre(has_x ? xv.s[v] : S(), has_b2 ? bv.s[v] : S(), kc, has_x, has_b2,
                                        col_cx<NT>(cxcol, chk[h] + v, kc));
        }
      }
      __syncwarp();
      if (lane32 == 0) {
        if (x_slot >= 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[x_slot])) : "memory");
        if (b2_slot >= 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[b2_slot])) : "memory");
      }
    }
    A a1[RPT][VL], a2[RPT][VL];
#pragma unroll
    for (int i = 0; i < RPT; i++)
#pragma unroll
      for (int v = 0; v < VL; v++) {
        a1[i][v] = NT::zero();
        a2[i][v] = NT::zero();
      }
    uint32_t key[RPT];  // s_lo | cross pattern << 16
    // ---- low bonds: gathers from the staged rows, neighbour lists from the record table
#pragma unroll
    for (int i = 0; i < RPT; i++) {
      const int row = unit + UNITS * i;
      const bool live = row < n_g;
      const uint8_t* r = sRec + (size_t)(cls_base + (live ? row : 0)) * RS;
      uint32_t rw[RS / 4];
#pragma unroll
      for (int qq = 0; qq < RS / 16; qq++) {
        const uint4 v = reinterpret_cast<const uint4*>(r)[qq];
        rw[4 * qq] = v.x;
        rw[4 * qq + 1] = v.y;
        rw[4 * qq + 2] = v.z;
        rw[4 * qq + 3] = v.w;
      }
#define PF_E(e) ((rw[(e) >> 2] >> (((e)&3) * 8)) & 0xFFu)
      const uint32_t s_lo = rw[0] & 0xFFFFu;
      const int n1 = live ? (int)PF_E(2) : 0;
      const int nl = live ? n1 + (J2 ? (int)PF_E(3) : 0) : 0;
      uint32_t pattern = 0;
#pragma unroll
      for (int k = 0; k < MAXCR; k++)
        if (live && k < g.n_cross && ((s_lo >> cr_lb[k]) & 1u) == ((need >> k) & 1)) pattern |= 1u << k;
      key[i] = s_lo | (pattern << 16);
      const int nmax = __reduce_max_sync(0xffffffffu, nl);
#pragma unroll
      for (int k0 = 0; k0 < LOWMAX; k0 += 2) {
        if (k0 >= nmax) break;
        V16<S> u[2][NCH];
#pragma unroll
        for (int j = 0; j < 2; j++) {
          const int k = k0 + j;
          if (k < LOWMAX && k < nl) {
            const size_t rr = (size_t)PF_E(4 + k) * W;
#pragma unroll
            for (int h = 0; h < NCH; h++) u[j][h].i = *reinterpret_cast<const int4*>(tile + rr + chk[h]);
          }
        }
#pragma unroll
        for (int j = 0; j < 2; j++) {
          const int k = k0 + j;
          if (k < LOWMAX && k < nl) {
            A* acc = (!J2 || k < n1) ? a1[i] : a2[i];
#pragma unroll
            for (int h = 0; h < NCH; h++) acc_chunk<NT>(acc + h * VEC, u[j][h]);
          }
        }
      }
#undef PF_E
    }
    // ---- ring items in the producer's order: cross blocks, high blocks
    for (int k = 0; k < MAXCR; k++) {
      if (!(k < g.n_cross && G->cr_n[k] > 0)) continue;
      const int slot = q % NS;
      if (!mbar_wait(&full[slot], (uint32_t)((q / NS) & 1), &s_abort, wait_cap)) s_abort = 1;
      if (s_abort) break;
      const S* blk = ring + (size_t)slot * stg;
      const bool c1 = !J2 || !cr_c2[k];
#pragma unroll
      for (int i = 0; i < RPT; i++) {
        if ((key[i] >> (16 + k)) & 1u) {
          const int row = unit + UNITS * i;
          const uint8_t* r = sRec + (size_t)(cls_base + row) * RS;
          acc2(c1 ? a1[i] : a2[i], blk, r[RS - 1 - k]);
        }
      }
      __syncwarp();
      if (lane32 == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[slot])) : "memory");
      q++;
    }
    if (s_abort) break;
    for (int k = 0; k < n_hn; k++) {
      const int slot = q % NS;
      if (!mbar_wait(&full[slot], (uint32_t)((q / NS) & 1), &s_abort, wait_cap)) s_abort = 1;
      if (s_abort) break;
      const S* blk = ring + (size_t)slot * stg;
      const bool c1 = !J2 || k < n_hn1;
#pragma unroll
      for (int i = 0; i < RPT; i++) {
        const int row = unit + UNITS * i;
        if (row < n_g) acc2(c1 ? a1[i] : a2[i], blk, row);
      }
      __syncwarp();
      if (lane32 == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[slot])) : "memory");
      q++;
    }
    if (s_abort) break;
    // ---- diagonal, combination, store
#pragma unroll
    for (int i = 0; i < RPT; i++) {
      const int row = unit + UNITS * i;
      if (row < n_g) {
        const uint32_t s_lo = key[i] & 0xFFFFu, pattern = key[i] >> 16;
        const C ad = NT::add3(sFlo[s_lo], fhi, sCx[pattern]);
#pragma unroll
        for (int h = 0; h < NCH; h++) {
          const size_t lo = (size_t)row * W + chk[h];
          V16<S> xo, res;
          xo.i = *reinterpret_cast<const int4*>(tile + lo);
#pragma unroll
          for (int v = 0; v < VEC; v++)
            res.s[v] = NT::fin(xo.s[v], a1[i][h * VEC + v], a2[i][h * VEC + v], ad, kc, J2, e[i][h * VEC + v]);
          __stcg(reinterpret_cast<int4*>(out + (size_t)(r0 + row) * W + chk[h]), res.i);
        }
      }
    }
    __syncwarp();
    if (lane32 == 0)
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&own_empty[ord & 1])) : "memory");
  }
  if (s_abort && ctid == 0) atomicExch(err, 1);
}

// ------------------------------------------------------ slice conversions
template <class NT>
struct Conv;
template <>
struct Conv<NF32> {
  static __device__ __forceinline__ float from_d(double v) { return (float)v; }
  static __device__ __forceinline__ float from_f(float v) { return v; }
  static __device__ __forceinline__ double to_d(float v) { return (double)v; }
  static __device__ __forceinline__ float to_f(float v) { return v; }
  static __device__ __forceinline__ float mul(float c, float v) { return c * v; }
  static __device__ __forceinline__ float zero() { return 0.f; }
};
template <>
struct Conv<NF64> {
  static __device__ __forceinline__ double from_d(double v) { return v; }
  static __device__ __forceinline__ double from_f(float v) { return (double)v; }
  static __device__ __forceinline__ double to_d(double v) { return v; }
  static __device__ __forceinline__ float to_f(double v) { return (float)v; }
  static __device__ __forceinline__ double mul(double c, double v) { return c * v; }
  static __device__ __forceinline__ double zero() { return 0.0; }
};
template <>
struct Conv<NDF> {
  static __device__ __forceinline__ float2 from_d(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
  }
  static __device__ __forceinline__ float2 from_f(float v) { return make_float2(v, 0.f); }
  static __device__ __forceinline__ double to_d(float2 v) { return (double)v.x + (double)v.y; }
  static __device__ __forceinline__ float to_f(float2 v) { return v.x + v.y; }
  static __device__ __forceinline__ float2 mul(float2 c, float2 v) { return df_mul(c, v); }
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
};

template <class NT>
__device__ __forceinline__ typename NT::C col_cx_scale(const float* colscale, int c, typename NT::C cscale) {
  if constexpr (std::is_same<NT, NF32>::value) {
    if (colscale) return colscale[c];
  }
  return cscale;
}

// Load columns [col0, col0+ncols) of a row-major ABI block (ld elements per
// row) into a slice buffer (zero padded to W columns), optionally also write a
// scaled copy and a zero buffer; records max |x| in flag[0] (as float bits).
template <class NT, class In>
__global__ void k_slice_in(const In* __restrict__ in, int64_t dim, int ld, int col0, int ncols, int W,
                           typename NT::S* xs, typename NT::S* a_scaled, typename NT::S* zero_buf,
                           typename NT::C cscale, float* flag, const float* colscale) {
  using S = typename NT::S;
  float mx = 0.f;
  const int64_t n = dim * W;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / W;
    const int c = (int)(e - r * W);
    S v;
    if (c < ncols) {
      const In raw = in[r * ld + col0 + c];
      if constexpr (sizeof(In) == 4) {
        v = Conv<NT>::from_f(raw);
        mx = fmaxf(mx, fabsf(raw));
      } else {
        v = Conv<NT>::from_d(raw);
        mx = fmaxf(mx, (float)fabs(raw));
      }
    } else {
      v = Conv<NT>::zero();
    }
    if (xs) xs[e] = v;
    if (a_scaled) a_scaled[e] = Conv<NT>::mul(col_cx_scale<NT>(colscale, c, cscale), v);
    if (zero_buf) zero_buf[e] = Conv<NT>::zero();
  }
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && flag) atomicMax(reinterpret_cast<int*>(flag), __float_as_int(mx));
}

// Slice buffer -> columns of a row-major ABI block; records max |y| in flag[1]
// and sets flag[2] (int) to 1 on a non-finite value.
template <class NT, class Out>
__global__ void k_slice_out(const typename NT::S* __restrict__ ys, int64_t dim, int W, int ncols, Out* out, int ld,
                            int col0, float* flag) {
  float mx = 0.f;
  int bad = 0;
  const int64_t n = dim * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ncols;
    const int c = (int)(e - r * ncols);
    const typename NT::S v = ys[r * W + c];
    if constexpr (sizeof(Out) == 4) {
      const float f = Conv<NT>::to_f(v);
      if (!isfinite(f)) bad = 1;
      mx = fmaxf(mx, fabsf(f));
      out[r * ld + col0 + c] = f;
    } else {
      const double d = Conv<NT>::to_d(v);
      if (!isfinite(d)) bad = 1;
      mx = fmaxf(mx, (float)fabs(d));
      out[r * ld + col0 + c] = d;
    }
  }
  for (int o = 16; o; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0 && flag) {
    atomicMax(reinterpret_cast<int*>(flag) + 1, __float_as_int(mx));
    if (bad) atomicExch(reinterpret_cast<int*>(flag) + 2, 1);
  }
}

// --------------------------------------------------------------- host side
size_t elem_bytes(int kind) { return kind == POLFED_F32 ? 4 : 8; }
int slice_width(int kind, int lpr) { return (int)(16 / elem_bytes(kind)) * lpr; }

int choose_lpr(int kind, int n_b) {
  const int vec = (int)(16 / elem_bytes(kind));
  int lpr = 1;
  while (lpr < 8 && vec * lpr < n_b) lpr *= 2;
  return lpr;
}

static size_t typed_size(int kind) { return kind == POLFED_F64 ? 8 : (kind == POLFED_F32 ? 4 : 8); }

int HamPlan::init(const polfed_model* m, cudaStream_t s, bool stream_ordered, int b_override) {
  release();
  upload_binomials();
  PF_CHECK(build_geometry(m, b_override, &geo));
  stream = s;
  const size_t nlo = (size_t)1 << geo.b, nhi = (size_t)1 << geo.nh, ncx = (size_t)1 << geo.n_cross;
  size_t bytes = 0;
  auto carve = [&](size_t n) {
    size_t o = bytes;
    bytes += (n + 255) & ~(size_t)255;
    return o;
  };
  const size_t oTlo = carve(nlo * 2), oUlo = carve(nlo * 2), oThi = carve(nhi * 4), oOrd = carve(nhi * 4),
               oFlo = carve(nlo * 8), oFhi = carve(nhi * 8), oCx = carve(ncx * 8),
               oRec = carve(nlo * (size_t)geo.rec_stride * 2), oGrp = carve((size_t)geo.n_groups * sizeof(GroupRec)),
               oErr = carve(64), oRec8 = carve(nlo * (size_t)geo.rec_stride);
  stream_alloc = stream_ordered;
  if (stream_ordered)
    PF_CUDA(cudaMallocAsync(&dev, bytes, s));
  else
    PF_CUDA(cudaMalloc(&dev, bytes));
  char* d = (char*)dev;
  tab.T_lo = (uint16_t*)(d + oTlo);
  tab.U_lo = (uint16_t*)(d + oUlo);
  tab.T_hi = (int32_t*)(d + oThi);
  tab.order = (int32_t*)(d + oOrd);
  tab.F_lo = (double*)(d + oFlo);
  tab.F_hi = (double*)(d + oFhi);
  tab.C_x = (double*)(d + oCx);
  tab.rec = (uint16_t*)(d + oRec);
  tab.grec = (GroupRec*)(d + oGrp);
  tab.rec8 = (uint8_t*)(d + oRec8);
  err_flag = (int*)(d + oErr);
  PF_CUDA(cudaMemsetAsync(err_flag, 0, 64, s));
  k_tables_lo<<<(unsigned)((nlo + 255) / 256), 256, 0, s>>>(geo, tab.T_lo, tab.U_lo, tab.F_lo);
  k_tables_rec<<<(unsigned)((nlo + 255) / 256), 256, 0, s>>>(geo, tab.T_lo, tab.rec);
  k_tables_rec8<<<(unsigned)((nlo + 255) / 256), 256, 0, s>>>(geo, tab.rec, tab.rec8);
  k_tables_hi<<<(unsigned)((nhi + 255) / 256), 256, 0, s>>>(geo, tab.T_hi, tab.F_hi);
  k_tables_cx<<<(unsigned)((ncx + 255) / 256), 256, 0, s>>>(geo, tab.C_x);
  PF_CUDA(cudaGetLastError());
  // group schedule: largest groups first (sizes depend only on popcount)
  std::vector<int32_t> order;
  order.reserve(geo.n_groups);
  std::vector<std::pair<int, int>> cls;  // (size, popcount)
  for (int pc = 0; pc <= geo.nh; pc++) {
    int n_lo = geo.n_up - pc;
    if (n_lo < 0 || n_lo > geo.b) continue;
    cls.push_back({(int)binom_host(geo.b, n_lo), pc});
  }
  std::stable_sort(cls.begin(), cls.end(), [](auto& x, auto& y) { return x.first > y.first; });
  for (auto& c : cls)
    for (uint32_t grp = 0; grp < (uint32_t)nhi; grp++)
      if (__builtin_popcount(grp) == c.second) order.push_back((int32_t)grp);
  PF_CUDA(cudaMemcpyAsync(tab.order, order.data(), order.size() * 4, cudaMemcpyHostToDevice, s));
  k_tables_groups<<<(unsigned)((geo.n_groups + 127) / 128), 128, 0, s>>>(geo, tab.T_hi, tab.order, tab.grec);
  PF_CUDA(cudaGetLastError());
  PF_CUDA(cudaStreamSynchronize(s));  // host vector goes out of scope
  return POLFED_OK;
}

int HamPlan::prepare_typed(int kind, double e_lo, double e_hi) {
  if (kind < 0 || kind > 2) return fail(POLFED_EINVAL, "bad dtype");
  if (typed_ok[kind] && typed_lo[kind] == e_lo && typed_hi[kind] == e_hi) return POLFED_OK;
  double alpha = 1.0, beta = 0.0;
  if (!(e_lo == 0.0 && e_hi == 0.0)) {
    if (!(e_hi > e_lo)) return fail(POLFED_EINVAL, "need e_lo < e_hi");
    alpha = 2.0 / (e_hi - e_lo);
    beta = 0.5 * (e_hi + e_lo);
  }
  const size_t nlo = (size_t)1 << geo.b, nhi = (size_t)1 << geo.nh, ncx = (size_t)1 << geo.n_cross;
  const size_t es = typed_size(kind);
  const size_t ngr = (size_t)geo.n_groups;
  const size_t need = (nlo + nhi + ncx + ngr) * es + 512;
  if (!typed[kind] || typed_bytes[kind] < need) {
    if (typed[kind]) {
      if (stream_alloc)
        cudaFreeAsync(typed[kind], stream);
      else
        cudaFree(typed[kind]);
      typed[kind] = nullptr;
    }
    if (stream_alloc)
      PF_CUDA(cudaMallocAsync(&typed[kind], need, stream));
    else
      PF_CUDA(cudaMalloc(&typed[kind], need));
    typed_bytes[kind] = need;
  }
  // scale on the host: copy the FP64 tables back (small), convert, upload
  std::vector<double> flo(nlo), fhi(nhi), cx(ncx);
  std::vector<int32_t> ord(ngr);
  PF_CUDA(cudaMemcpyAsync(flo.data(), tab.F_lo, nlo * 8, cudaMemcpyDeviceToHost, stream));
  PF_CUDA(cudaMemcpyAsync(fhi.data(), tab.F_hi, nhi * 8, cudaMemcpyDeviceToHost, stream));
  PF_CUDA(cudaMemcpyAsync(cx.data(), tab.C_x, ncx * 8, cudaMemcpyDeviceToHost, stream));
  PF_CUDA(cudaMemcpyAsync(ord.data(), tab.order, ngr * 4, cudaMemcpyDeviceToHost, stream));
  PF_CUDA(cudaStreamSynchronize(stream));
  std::vector<unsigned char> buf((nlo + nhi + ncx + ngr) * es);
  size_t pos = 0;
  auto put = [&](double v) {
    if (kind == POLFED_F32) {
      float f = (float)v;
      memcpy(&buf[pos], &f, 4);
    } else if (kind == POLFED_F64) {
      memcpy(&buf[pos], &v, 8);
    } else {
      float hi = (float)v;
      float lo = (float)(v - (double)hi);
      memcpy(&buf[pos], &hi, 4);
      memcpy(&buf[pos + 4], &lo, 4);
    }
    pos += es;
  };
  for (size_t i = 0; i < nlo; i++) put(alpha * flo[i]);
  for (size_t i = 0; i < nhi; i++) put(alpha * (fhi[i] - beta));
  for (size_t i = 0; i < ncx; i++) put(alpha * cx[i]);
  for (size_t i = 0; i < ngr; i++) put(alpha * (fhi[ord[i]] - beta));  // F_hi in schedule order
  PF_CUDA(cudaMemcpyAsync(typed[kind], buf.data(), buf.size(), cudaMemcpyHostToDevice, stream));
  PF_CUDA(cudaStreamSynchronize(stream));
  typed_ok[kind] = true;
  typed_lo[kind] = e_lo;
  typed_hi[kind] = e_hi;
  return POLFED_OK;
}

void HamPlan::release() {
  for (StepGraph& gr : graphs)
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
  graphs.clear();
  if (dev) {
    if (stream_alloc)
      cudaFreeAsync(dev, stream);
    else
      cudaFree(dev);
  }
  for (int k = 0; k < 3; k++) {
    if (typed[k]) {
      if (stream_alloc)
        cudaFreeAsync(typed[k], stream);
      else
        cudaFree(typed[k]);
    }
    typed[k] = nullptr;
    typed_bytes[k] = 0;
    typed_ok[k] = false;
  }
  dev = nullptr;
}

static void split_df(double v, float2& o) {
  o.x = (float)v;
  o.y = (float)(v - (double)o.x);
}

// 0 or +-2^k (with k in the float exponent range): scaling by it is exact
static bool pow2_or_zero(double v) {
  if (v == 0.0) return true;
  int e = 0;
  const double m = std::frexp(std::fabs(v), &e);
  return m == 0.5 && e > -120 && e < 120;
}

// Per-kernel, per-device launch configuration (shared-memory limit, SM count,
// occupancy), filled once under its mutex.
struct LaunchCache {
  static constexpr int kDevices = 64;
  struct Dev {
    bool set = false;
    int nsm = 0;
    size_t maxdyn = 0;
    size_t occ_smem = 0;
    int occ = 0;
  };
  std::mutex mu;
  Dev d[kDevices];
};

template <class NT, int LPR, bool J2>
static int launch_step_t(const HamPlan& p, const StepArgs& a, cudaStream_t s) {
  if (p.geo.n_cross > (J2 ? 6 : 2)) return fail(POLFED_EINVAL, "more cross bonds than the kernel handles");
  using S = typename NT::S;
  using C = typename NT::C;
  constexpr int W = (16 / sizeof(S)) * LPR;
  const HamGeometry& g = p.geo;
  const size_t smem = (size_t)g.max_group * W * sizeof(S) + (((size_t)1 << g.b) + ((size_t)1 << g.n_cross)) * sizeof(C);
  auto kern = k_ham_step<NT, LPR, J2>;
  // per-device launch configuration of this kernel, computed once under a
  // mutex (the batched runner's worker threads launch concurrently)
  static LaunchCache cache;
  int dev = 0;
  PF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= LaunchCache::kDevices) return fail(POLFED_EINVAL, "device ordinal beyond the launch cache");
  const int threads = 256;
  int nsm = 0, occ = 0;
  {
    std::lock_guard<std::mutex> lk(cache.mu);
    LaunchCache::Dev& c = cache.d[dev];
    if (!c.set) {
      int optin = 0;
      PF_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      cudaFuncAttributes fa;
      PF_CUDA(cudaFuncGetAttributes(&fa, kern));
      const int maxdyn = optin - (int)fa.sharedSizeBytes;
      PF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, maxdyn));
      PF_CUDA(cudaDeviceGetAttribute(&c.nsm, cudaDevAttrMultiProcessorCount, dev));
      c.maxdyn = (size_t)maxdyn;
      c.set = true;
    }
    if (smem > c.maxdyn) return fail(POLFED_EINVAL, "slice tile does not fit in shared memory");
    if (c.occ_smem != smem || c.occ <= 0) {
      PF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c.occ, kern, threads, smem));
      c.occ_smem = smem;
    }
    nsm = c.nsm;
    occ = c.occ;
  }
  if (occ < 1) return fail(POLFED_EINVAL, "step kernel cannot be resident (shared memory)");
  int grid = std::min(g.n_groups, nsm * occ);
  StepTables t{p.tab.rec, p.tab.rec8, p.tab.grec, nullptr, nullptr, nullptr, p.tab.order};
  if (g.rec_stride != (J2 ? 32 : 16)) return fail(POLFED_EINVAL, "record layout does not match the kernel");
  const size_t es = sizeof(C);
  const char* base = (const char*)p.typed[std::is_same<NT, NF32>::value ? POLFED_F32 : (std::is_same<NT, NF64>::value ? POLFED_F64 : POLFED_DF64)];
  t.F_lo = base;
  t.F_hi = base + ((size_t)1 << g.b) * es;
  t.C_x = base + (((size_t)1 << g.b) + ((size_t)1 << g.nh)) * es;
  typename NT::KC kc;
  const int kk = std::is_same<NT, NF32>::value ? POLFED_F32 : (std::is_same<NT, NF64>::value ? POLFED_F64 : POLFED_DF64);
  const double alpha = (p.typed_lo[kk] == 0.0 && p.typed_hi[kk] == 0.0) ? 1.0 : 2.0 / (p.typed_hi[kk] - p.typed_lo[kk]);
  const double o1 = alpha * 0.5 * g.J1, o2 = alpha * 0.5 * g.J2;
  if constexpr (std::is_same<NT, NDF>::value) {
    split_df(a.cX, kc.cX);
    split_df(a.cH, kc.cH);
    split_df(a.cB, kc.cB);
    split_df(o1, kc.o1);
    split_df(o2, kc.o2);
    kc.exact = pow2_or_zero(a.cX) && pow2_or_zero(a.cH) && pow2_or_zero(a.cB);
  } else {
    kc.cX = (C)a.cX;
    kc.cH = (C)a.cH;
    kc.cB = (C)a.cB;
    kc.o1 = (C)o1;
    kc.o2 = (C)o2;
  }
  const bool hx = a.x != nullptr && (a.cX != 0.0 || a.cxcol != nullptr);
  kern<<<grid, threads, smem, s>>>(g, t, (const S*)a.b1, (const S*)a.b2, (const S*)a.x, (S*)a.out, kc, hx,
                                   a.cB != 0.0 && a.b2 != nullptr, a.cxcol);
  PF_CUDA(cudaGetLastError());
  count_step(kk, (double)g.dim * W * sizeof(S) * (3.0 + (hx ? 1.0 : 0.0)));
  return POLFED_OK;
}

static size_t tma_smem_bytes(const HamGeometry& g, size_t esz_c, bool j2) {
  const size_t stg = (size_t)g.max_group * 128;
  return (2 + tma_stages(j2)) * stg + ((size_t)g.rec_stride << g.b) +
         (((size_t)1 << g.b) + ((size_t)1 << g.n_cross)) * esz_c;
}

static bool tma_disabled() {
  static const bool v = [] {
    const char* e = getenv("POLFED_NO_TMA");
    return e && e[0] == '1';
  }();
  return v;
}

template <class NT, bool J2, class SH>
static int launch_step_tma(const HamPlan& p, const StepArgs& a, cudaStream_t s) {
  using S = typename NT::S;
  using C = typename NT::C;
  const HamGeometry& g = p.geo;
  const size_t smem = tma_smem_bytes(g, sizeof(C), J2);
  auto kern = k_ham_step_tma<NT, J2, SH>;
  static LaunchCache cache;  // see launch_step_t
  int dev = 0;
  PF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= LaunchCache::kDevices) return fail(POLFED_EINVAL, "device ordinal beyond the launch cache");
  int nsm = 0;
  {
    std::lock_guard<std::mutex> lk(cache.mu);
    LaunchCache::Dev& c = cache.d[dev];
    if (!c.set) {
      int optin = 0;
      PF_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      cudaFuncAttributes fa;
      PF_CUDA(cudaFuncGetAttributes(&fa, kern));
      PF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
      PF_CUDA(cudaDeviceGetAttribute(&c.nsm, cudaDevAttrMultiProcessorCount, dev));
      c.set = true;
    }
    nsm = c.nsm;
  }
  const int grid = std::min(g.n_groups, nsm);
  const int kk = std::is_same<NT, NF32>::value ? POLFED_F32 : (std::is_same<NT, NF64>::value ? POLFED_F64 : POLFED_DF64);
  StepTables t{p.tab.rec, p.tab.rec8, p.tab.grec, nullptr, nullptr, nullptr, p.tab.order};
  const size_t es = sizeof(C);
  const char* base = (const char*)p.typed[kk];
  t.F_lo = base;
  t.F_hi = base + ((size_t)1 << g.b) * es;
  t.C_x = base + (((size_t)1 << g.b) + ((size_t)1 << g.nh)) * es;
  t.F_hi = base + (((size_t)1 << g.b) + ((size_t)1 << g.nh) + ((size_t)1 << g.n_cross)) * es;  // schedule order
  typename NT::KC kc;
  const double alpha = (p.typed_lo[kk] == 0.0 && p.typed_hi[kk] == 0.0) ? 1.0 : 2.0 / (p.typed_hi[kk] - p.typed_lo[kk]);
  const double o1 = alpha * 0.5 * g.J1, o2 = alpha * 0.5 * g.J2;
  if constexpr (std::is_same<NT, NDF>::value) {
    split_df(a.cX, kc.cX);
    split_df(a.cH, kc.cH);
    split_df(a.cB, kc.cB);
    split_df(o1, kc.o1);
    split_df(o2, kc.o2);
    kc.exact = pow2_or_zero(a.cX) && pow2_or_zero(a.cH) && pow2_or_zero(a.cB);
  } else {
    kc.cX = (C)a.cX;
    kc.cH = (C)a.cH;
    kc.cB = (C)a.cB;
    kc.o1 = (C)o1;
    kc.o2 = (C)o2;
  }
  const bool hx = a.x != nullptr && (a.cX != 0.0 || a.cxcol != nullptr);
  kern<<<grid, SH::THREADS, smem, s>>>(g, t, (const S*)a.b1, (const S*)a.b2, (const S*)a.x, (S*)a.out, kc, hx,
                                       a.cB != 0.0 && a.b2 != nullptr, p.err_flag, wait_cap(kMbarWaitPolls), a.cxcol);
  PF_CUDA(cudaGetLastError());
  count_step(kk, (double)g.dim * 128.0 * (3.0 + (hx ? 1.0 : 0.0)));
  return POLFED_OK;
}

template <class NT>
static int launch_step_n(const HamPlan& p, const StepArgs& a, cudaStream_t s) {
  const bool j2 = p.geo.n_low2 + p.geo.n_high2 > 0 || p.geo.J2 != 0.0;
  if (a.lpr == 8 && !tma_disabled() && p.geo.max_group <= 252 &&
      p.geo.n_high1 + p.geo.n_high2 <= 4 * tma_high_words(j2) &&
      4 + p.geo.n_low1 + p.geo.n_low2 + (j2 ? 6 : 2) <= p.geo.rec_stride &&
      tma_smem_bytes(p.geo, sizeof(typename NT::C), j2) <= 220 * 1024 && p.geo.max_group >= 32 &&
      p.geo.rec_stride == (j2 ? 32 : 16)) {
    return j2 ? launch_step_tma<NT, true, TmaShapeA>(p, a, s) : launch_step_tma<NT, false, TmaShapeA>(p, a, s);
  }
  switch (a.lpr) {
#define PF_CASE(L_)                                                               \
  case L_:                                                                        \
    return j2 ? launch_step_t<NT, L_, true>(p, a, s) : launch_step_t<NT, L_, false>(p, a, s);
    PF_CASE(1)
    PF_CASE(2)
    PF_CASE(4)
    PF_CASE(8)
#undef PF_CASE
    default:
      return fail(POLFED_EINVAL, "unsupported lanes-per-row");
  }
}

int launch_ham_step(const HamPlan& p, int kind, const StepArgs& a, cudaStream_t s) {
  if (kind < 0 || kind > 2 || !p.typed_ok[kind]) return fail(POLFED_EINVAL, "operator tables not prepared for this precision");
  if (a.cxcol && kind != POLFED_F32) return fail(POLFED_EINVAL, "per-column coefficients need FP32 storage");
  switch (kind) {
    case POLFED_F32:
      return launch_step_n<NF32>(p, a, s);
    case POLFED_F64:
      return launch_step_n<NF64>(p, a, s);
    case POLFED_DF64:
      return launch_step_n<NDF>(p, a, s);
  }
  return fail(POLFED_EINVAL, "unknown dtype");
}

size_t filter_scratch_bytes(const HamPlan& plan, int kind, int lpr) {
  const size_t slice = (size_t)plan.geo.dim * slice_width(kind, lpr) * elem_bytes(kind);
  const size_t a = (slice + 255) & ~(size_t)255;
  return 3 * a + 256;
}

static int ensure_scratch(FilterScratch& scr, size_t need, const HamPlan& plan, int kind, int lpr) {
  if (scr.xs && scr.bytes >= need) return POLFED_OK;
  return fail(POLFED_ENOMEM, "filter scratch too small");
}

static void carve_scratch(FilterScratch& scr, const HamPlan& plan, int kind, int lpr) {
  const size_t slice = (size_t)plan.geo.dim * slice_width(kind, lpr) * elem_bytes(kind);
  const size_t a = (slice + 255) & ~(size_t)255;
  char* base = (char*)scr.xs;
  scr.ba = base + a;
  scr.bb = base + 2 * a;
  scr.flag = (float*)(base + 3 * a);
}

template <class NT, class In>
static int slice_in_t(const void* in, int64_t dim, int ld, int col0, int ncols, int W, void* xs, void* as,
                      void* zb, double scale, float* flag, cudaStream_t s, const float* colscale) {
  typename NT::C cs;
  if constexpr (std::is_same<NT, NDF>::value)
    split_df(scale, cs);
  else
    cs = (typename NT::C)scale;
  const int64_t n = dim * W;
  int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
  k_slice_in<NT, In><<<grid, 256, 0, s>>>((const In*)in, dim, ld, col0, ncols, W, (typename NT::S*)xs,
                                           (typename NT::S*)as, (typename NT::S*)zb, cs, flag, colscale);
  PF_CUDA(cudaGetLastError());
  count_launch();
  return POLFED_OK;
}

static int slice_in(int kind, int abi_kind, const void* in, int64_t dim, int ld, int col0, int ncols, int W,
                    void* xs, void* as, void* zb, double scale, float* flag, cudaStream_t s,
                    const float* colscale = nullptr) {
  const bool f32in = abi_kind == POLFED_F32;
  switch (kind) {
    case POLFED_F32:
      return f32in ? slice_in_t<NF32, float>(in, dim, ld, col0, ncols, W, xs, as, zb, scale, flag, s, colscale)
                   : slice_in_t<NF32, double>(in, dim, ld, col0, ncols, W, xs, as, zb, scale, flag, s, colscale);
    case POLFED_F64:
      return f32in ? slice_in_t<NF64, float>(in, dim, ld, col0, ncols, W, xs, as, zb, scale, flag, s, colscale)
                   : slice_in_t<NF64, double>(in, dim, ld, col0, ncols, W, xs, as, zb, scale, flag, s, colscale);
    default:
      return f32in ? slice_in_t<NDF, float>(in, dim, ld, col0, ncols, W, xs, as, zb, scale, flag, s, colscale)
                   : slice_in_t<NDF, double>(in, dim, ld, col0, ncols, W, xs, as, zb, scale, flag, s, colscale);
  }
}

template <class NT>
static void slice_out_t(const void* ys, int64_t dim, int W, int ncols, void* out, bool f32out, int ld, int col0,
                        float* flag, int grid, cudaStream_t s) {
  if (f32out)
    k_slice_out<NT, float><<<grid, 256, 0, s>>>((const typename NT::S*)ys, dim, W, ncols, (float*)out, ld, col0, flag);
  else
    k_slice_out<NT, double><<<grid, 256, 0, s>>>((const typename NT::S*)ys, dim, W, ncols, (double*)out, ld, col0,
                                                  flag);
}

static int slice_out(int kind, int abi_kind, const void* ys, int64_t dim, int W, int ncols, void* out, int ld,
                     int col0, float* flag, cudaStream_t s) {
  const int64_t n = dim * ncols;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
  const bool f32out = abi_kind == POLFED_F32;
  if (kind == POLFED_F32)
    slice_out_t<NF32>(ys, dim, W, ncols, out, f32out, ld, col0, flag, grid, s);
  else if (kind == POLFED_F64)
    slice_out_t<NF64>(ys, dim, W, ncols, out, f32out, ld, col0, flag, grid, s);
  else
    slice_out_t<NDF>(ys, dim, W, ncols, out, f32out, ld, col0, flag, grid, s);
  PF_CUDA(cudaGetLastError());
  count_launch();
  return POLFED_OK;
}

// Device time of a run of step launches, by a pair of CUDA events on the launching stream.
// The launches of storage kind `kind` issued between construction and stop()
// are credited to the timed counters with the measured time.
struct StepTimer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s;
  int kind;
  int64_t n0;
  double b0;
  StepTimer(cudaStream_t st, int k) : s(st), kind(k) {
    n0 = counters().all_launches[kind];
    b0 = counters().all_alg_bytes[kind];
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) cudaEventRecord(e0, s);
  }
  int stop() {
    if (!e0 || !e1) return POLFED_OK;
    PF_CUDA(cudaEventRecord(e1, s));
    PF_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    PF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    Counters& c = counters();
    const int64_t n = c.all_launches[kind] - n0;
    const double b = c.all_alg_bytes[kind] - b0;
    c.step_gpu_s += 1e-3 * ms;
    c.step_launches += n;
    c.step_alg_bytes += b;
    c.kind_gpu_s[kind] += 1e-3 * ms;
    c.kind_launches[kind] += n;
    c.kind_alg_bytes[kind] += b;
    return POLFED_OK;
  }
  ~StepTimer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

// A step kernel whose bounded wait expired leaves plan.err_flag set.
static int check_timeout(HamPlan& plan, cudaStream_t s) {
  int e = 0;
  PF_CUDA(cudaMemcpyAsync(&e, plan.err_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  if (e) {
    cudaMemsetAsync(plan.err_flag, 0, sizeof(int), s);
    return fail(POLFED_ETIMEOUT, "a bounded device wait in the step kernel expired");
  }
  return POLFED_OK;
}

// Launch the Clenshaw steps k = K-1..1 and the final step of Eq. (2) on the
// scratch slices (b_K in ba, b_{K+1} = 0 in bb, X in xs; result in the buffer
// the last step writes, returned in *res).
static int clenshaw_steps(HamPlan& plan, int kind, const double* c, int K, double invD, FilterScratch& scr, int lpr,
                          cudaStream_t s, void** res) {
  void* cur = scr.ba;  // b_{k+1}
  void* oth = scr.bb;  // b_{k+2}, overwritten in place by b_k
  for (int k = K - 1; k >= 1; k--) {
    StepArgs a{cur, oth, scr.xs, oth, c[k], 2.0, (k == K - 1) ? 0.0 : -1.0, lpr};
    PF_CHECK(launch_ham_step(plan, kind, a, s));
    std::swap(cur, oth);
  }
  // Y = (c_0 X + H~ b_1 - b_2) / D
  StepArgs a{cur, oth, scr.xs, oth, c[0] * invD, invD, (K == 1) ? 0.0 : -invD, lpr};
  PF_CHECK(launch_ham_step(plan, kind, a, s));
  *res = oth;
  return POLFED_OK;
}

static uint64_t fnv_hash(const double* v, int n) {
  uint64_t h = 1469598103934665603ull;
  const unsigned char* b = (const unsigned char*)v;
  for (size_t i = 0; i < (size_t)n * sizeof(double); i++) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

static bool graphs_disabled() {
  static const bool v = [] {
    const char* e = getenv("POLFED_NO_GRAPHS");
    return e && e[0] == '1';
  }();
  return v;
}

// The recurrence only touches the scratch slices, so one CUDA graph of its K
// launches serves every slice of every call with the same operator tables,
// coefficients and scratch: a key seen a second time on a plan is captured
// once and replayed from then on (kernels of K >= 16 steps).  Counters are
// credited per replay.
static int clenshaw_graph(HamPlan& plan, int kind, const double* c, int K, double invD, FilterScratch& scr, int lpr,
                          cudaStream_t s, void** res) {
  // the legacy default stream cannot be captured (and the per-thread one is left alone too)
  if (K < 16 || graphs_disabled() || s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread)
    return clenshaw_steps(plan, kind, c, K, invD, scr, lpr, s, res);
  StepGraph key;
  key.kind = kind;
  key.K = K;
  key.lpr = lpr;
  key.invD = invD;
  key.lo = plan.typed_lo[kind];
  key.hi = plan.typed_hi[kind];
  key.coef_hash = fnv_hash(c, K + 1);
  key.wait_cap = wait_cap(kMbarWaitPolls);
  key.xs = scr.xs;
  key.ba = scr.ba;
  key.bb = scr.bb;
  StepGraph* hit = nullptr;
  for (StepGraph& gr : plan.graphs)
    if (gr.kind == key.kind && gr.K == key.K && gr.uses < 0 && gr.xs == key.xs && gr.coef_hash == key.coef_hash)
      return clenshaw_steps(plan, kind, c, K, invD, scr, lpr, s, res);  // capture failed before: stay eager
  for (StepGraph& gr : plan.graphs)
    if (gr.kind == key.kind && gr.K == key.K && gr.lpr == key.lpr && gr.invD == key.invD && gr.lo == key.lo &&
        gr.hi == key.hi && gr.coef_hash == key.coef_hash && gr.wait_cap == key.wait_cap && gr.xs == key.xs &&
        gr.ba == key.ba && gr.bb == key.bb)
      hit = &gr;
  // the result buffer: K - 1 swaps after starting in ba
  void* out_buf = (K % 2 == 0) ? scr.ba : scr.bb;
  if (!hit) {  // first sighting: run eagerly, remember the key
    if (plan.graphs.size() >= 8) {
      if (plan.graphs.front().exec) cudaGraphExecDestroy(plan.graphs.front().exec);
      plan.graphs.erase(plan.graphs.begin());
    }
    plan.graphs.push_back(key);
    return clenshaw_steps(plan, kind, c, K, invD, scr, lpr, s, res);
  }
  if (!hit->exec) {
    Counters& cn = counters();
    const int64_t l0 = cn.launches, n0 = cn.all_launches[kind];
    const double b0 = cn.all_alg_bytes[kind];
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaGetLastError();  // not capturable here (e.g. the stream is already being captured): run eagerly
      hit->uses = -1;
      return clenshaw_steps(plan, kind, c, K, invD, scr, lpr, s, res);
    }
    void* r = nullptr;
    const int rc = clenshaw_steps(plan, kind, c, K, invD, scr, lpr, s, &r);
    const cudaError_t ec = cudaStreamEndCapture(s, &graph);
    // the capture executed nothing: take its counts back, credit them per replay
    hit->launches = cn.all_launches[kind] - n0;
    hit->alg_bytes = cn.all_alg_bytes[kind] - b0;
    cn.launches = l0;
    cn.all_launches[kind] = n0;
    cn.all_alg_bytes[kind] = b0;
    if (rc != POLFED_OK || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc != POLFED_OK ? rc : fail(POLFED_ECUDA, std::string("stream capture: ") + cudaGetErrorString(ec));
    }
    const cudaError_t ei = cudaGraphInstantiate(&hit->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      hit->exec = nullptr;
      cudaGetLastError();
      return fail(POLFED_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
    }
  }
  PF_CUDA(cudaGraphLaunch(hit->exec, s));
  Counters& cn = counters();
  cn.launches += hit->launches;
  cn.all_launches[kind] += hit->launches;
  cn.all_alg_bytes[kind] += hit->alg_bytes;
  hit->uses++;
  *res = out_buf;
  return POLFED_OK;
}

int filter_block(HamPlan& plan, int kind, const double* c, int K, double invD, const void* in, void* out, int n_b,
                 int abi_kind, FilterScratch& scr, cudaStream_t s, int lpr_hint) {
  const int lpr = lpr_hint > 0 ? lpr_hint : choose_lpr(kind, n_b);
  const int W = slice_width(kind, lpr);
  PF_CHECK(ensure_scratch(scr, filter_scratch_bytes(plan, kind, lpr), plan, kind, lpr));
  carve_scratch(scr, plan, kind, lpr);
  const int64_t dim = plan.geo.dim;
  PF_CUDA(cudaMemsetAsync(scr.flag, 0, 16, s));
  for (int col0 = 0; col0 < n_b; col0 += W) {
    const int ncols = std::min(W, n_b - col0);
    if (K == 0) {
      PF_CHECK(slice_in(kind, abi_kind, in, dim, n_b, col0, ncols, W, nullptr, scr.ba, nullptr, c[0] * invD,
                        scr.flag, s));
      PF_CHECK(slice_out(kind, abi_kind, scr.ba, dim, W, ncols, out, n_b, col0, scr.flag, s));
      continue;
    }
    // b_K = c_K X (in ba), b_{K+1} = 0 (in bb)
    PF_CHECK(slice_in(kind, abi_kind, in, dim, n_b, col0, ncols, W, scr.xs, scr.ba, scr.bb, c[K], scr.flag, s));
    void* res = nullptr;
    StepTimer tm(s, kind);
    PF_CHECK(clenshaw_graph(plan, kind, c, K, invD, scr, lpr, s, &res));
    PF_CHECK(tm.stop());
    PF_CHECK(check_timeout(plan, s));
    PF_CHECK(slice_out(kind, abi_kind, res, dim, W, ncols, out, n_b, col0, scr.flag, s));
  }
  return POLFED_OK;
}

int filter_block_cols(HamPlan& plan, const float* d_coef, int K, const void* in, void* out, int n_b, int abi_kind,
                      FilterScratch& scr, cudaStream_t s) {
  const int kind = POLFED_F32;
  const int lpr = choose_lpr(kind, n_b);
  const int W = slice_width(kind, lpr);
  if (K < 1) return fail(POLFED_EINVAL, "per-column filter needs K >= 1");
  PF_CHECK(ensure_scratch(scr, filter_scratch_bytes(plan, kind, lpr), plan, kind, lpr));
  carve_scratch(scr, plan, kind, lpr);
  const int64_t dim = plan.geo.dim;
  PF_CUDA(cudaMemsetAsync(scr.flag, 0, 16, s));
  for (int col0 = 0, q = 0; col0 < n_b; col0 += W, q++) {
    const int ncols = std::min(W, n_b - col0);
    const float* cq = d_coef + (size_t)q * (K + 1) * W;  // rows n = 0..K of this slice's W columns
    // b_K = c_K X (per column), b_{K+1} = 0
    PF_CHECK(slice_in(kind, abi_kind, in, dim, n_b, col0, ncols, W, scr.xs, scr.ba, scr.bb, 1.0, scr.flag, s,
                      cq + (size_t)K * W));
    void* cur = scr.ba;
    void* oth = scr.bb;
    StepTimer tm(s, kind);
    for (int k = K - 1; k >= 1; k--) {
      StepArgs a{cur, oth, scr.xs, oth, 1.0, 2.0, (k == K - 1) ? 0.0 : -1.0, lpr, cq + (size_t)k * W};
      PF_CHECK(launch_ham_step(plan, kind, a, s));
      std::swap(cur, oth);
    }
    // Y = c_0 X + H~ b_1 - b_2
    StepArgs a{cur, oth, scr.xs, oth, 1.0, 1.0, (K == 1) ? 0.0 : -1.0, lpr, cq};
    PF_CHECK(launch_ham_step(plan, kind, a, s));
    PF_CHECK(tm.stop());
    PF_CHECK(check_timeout(plan, s));
    PF_CHECK(slice_out(kind, abi_kind, oth, dim, W, ncols, out, n_b, col0, scr.flag, s));
  }
  return POLFED_OK;
}

int apply_block(HamPlan& plan, int kind, const void* in, void* out, int n_b, int abi_kind, FilterScratch& scr,
                cudaStream_t s, int lpr_hint) {
  const int lpr = lpr_hint > 0 ? lpr_hint : choose_lpr(kind, n_b);
  const int W = slice_width(kind, lpr);
  PF_CHECK(ensure_scratch(scr, filter_scratch_bytes(plan, kind, lpr), plan, kind, lpr));
  carve_scratch(scr, plan, kind, lpr);
  const int64_t dim = plan.geo.dim;
  PF_CUDA(cudaMemsetAsync(scr.flag, 0, 16, s));
  for (int col0 = 0; col0 < n_b; col0 += W) {
    const int ncols = std::min(W, n_b - col0);
    PF_CHECK(slice_in(kind, abi_kind, in, dim, n_b, col0, ncols, W, scr.xs, nullptr, nullptr, 0.0, scr.flag, s));
    StepArgs a{scr.xs, nullptr, nullptr, scr.ba, 0.0, 1.0, 0.0, lpr};
    PF_CHECK(launch_ham_step(plan, kind, a, s));
    PF_CHECK(slice_out(kind, abi_kind, scr.ba, dim, W, ncols, out, n_b, col0, scr.flag, s));
  }
  PF_CHECK(check_timeout(plan, s));
  return POLFED_OK;
}

// ------------------------------------------------ batched filter (host side)
namespace {

struct BatchLayout {
  size_t jobs_off, coef_off, flags_off, bar_off, slices_off, total;
  int n_jobs;
};

int batch_width(int kind) { return slice_width(kind, 8); }

BatchLayout batch_layout(const std::vector<BatchFilterItem>& items, int kind) {
  BatchLayout L{};
  const int W = batch_width(kind);
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  int n_jobs = 0;
  size_t coefs = 0, slices = 0;
  for (const auto& it : items) {
    const int ns = (it.n_b + W - 1) / W;
    n_jobs += ns;
    coefs += (size_t)it.K + 1;
    const size_t sb = al((size_t)it.plan->geo.dim * W * elem_bytes(kind));
    slices += (size_t)ns * 3 * sb;
  }
  L.n_jobs = n_jobs;
  L.jobs_off = 0;
  L.coef_off = al(sizeof(BatchJob) * std::max(1, n_jobs));
  L.flags_off = L.coef_off + al(sizeof(double) * std::max<size_t>(1, coefs));
  L.bar_off = L.flags_off + al(16 * std::max<size_t>(1, items.size()));
  L.slices_off = L.bar_off + 256;
  L.total = L.slices_off + slices;
  return L;
}

template <class NT, bool J2>
int launch_batched(const BatchJob* d_jobs, int n_jobs, int n_steps, int tile_elems, int nlo_max, unsigned* bar,
                   int* err, int ctas_per_sm, cudaStream_t s, int* grid_out) {
  using S = typename NT::S;
  using C = typename NT::C;
  auto kern = k_filter_batched<NT, J2>;
  const size_t smem = (size_t)tile_elems * sizeof(S) + ((size_t)nlo_max + 64) * sizeof(C);
  int dev = 0;
  PF_CUDA(cudaGetDevice(&dev));
  int optin = 0, nsm = 0, coop = 0;
  PF_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  PF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  PF_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return fail(POLFED_ECUDA, "device does not support cooperative launches");
  cudaFuncAttributes fa;
  PF_CUDA(cudaFuncGetAttributes(&fa, kern));
  if (smem + fa.sharedSizeBytes > (size_t)optin) return fail(POLFED_EINVAL, "batched filter tile does not fit");
  PF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  PF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, smem));
  if (occ < 1) return fail(POLFED_EINVAL, "batched filter kernel cannot be resident");
  const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
  int grid = nsm * per_sm;  // every CTA co-resident: the grid barrier cannot deadlock
  unsigned* count = bar;
  unsigned* gen = bar + 1;
  uint32_t cap = wait_cap(kBarrierWaitPolls);
  void* args[] = {(void*)&d_jobs, (void*)&n_jobs, (void*)&n_steps, (void*)&tile_elems, (void*)&nlo_max,
                  (void*)&count, (void*)&gen, (void*)&err, (void*)&cap};
  PF_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(256), args, smem, s));
  *grid_out = grid;
  return POLFED_OK;
}

}  // namespace

size_t batch_scratch_bytes(const std::vector<BatchFilterItem>& items, int kind) {
  return batch_layout(items, kind).total;
}

int filter_batched(std::vector<BatchFilterItem>& items, int kind, int abi_kind, void* scratch, size_t bytes,
                   cudaStream_t s, int ctas_per_sm, BatchStats* bst) {
  if (items.empty()) return POLFED_OK;
  if (kind != POLFED_F32 && kind != POLFED_DF64) return fail(POLFED_EINVAL, "batched filter: FP32 or DF64 only");
  const BatchLayout Lo = batch_layout(items, kind);
  if (!scratch || bytes < Lo.total) return fail(POLFED_ENOMEM, "batched filter scratch too small");
  const int W = batch_width(kind);
  const size_t es = elem_bytes(kind);
  char* base = (char*)scratch;
  const bool j2 = items[0].plan->geo.J2 != 0.0;
  std::vector<BatchJob> jobs;
  std::vector<double> coefs;
  jobs.reserve(Lo.n_jobs);
  size_t slice_pos = Lo.slices_off;
  int n_steps = 0, tile_elems = 0, nlo_max = 1;
  double alg = 0.0;
  const int kk = kind;
  PF_CUDA(cudaMemsetAsync(base + Lo.flags_off, 0, 16 * items.size(), s));
  PF_CUDA(cudaMemsetAsync(base + Lo.bar_off, 0, 256, s));
  for (size_t q = 0; q < items.size(); q++) {
    BatchFilterItem& it = items[q];
    HamPlan& p = *it.plan;
    const HamGeometry& g = p.geo;
    if ((g.J2 != 0.0) != j2) return fail(POLFED_EINVAL, "batched filter: all jobs must agree on J2 = 0 or not");
    if (g.n_cross > (j2 ? 6 : 2)) return fail(POLFED_EINVAL, "more cross bonds than the kernel handles");
    if (g.rec_stride != (j2 ? 32 : 16)) return fail(POLFED_EINVAL, "record layout does not match the kernel");
    if (!p.typed_ok[kk]) return fail(POLFED_EINVAL, "batched filter: typed tables not prepared");
    float* flag = (float*)(base + Lo.flags_off + 16 * q);
    const size_t sb = ((size_t)g.dim * W * es + 255) & ~(size_t)255;
    const double alpha = (p.typed_lo[kk] == 0.0 && p.typed_hi[kk] == 0.0) ? 1.0 : 2.0 / (p.typed_hi[kk] - p.typed_lo[kk]);
    const size_t cs = (kk == POLFED_F32 ? 4 : 8);
    const char* tb = (const char*)p.typed[kk];
    const size_t coef_idx = coefs.size();
    coefs.insert(coefs.end(), it.coef, it.coef + it.K + 1);
    for (int col0 = 0; col0 < it.n_b; col0 += W) {
      const int ncols = std::min(W, it.n_b - col0);
      void* xs = base + slice_pos;
      void* ba = base + slice_pos + sb;
      void* bb = base + slice_pos + 2 * sb;
      slice_pos += 3 * sb;
      if (it.K == 0) {
        PF_CHECK(slice_in(kind, abi_kind, it.in, g.dim, it.n_b, col0, ncols, W, nullptr, ba, nullptr,
                          it.coef[0] * it.invD, flag, s));
        continue;
      }
      PF_CHECK(slice_in(kind, abi_kind, it.in, g.dim, it.n_b, col0, ncols, W, xs, ba, bb, it.coef[it.K], flag, s));
      BatchJob J{};
      J.t = StepTables{p.tab.rec, p.tab.rec8, p.tab.grec, tb, tb + ((size_t)1 << g.b) * cs,
                       tb + (((size_t)1 << g.b) + ((size_t)1 << g.nh)) * cs, p.tab.order};
      J.coef = (const double*)(base + Lo.coef_off) + coef_idx;
      J.xs = xs;
      J.ba = ba;
      J.bb = bb;
      J.invD = it.invD;
      J.o1 = alpha * 0.5 * g.J1;
      J.o2 = alpha * 0.5 * g.J2;
      J.K = it.K;
      J.n_groups = g.n_groups;
      J.n_cross = g.n_cross;
      J.nlo_tab = 1 << g.b;
      for (int k = 0; k < g.n_cross && k < 6; k++) {
        J.cross_lo[k] = g.cross_lo[k];
        J.cross_cls[k] = g.cross_cls[k];
      }
      jobs.push_back(J);
      n_steps = std::max(n_steps, it.K);
      tile_elems = std::max(tile_elems, g.max_group * W);
      nlo_max = std::max(nlo_max, 1 << g.b);
      // Clenshaw minimum per step: read b_{k+1}, b_{k+2}, write b_k, read X when c_k != 0
      for (int k = it.K - 1; k >= 0; k--) {
        const bool hx = (k >= 1 ? it.coef[k] : it.coef[0]) != 0.0;
        alg += (double)g.dim * W * es * (3.0 + (hx ? 1.0 : 0.0));
      }
    }
  }
  if (!jobs.empty()) {
    PF_CUDA(cudaMemcpyAsync(base + Lo.coef_off, coefs.data(), coefs.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    PF_CUDA(cudaMemcpyAsync(base + Lo.jobs_off, jobs.data(), jobs.size() * sizeof(BatchJob), cudaMemcpyHostToDevice, s));
    unsigned* bar = (unsigned*)(base + Lo.bar_off);
    int* err = (int*)(bar + 2);
    int grid = 0;
    StepTimer tm(s, kind);
    int rc;
    if (kind == POLFED_F32)
      rc = j2 ? launch_batched<NF32, true>((const BatchJob*)base, (int)jobs.size(), n_steps, tile_elems, nlo_max, bar,
                                           err, ctas_per_sm, s, &grid)
              : launch_batched<NF32, false>((const BatchJob*)base, (int)jobs.size(), n_steps, tile_elems, nlo_max, bar,
                                            err, ctas_per_sm, s, &grid);
    else
      rc = j2 ? launch_batched<NDF, true>((const BatchJob*)base, (int)jobs.size(), n_steps, tile_elems, nlo_max, bar,
                                          err, ctas_per_sm, s, &grid)
              : launch_batched<NDF, false>((const BatchJob*)base, (int)jobs.size(), n_steps, tile_elems, nlo_max, bar,
                                           err, ctas_per_sm, s, &grid);
    if (rc != POLFED_OK) return rc;
    count_step(kind, alg);  // one launch carrying every job's steps
    const double g0 = counters().step_gpu_s;
    PF_CHECK(tm.stop());
    Counters& cn = counters();
    if (bst) {
      bst->n_jobs = (int)jobs.size();
      bst->n_steps = n_steps;
      bst->grid = grid;
      bst->gpu_s = cn.step_gpu_s - g0;
      bst->alg_bytes = alg;
    }
    int e = 0;
    PF_CUDA(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PF_CUDA(cudaStreamSynchronize(s));
    if (e) return fail(POLFED_ETIMEOUT, "a grid barrier of the batched filter timed out");
  }
  // outputs: the buffer written by each job's last step
  slice_pos = Lo.slices_off;
  for (size_t q = 0; q < items.size(); q++) {
    BatchFilterItem& it = items[q];
    const HamGeometry& g = it.plan->geo;
    float* flag = (float*)(base + Lo.flags_off + 16 * q);
    const size_t sb = ((size_t)g.dim * W * es + 255) & ~(size_t)255;
    for (int col0 = 0; col0 < it.n_b; col0 += W) {
      const int ncols = std::min(W, it.n_b - col0);
      char* ba = base + slice_pos + sb;
      char* bb = base + slice_pos + 2 * sb;
      slice_pos += 3 * sb;
      const void* res = it.K == 0 ? (const void*)ba : (((it.K - 1) & 1) ? (const void*)ba : (const void*)bb);
      PF_CHECK(slice_out(kind, abi_kind, res, g.dim, W, ncols, it.out, it.n_b, col0, flag, s));
    }
  }
  std::vector<float> fl(4 * items.size());
  PF_CUDA(cudaMemcpyAsync(fl.data(), base + Lo.flags_off, 16 * items.size(), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  for (size_t q = 0; q < items.size(); q++) {
    int bad = 0;
    memcpy(&bad, &fl[4 * q + 2], 4);
    double csum = 0.0;
    for (int n = 0; n <= items[q].K; n++) csum += std::fabs(items[q].coef[n]);
    const double bound = csum * items[q].invD * std::sqrt((double)items[q].plan->geo.dim) * fl[4 * q] * 1.01 + 1e-300;
    items[q].bounds_error = bad || (double)fl[4 * q + 1] > bound;
  }
  return POLFED_OK;
}

void cheb_coeffs(double sigma, int K, std::vector<double>& c, double& D) {
  // Eq. (2): c_n = sqrt(4 - 3 delta_{0n}) cos(n arccos sigma); D = sum_n c_n T_n(sigma)
  // with T_n(sigma) = cos(n arccos sigma).  At sigma = 0, cos(n pi/2) is 0, +-1 exactly.
  c.assign(K + 1, 0.0);
  D = 0.0;
  const double phi = std::acos(sigma);
  for (int n = 0; n <= K; n++) {
    double cn;
    if (sigma == 0.0) {
      cn = (n & 1) ? 0.0 : ((n / 2) & 1 ? -1.0 : 1.0);
    } else {
      cn = std::cos(n * phi);
    }
    c[n] = (n == 0 ? 1.0 : 2.0) * cn;
    D += c[n] * cn;
  }
}

// ------------------------------------------------------------- basis kernel
// Unrank: the r-th L-bit string with n_up set bits in ascending order, by the
// combinatorial number system (greedy from the top bit).
__global__ void k_basis(int L, int n_up, uint32_t* states, int64_t dim) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < dim; r += (int64_t)gridDim.x * blockDim.x) {
    uint32_t rem = (uint32_t)r, s = 0;
    int k = n_up;
    for (int p = L - 1; p >= 0 && k > 0; p--) {
      const uint32_t c = c_binom[p][k];  // states with the top set bit below p
      if (rem >= c) {
        s |= 1u << p;
        rem -= c;
        k--;
      }
    }
    states[r] = s;
  }
}

int launch_basis(int L, int n_up, uint32_t* d_states, int64_t dim, cudaStream_t s) {
  upload_binomials();
  if (dim == 0) return POLFED_OK;
  int grid = (int)std::min<int64_t>((dim + 255) / 256, 152 * 32);
  k_basis<<<grid, 256, 0, s>>>(L, n_up, d_states, dim);
  PF_CUDA(cudaGetLastError());
  return POLFED_OK;
}

}  // namespace polfed

// ===================================================================== no-alloc
// polfed_cheb_filter_static: the Chebyshev filter with every table and every
// recurrence buffer carved out of one fixed device array instead of allocated
// memory.  It exists for callers that cannot allocate device memory while they
// run, e.g. code executing inside a memory pool or allocator callback, a
// library embedded in a host application that owns all device allocations, or
// a real-time loop that must not call into the allocator.  The array is a
// file-scope __device__ object: every GPU that loads this library holds it
// (kStaticScratchBytes) until the process exits, whether or not it is used.
namespace polfed {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;  // 32 MiB: dim <= 48620 (L <= 18) at 128-byte slices
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device (host code must not use the
// symbol itself: on the host it names a stand-in, not device memory).
static void* g_static_addr[64] = {nullptr};
static std::mutex g_static_mu;

static int static_scratch_addr(void** out) {
  int dev = 0;
  PF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(POLFED_EINVAL, "device ordinal out of range for the static scratch table");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return fail(POLFED_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return POLFED_OK;
}

// Schedule order of the groups on the device: classes (popcount of s_hi) by
// decreasing group size, groups of a class in ascending s_hi (same order as
// HamPlan::init builds on the host).
__global__ void k_static_order(const HamGeometry g, const int32_t* cls_start, int32_t* order) {
  const int grp = blockIdx.x * blockDim.x + threadIdx.x;
  if (grp >= (1 << g.nh)) return;
  const int pc = __popc(grp);
  const int n_lo = g.n_up - pc;
  if (n_lo < 0 || n_lo > g.b) return;
  uint32_t r = 0;
  int k = 0;
  for (int q = 0; q < g.nh; q++)
    if ((grp >> q) & 1) r += c_binom[q][++k];  // rank among nh-bit strings of popcount pc
  order[cls_start[pc] + (int)r] = grp;
}

// Typed, alpha/beta-scaled diagonal tables (same layout prepare_typed writes).
template <class NT>
__global__ void k_static_typed(const double* F_lo, const double* F_hi, const double* C_x, const int32_t* order,
                               int nlo, int nhi, int ncx, int ngr, double alpha, double beta, typename NT::C* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = nlo + nhi + ncx + ngr;
  if (i >= n) return;
  double v;
  if (i < nlo)
    v = alpha * F_lo[i];
  else if (i < nlo + nhi)
    v = alpha * (F_hi[i - nlo] - beta);
  else if (i < nlo + nhi + ncx)
    v = alpha * C_x[i - nlo - nhi];
  else
    v = alpha * (F_hi[order[i - nlo - nhi - ncx]] - beta);
  out[i] = Conv<NT>::from_d(v);
}

// c_n of Eq. (2) computed on the fly (same expression as cheb_coeffs) or read
// from the caller's array; no storage.
struct CoefSource {
  const double* user;
  double sigma, phi;
  double operator[](int n) const {
    if (user) return user[n];
    const double cn = (sigma == 0.0) ? ((n & 1) ? 0.0 : ((n / 2) & 1 ? -1.0 : 1.0)) : std::cos(n * phi);
    return (n == 0 ? 1.0 : 2.0) * cn;
  }
  double T(int n) const {  // T_n(sigma)
    return (sigma == 0.0) ? ((n & 1) ? 0.0 : ((n / 2) & 1 ? -1.0 : 1.0)) : std::cos(n * phi);
  }
};

static int static_filter(const polfed_model* model, double e_lo, double e_hi, const CoefSource& c, int K, double invD,
                         const void* d_X, void* d_Y, int n_b, int dtype, cudaStream_t s) {
  upload_binomials();
  HamPlan plan;  // borrowed memory: pointers are cleared before it is destroyed
  struct Unborrow {
    HamPlan& p;
    ~Unborrow() {
      p.dev = nullptr;
      for (int k = 0; k < 3; k++) p.typed[k] = nullptr;
    }
  } unborrow{plan};
  PF_CHECK(build_geometry(model, -1, &plan.geo));
  const HamGeometry& g = plan.geo;
  const size_t nlo = (size_t)1 << g.b, nhi = (size_t)1 << g.nh, ncx = (size_t)1 << g.n_cross;
  const int lpr = choose_lpr(dtype, n_b);
  const size_t es_c = dtype == POLFED_F32 ? 4 : 8;
  size_t bytes = 0;
  auto carve = [&](size_t n) {
    size_t o = bytes;
    bytes += (n + 255) & ~(size_t)255;
    return o;
  };
  const size_t oTlo = carve(nlo * 2), oUlo = carve(nlo * 2), oThi = carve(nhi * 4), oOrd = carve(nhi * 4),
               oFlo = carve(nlo * 8), oFhi = carve(nhi * 8), oCx = carve(ncx * 8),
               oRec = carve(nlo * (size_t)g.rec_stride * 2), oGrp = carve((size_t)g.n_groups * sizeof(GroupRec)),
               oErr = carve(64), oCls = carve(34 * 4), oTyp = carve((nlo + nhi + ncx + (size_t)g.n_groups) * es_c),
               oRec8 = carve(nlo * (size_t)g.rec_stride),
               oScr = carve(filter_scratch_bytes(plan, dtype, lpr));
  if (bytes > kStaticScratchBytes)
    return fail(POLFED_ENOMEM, "polfed_cheb_filter_static needs " + std::to_string(bytes) +
                                   " bytes of scratch; the static array holds " + std::to_string(kStaticScratchBytes) +
                                   " (use polfed_cheb_filter for this size)");
  void* base = nullptr;
  PF_CHECK(static_scratch_addr(&base));
  char* d = (char*)base;
  plan.stream = s;
  plan.stream_alloc = false;
  plan.tab.T_lo = (uint16_t*)(d + oTlo);
  plan.tab.U_lo = (uint16_t*)(d + oUlo);
  plan.tab.T_hi = (int32_t*)(d + oThi);
  plan.tab.order = (int32_t*)(d + oOrd);
  plan.tab.F_lo = (double*)(d + oFlo);
  plan.tab.F_hi = (double*)(d + oFhi);
  plan.tab.C_x = (double*)(d + oCx);
  plan.tab.rec = (uint16_t*)(d + oRec);
  plan.tab.grec = (GroupRec*)(d + oGrp);
  plan.tab.rec8 = (uint8_t*)(d + oRec8);
  plan.err_flag = (int*)(d + oErr);
  // group schedule: class start offsets (host arithmetic on fixed arrays only)
  int32_t cls_start[34] = {0};
  {
    int pcs[34], sizes[34], n = 0;
    for (int pc = 0; pc <= g.nh; pc++) {
      const int n_lo = g.n_up - pc;
      if (n_lo < 0 || n_lo > g.b) continue;
      pcs[n] = pc;
      sizes[n] = (int)binom_host(g.b, n_lo);
      n++;
    }
    for (int i = 1; i < n; i++)  // stable insertion sort by decreasing size
      for (int j = i; j > 0 && sizes[j] > sizes[j - 1]; j--) {
        std::swap(sizes[j], sizes[j - 1]);
        std::swap(pcs[j], pcs[j - 1]);
      }
    int pos = 0;
    for (int i = 0; i < n; i++) {
      cls_start[pcs[i]] = pos;
      pos += (int)binom_host(g.nh, pcs[i]);
    }
  }
  int32_t* d_cls = (int32_t*)(d + oCls);
  PF_CUDA(cudaMemcpyAsync(d_cls, cls_start, sizeof(cls_start), cudaMemcpyHostToDevice, s));
  PF_CUDA(cudaMemsetAsync(plan.err_flag, 0, 64, s));
  k_tables_lo<<<(unsigned)((nlo + 255) / 256), 256, 0, s>>>(g, plan.tab.T_lo, plan.tab.U_lo, plan.tab.F_lo);
  k_tables_rec<<<(unsigned)((nlo + 255) / 256), 256, 0, s>>>(g, plan.tab.T_lo, plan.tab.rec);
  k_tables_rec8<<<(unsigned)((nlo + 255) / 256), 256, 0, s>>>(g, plan.tab.rec, plan.tab.rec8);
  k_tables_hi<<<(unsigned)((nhi + 255) / 256), 256, 0, s>>>(g, plan.tab.T_hi, plan.tab.F_hi);
  k_tables_cx<<<(unsigned)((ncx + 255) / 256), 256, 0, s>>>(g, plan.tab.C_x);
  k_static_order<<<(unsigned)((nhi + 255) / 256), 256, 0, s>>>(g, d_cls, plan.tab.order);
  k_tables_groups<<<(unsigned)((g.n_groups + 127) / 128), 128, 0, s>>>(g, plan.tab.T_hi, plan.tab.order, plan.tab.grec);
  PF_CUDA(cudaGetLastError());
  double alpha = 1.0, beta = 0.0;
  if (!(e_lo == 0.0 && e_hi == 0.0)) {
    alpha = 2.0 / (e_hi - e_lo);
    beta = 0.5 * (e_hi + e_lo);
  }
  const int ntyp = (int)(nlo + nhi + ncx) + g.n_groups;
  void* typ = d + oTyp;
  if (dtype == POLFED_F32)
    k_static_typed<NF32><<<(ntyp + 255) / 256, 256, 0, s>>>(plan.tab.F_lo, plan.tab.F_hi, plan.tab.C_x, plan.tab.order,
                                                             (int)nlo, (int)nhi, (int)ncx, g.n_groups, alpha, beta,
                                                             (float*)typ);
  else if (dtype == POLFED_F64)
    k_static_typed<NF64><<<(ntyp + 255) / 256, 256, 0, s>>>(plan.tab.F_lo, plan.tab.F_hi, plan.tab.C_x, plan.tab.order,
                                                             (int)nlo, (int)nhi, (int)ncx, g.n_groups, alpha, beta,
                                                             (double*)typ);
  else
    k_static_typed<NDF><<<(ntyp + 255) / 256, 256, 0, s>>>(plan.tab.F_lo, plan.tab.F_hi, plan.tab.C_x, plan.tab.order,
                                                           (int)nlo, (int)nhi, (int)ncx, g.n_groups, alpha, beta,
                                                           (float2*)typ);
  PF_CUDA(cudaGetLastError());
  plan.typed[dtype] = typ;
  plan.typed_ok[dtype] = true;
  plan.typed_lo[dtype] = e_lo;
  plan.typed_hi[dtype] = e_hi;
  // Clenshaw recurrence, slice by slice (same steps as filter_block)
  FilterScratch scr;
  scr.xs = d + oScr;
  scr.bytes = filter_scratch_bytes(plan, dtype, lpr);
  carve_scratch(scr, plan, dtype, lpr);
  const int W = slice_width(dtype, lpr);
  const int abi = dtype == POLFED_F32 ? POLFED_F32 : POLFED_F64;
  PF_CUDA(cudaMemsetAsync(scr.flag, 0, 16, s));
  for (int col0 = 0; col0 < n_b; col0 += W) {
    const int ncols = std::min(W, n_b - col0);
    if (K == 0) {
      PF_CHECK(slice_in(dtype, abi, d_X, g.dim, n_b, col0, ncols, W, nullptr, scr.ba, nullptr, c[0] * invD, scr.flag, s));
      PF_CHECK(slice_out(dtype, abi, scr.ba, g.dim, W, ncols, d_Y, n_b, col0, scr.flag, s));
      continue;
    }
    PF_CHECK(slice_in(dtype, abi, d_X, g.dim, n_b, col0, ncols, W, scr.xs, scr.ba, scr.bb, c[K], scr.flag, s));
    void* cur = scr.ba;
    void* oth = scr.bb;
    for (int k = K - 1; k >= 1; k--) {
      StepArgs a{cur, oth, scr.xs, oth, c[k], 2.0, (k == K - 1) ? 0.0 : -1.0, lpr};
      PF_CHECK(launch_ham_step(plan, dtype, a, s));
      std::swap(cur, oth);
    }
    StepArgs a{cur, oth, scr.xs, oth, c[0] * invD, invD, (K == 1) ? 0.0 : -invD, lpr};
    PF_CHECK(launch_ham_step(plan, dtype, a, s));
    PF_CHECK(check_timeout(plan, s));
    PF_CHECK(slice_out(dtype, abi, oth, g.dim, W, ncols, d_Y, n_b, col0, scr.flag, s));
  }
  float flag[3] = {0, 0, 0};
  PF_CUDA(cudaMemcpyAsync(flag, scr.flag, sizeof(flag), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  int bad = 0;
  memcpy(&bad, &flag[2], 4);
  double csum = 0.0;
  for (int n = 0; n <= K; n++) csum += std::fabs(c[n]);
  const double bound = csum * invD * std::sqrt((double)g.dim) * (double)flag[0] * 1.01 + 1e-300;
  if (bad || (double)flag[1] > bound)
    return fail(POLFED_EBOUNDS, "filter output grew beyond the Chebyshev bound: spectrum outside [e_lo, e_hi]");
  return POLFED_OK;
}

}  // namespace polfed

extern "C" int polfed_set_wait_limit(uint32_t polls) {
  polfed::g_wait_limit.store(polls);
  return POLFED_OK;
}

extern "C" int polfed_cheb_filter_static(const polfed_model* model, const uint32_t* d_states, int64_t dim,
                                         double e_lo, double e_hi, double sigma, int32_t K, const double* coeffs,
                                         const void* d_X, void* d_Y, int32_t n_b, int32_t dtype,
                                         polfed_stream_t stream) {
  using namespace polfed;
  clear_error();
  if (!model) return fail(POLFED_EINVAL, "model is NULL");
  if (model->L < 4 || model->L > 32 || (model->L & 1)) return fail(POLFED_EINVAL, "L must be even, 4 <= L <= 32");
  if (dim != (int64_t)binom_host(model->L, model->L / 2)) return fail(POLFED_EINVAL, "dim != C(L, L/2)");
  if (!d_states || !d_X || !d_Y) return fail(POLFED_EINVAL, "NULL device pointer");
  if (n_b < 1 || n_b > 128) return fail(POLFED_EINVAL, "n_b must be in 1..128");
  if (dtype != POLFED_F32 && dtype != POLFED_F64 && dtype != POLFED_DF64) return fail(POLFED_EINVAL, "bad dtype");
  {
    const size_t es = dtype == POLFED_F32 ? 4 : 8;
    const char* x = (const char*)d_X;
    const char* y = (const char*)d_Y;
    const size_t nbytes = (size_t)dim * n_b * es;
    if (x < y + nbytes && y < x + nbytes) return fail(POLFED_EINVAL, "X and Y must not overlap");
  }
  if (!std::isfinite(e_lo) || !std::isfinite(e_hi) || (!(e_lo == 0.0 && e_hi == 0.0) && !(e_lo < e_hi)))
    return fail(POLFED_EINVAL, "need e_lo < e_hi (or both 0)");
  if (K < 0 || K > 10000000) return fail(POLFED_EINVAL, "K must be in 0..1e7");
  if (!coeffs && !(sigma > -1.0 && sigma < 1.0)) return fail(POLFED_EINVAL, "sigma must be in (-1, 1)");
  CoefSource c{coeffs, sigma, coeffs ? 0.0 : std::acos(sigma)};
  double invD = 1.0;
  if (coeffs) {
    for (int n = 0; n <= K; n++)
      if (!std::isfinite(coeffs[n])) return fail(POLFED_EINVAL, "non-finite coefficient");
  } else {
    double D = 0.0;
    for (int n = 0; n <= K; n++) D += c[n] * c.T(n);
    invD = 1.0 / D;
  }
  return static_filter(model, e_lo, e_hi, c, K, invD, d_X, d_Y, n_b, dtype, (cudaStream_t)stream);
}
