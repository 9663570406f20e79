// Stage 2 of the two-stage method on the GPU: the primal-dual interior point
// method of Sec. 3 with the transition of Sec. 4 (Alg. "alg:fast" after its
// stage 1), for min 1/2||XY - M||^2 s.t. X, Y >= 0 on a handle's resident
// window.  FP64 throughout.  The Newton direction of eq. "eqn:equation" is
// formed as in Sec. 3.2: the reduced system eq. "eqn:p"
//   [R1  Cb^T; Cb  R2] [dx; dy] = -grad phi,
//   R1 = blkdiag_n(Y Y^T) + rho I + Diag(x)^-1 Diag(r),
//   R2 = blkdiag_m(X^T X) + rho I + Diag(y)^-1 Diag(s),
// block-Cholesky R1 = P^T P (n independent k x k blocks, one thread each),
// W = Cb P^-1 (one thread per (column, row) block), the Schur complement
// R2 - W W^T (mk x mk, one thread per entry) and its dense Cholesky and
// triangular solves (one CTA), then dx by back substitution (eqs.
// "eqn:step", "eqn:step2") and dr, ds from the complementarity rows.  The
// outer loop on mu, the inner Newton loop with the fraction-to-boundary rule,
// Armijo backtracking on the barrier merit function, the predictor-based
// sigma and the Hessian switch follow Sec. 3-4 step by step on the host, every
// vector operation and reduction in the kernels below (fixed-order sums).
// Sizes: the dense Schur matrix limits m k (see nmf.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "nmf.h"
#include "nmf_internal.h"

using namespace nmfgb;

namespace {

constexpr int RT = 1024;   // threads of the one-block reductions and of the dense solve

// ---------------------------------------------------------------------------
// residual, objective and gradients of eq. "eqn:kkt"
// ---------------------------------------------------------------------------
template <typename TM>
__device__ __forceinline__ double mval(const TM* M, int ld, int head, int mcap, int i, int j) {
  int ph = head + j;
  if (ph >= mcap) ph -= mcap;
  return (double)M[(size_t)ph * ld + i];
}

// Per row i: graX_i = sum_j (x_i . y_j - M_ij) y_j and the row's part of
// 1/2 ||XY - M||^2 (columns in order).
template <typename TM>
__global__ void ipm_grad_rows(const TM* M, int ld, int head, int mcap, int n, int m, int k, const double* x,
                              const double* y, double* gX, double* frow) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double g[KMAX];
  for (int a = 0; a < k; ++a) g[a] = 0.0;
  double f = 0.0;
  for (int j = 0; j < m; ++j) {
    double res = -mval(M, ld, head, mcap, i, j);
    for (int a = 0; a < k; ++a) res = fma(x[(size_t)i * k + a], y[(size_t)j * k + a], res);
    f = fma(0.5 * res, res, f);
    for (int a = 0; a < k; ++a) g[a] = fma(res, y[(size_t)j * k + a], g[a]);
  }
  for (int a = 0; a < k; ++a) gX[(size_t)i * k + a] = g[a];
  frow[i] = f;
}

// Per column j: graY_j = sum_i x_i (x_i . y_j - M_ij) (rows in order).
template <typename TM>
__global__ void ipm_grad_cols(const TM* M, int ld, int head, int mcap, int n, int m, int k, const double* x,
                              const double* y, double* gY) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double g[KMAX];
  for (int a = 0; a < k; ++a) g[a] = 0.0;
  for (int i = 0; i < n; ++i) {
    double res = -mval(M, ld, head, mcap, i, j);
    for (int a = 0; a < k; ++a) res = fma(x[(size_t)i * k + a], y[(size_t)j * k + a], res);
    for (int a = 0; a < k; ++a) g[a] = fma(x[(size_t)i * k + a], res, g[a]);
  }
  for (int a = 0; a < k; ++a) gY[(size_t)j * k + a] = g[a];
}

// Objective only, per row (Armijo trials): 1/2 sum_j (x_i . y_j - M_ij)^2.
template <typename TM>
__global__ void ipm_obj_rows(const TM* M, int ld, int head, int mcap, int n, int m, int k, const double* x,
                             const double* y, double* frow) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f = 0.0;
  for (int j = 0; j < m; ++j) {
    double res = -mval(M, ld, head, mcap, i, j);
    for (int a = 0; a < k; ++a) res = fma(x[(size_t)i * k + a], y[(size_t)j * k + a], res);
    f = fma(0.5 * res, res, f);
  }
  frow[i] = f;
}

// ---------------------------------------------------------------------------
// one-block reductions (fixed order: strided per-thread sums, then a tree)
// ---------------------------------------------------------------------------
__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}
__device__ double block_min(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}
__device__ double block_max(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// out[0] = sum of a (the row parts of f)
__global__ void ipm_sum(const double* a, long long N, double* out) {
  __shared__ double sh[RT];
  double t = 0.0;
  for (long long q = threadIdx.x; q < N; q += blockDim.x) t += a[q];
  const double r = block_sum(t, sh);
  if (threadIdx.x == 0) out[0] = r;
}

// E(x, y, r, s; mu) of eq. "error": out[0] += sum (g - r)^2, out[1] += sum (r x - mu)^2
// over one block of variables (x, gX, r) or (y, gY, s); acc selects accumulate.
__global__ void ipm_err_terms(const double* v, const double* g, const double* d, long long N, double mu,
                              double* out, int acc) {
  __shared__ double sh[RT];
  double a = 0.0, c = 0.0;
  for (long long q = threadIdx.x; q < N; q += blockDim.x) {
    a += (g[q] - d[q]) * (g[q] - d[q]);
    c += (d[q] * v[q] - mu) * (d[q] * v[q] - mu);
  }
  const double ra = block_sum(a, sh), rc = block_sum(c, sh);
  if (threadIdx.x == 0) {
    out[0] = acc ? out[0] + ra : ra;
    out[1] = acc ? out[1] + rc : rc;
  }
}

// out[0] = max |g| over N values, out[1] = max v (transition)
__global__ void ipm_maxes(const double* g, const double* v, long long N, double* out) {
  __shared__ double sh[RT];
  double a = 0.0, b = 0.0;
  for (long long q = threadIdx.x; q < N; q += blockDim.x) {
    a = fmax(a, fabs(g[q]));
    b = fmax(b, v[q]);
  }
  const double ra = block_max(a, sh), rb = block_max(b, sh);
  if (threadIdx.x == 0) {
    out[0] = ra;
    out[1] = rb;
  }
}

// v := max(v, floor) elementwise (the transition's rho0)
__global__ void ipm_floor(double* v, long long N, double floor_v) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x)
    if (v[q] < floor_v) v[q] = floor_v;
}

__global__ void ipm_fill(double* v, long long N, double val) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x)
    v[q] = val;
}

// out[0] = sum a_q b_q, out[1] = sum v_q w_q (two dot products at once)
__global__ void ipm_dot2(const double* a, const double* b, long long Na, const double* v, const double* w,
                         long long Nv, double* out) {
  __shared__ double sh[RT];
  double s1 = 0.0, s2 = 0.0;
  for (long long q = threadIdx.x; q < Na; q += blockDim.x) s1 += a[q] * b[q];
  for (long long q = threadIdx.x; q < Nv; q += blockDim.x) s2 += v[q] * w[q];
  const double r1 = block_sum(s1, sh), r2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    out[0] = r1;
    out[1] = r2;
  }
}

// slope of phi along (dx, dy): sum dx (gX - mu/x) + sum dy (gY - mu/y)
__global__ void ipm_slope(const double* dx, const double* gX, const double* x, long long nk, const double* dy,
                          const double* gY, const double* y, long long mk, double mu, double* out) {
  __shared__ double sh[RT];
  double t = 0.0, u = 0.0;
  for (long long q = threadIdx.x; q < nk; q += blockDim.x) t += dx[q] * (gX[q] - mu / x[q]);
  for (long long q = threadIdx.x; q < mk; q += blockDim.x) u += dy[q] * (gY[q] - mu / y[q]);
  const double r = block_sum(t, sh), r2 = block_sum(u, sh);
  if (threadIdx.x == 0) out[0] = r + r2;
}

// fraction to the boundary: min(1, min over dv < 0 of -tau v / dv), for two
// vectors (v1, dv1) and (v2, dv2) at once: out[0], out[1]
__global__ void ipm_frac2(const double* v1, const double* dv1, long long N1, const double* v2, const double* dv2,
                          long long N2, double tau, double* out) {
  __shared__ double sh[RT];
  double a = 1.0, b = 1.0;
  for (long long q = threadIdx.x; q < N1; q += blockDim.x)
    if (dv1[q] < 0.0) a = fmin(a, -tau * v1[q] / dv1[q]);
  for (long long q = threadIdx.x; q < N2; q += blockDim.x)
    if (dv2[q] < 0.0) b = fmin(b, -tau * v2[q] / dv2[q]);
  const double ra = block_min(a, sh), rb = block_min(b, sh);
  if (threadIdx.x == 0) {
    out[0] = ra;
    out[1] = rb;
  }
}

// barrier part of phi: out[0] = sum log x + sum log y, out[1] = 1 if some
// entry is not positive (phi = +inf there)
__global__ void ipm_logs(const double* x, long long nk, const double* y, long long mk, double* out) {
  __shared__ double sh[RT];
  double t = 0.0, bad = 0.0;
  for (long long q = threadIdx.x; q < nk; q += blockDim.x) {
    if (!(x[q] > 0.0)) bad = 1.0;
    else t += log(x[q]);
  }
  for (long long q = threadIdx.x; q < mk; q += blockDim.x) {
    if (!(y[q] > 0.0)) bad = 1.0;
    else t += log(y[q]);
  }
  const double r = block_sum(t, sh), rb = block_max(bad, sh);
  if (threadIdx.x == 0) {
    out[0] = r;
    out[1] = rb;
  }
}

// out = v + a dv
__global__ void ipm_axpy(double* out, const double* v, double a, const double* dv, long long N) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x)
    out[q] = v[q] + a * dv[q];
}

// predictor: out[0] = sum (v + a1 dv)(w + a2 dw), out[1] = sum v w, over two blocks
__global__ void ipm_mu_aff(const double* x, const double* dx, const double* r, const double* dr, long long nk,
                           const double* y, const double* dy, const double* s, const double* ds, long long mk,
                           double a1, double a2, double* out) {
  __shared__ double sh[RT];
  double t = 0.0, c = 0.0;
  for (long long q = threadIdx.x; q < nk; q += blockDim.x) {
    t += (x[q] + a1 * dx[q]) * (r[q] + a2 * dr[q]);
    c += x[q] * r[q];
  }
  for (long long q = threadIdx.x; q < mk; q += blockDim.x) {
    t += (y[q] + a1 * dy[q]) * (s[q] + a2 * ds[q]);
    c += y[q] * s[q];
  }
  const double rt = block_sum(t, sh), rc = block_sum(c, sh);
  if (threadIdx.x == 0) {
    out[0] = rt;
    out[1] = rc;
  }
}

// ---------------------------------------------------------------------------
// the Newton direction (Sec. 3.2)
// ---------------------------------------------------------------------------
// YY = Y Y^T and XX = X^T X (k x k each; one thread per entry)
__global__ void ipm_grams(const double* x, const double* y, int n, int m, int k, double* YY, double* XX) {
  const int e = threadIdx.x;
  if (e >= k * k) return;
  const int a = e / k, c = e % k;
  double t1 = 0.0, t2 = 0.0;
  for (int j = 0; j < m; ++j) t1 += y[(size_t)j * k + a] * y[(size_t)j * k + c];
  for (int i = 0; i < n; ++i) t2 += x[(size_t)i * k + a] * x[(size_t)i * k + c];
  YY[e] = t1;
  XX[e] = t2;
}

// Per row i: the block R1_i = YY + diag(rho + r_i / x_i) = L_i L_i^T (Cholesky,
// lower factor into L1[i]) and u_i = L_i^-1 b1_i with b1 = -(gX - mu / x).
__global__ void ipm_blocks(const double* x, const double* r, const double* gX, const double* YY, double rho,
                           double mu, int n, int k, double* L1, double* u, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* L = L1 + (size_t)i * k * k;
  for (int a = 0; a < k; ++a)
    for (int c = 0; c < k; ++c)
      L[a * k + c] = YY[a * k + c] + (a == c ? rho + r[(size_t)i * k + a] / x[(size_t)i * k + a] : 0.0);
  for (int c = 0; c < k; ++c) {
    double s = L[c * k + c];
    for (int l = 0; l < c; ++l) s -= L[c * k + l] * L[c * k + l];
    if (!(s > 0.0) || !isfinite(s)) {
      atomicExch(status, 1);
      return;
    }
    const double d = sqrt(s);
    L[c * k + c] = d;
    for (int rr = c + 1; rr < k; ++rr) {
      double t = L[rr * k + c];
      for (int l = 0; l < c; ++l) t -= L[rr * k + l] * L[c * k + l];
      L[rr * k + c] = t / d;
    }
  }
  for (int a = 0; a < k; ++a) {
    double t = -(gX[(size_t)i * k + a] - mu / x[(size_t)i * k + a]);
    for (int l = 0; l < a; ++l) t -= L[a * k + l] * u[(size_t)i * k + l];
    u[(size_t)i * k + a] = t / L[a * k + a];
  }
}

// W = Cb P^-1: for column j and row i, the k x k block whose row (j, a) solves
// L_i w = c with c_b = x_ia y_jb (+ the residual when a == b and full).
template <typename TM>
__global__ void ipm_W(const TM* M, int ld, int head, int mcap, const double* x, const double* y, const double* L1,
                      int n, int m, int k, int full, double* W) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * m) return;
  const int i = (int)(t % n), j = (int)(t / n);
  const long long nk = (long long)n * k;
  const double* L = L1 + (size_t)i * k * k;
  double res = -mval(M, ld, head, mcap, i, j);
  for (int a = 0; a < k; ++a) res = fma(x[(size_t)i * k + a], y[(size_t)j * k + a], res);
  for (int a = 0; a < k; ++a) {
    double* wrow = W + ((size_t)j * k + a) * nk + (size_t)i * k;
    for (int b = 0; b < k; ++b) {
      double cab = x[(size_t)i * k + a] * y[(size_t)j * k + b];
      if (full && a == b) cab += res;
      double tt = cab;
      for (int l = 0; l < b; ++l) tt -= L[b * k + l] * wrow[l];
      wrow[b] = tt / L[b * k + b];
    }
  }
}

// Schur matrix S = R2 - W W^T (one thread per entry) with
// R2 = blkdiag(XX) + diag(rho + s / y)
__global__ void ipm_schur(const double* W, const double* XX, const double* y, const double* s, double rho, int mk,
                          long long nk, int k, double* S) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)mk * mk) return;
  const int p1 = (int)(t / mk), p2 = (int)(t % mk);
  const int j1 = p1 / k, a1 = p1 % k, j2 = p2 / k, a2 = p2 % k;
  double v = 0.0;
  if (j1 == j2) v = XX[a1 * k + a2] + (a1 == a2 ? rho + s[p1] / y[p1] : 0.0);
  const double* w1 = W + (size_t)p1 * nk;
  const double* w2 = W + (size_t)p2 * nk;
  for (long long q = 0; q < nk; ++q) v -= w1[q] * w2[q];
  S[t] = v;
}

// rhs = b2 - W u, b2 = -(gY - mu / y) (one thread per row of W)
__global__ void ipm_rhs(const double* W, const double* u, const double* gY, const double* y, double mu, int mk,
                        long long nk, double* rhs) {
  const int p1 = blockIdx.x * blockDim.x + threadIdx.x;
  if (p1 >= mk) return;
  double t = -(gY[p1] - mu / y[p1]);
  const double* w1 = W + (size_t)p1 * nk;
  for (long long q = 0; q < nk; ++q) t -= w1[q] * u[q];
  rhs[p1] = t;
}

// Dense Cholesky of the mk x mk Schur matrix (lower factor, in place, column
// by column) and the two triangular solves L L^T dy = rhs: one CTA.
__global__ void ipm_chol_solve(double* S, const double* rhs, int mk, double* dy, int* status) {
  __shared__ double sh[RT];
  __shared__ double sd;
  for (int c = 0; c < mk; ++c) {
    double t = 0.0;
    for (int l = threadIdx.x; l < c; l += blockDim.x) t += S[(size_t)c * mk + l] * S[(size_t)c * mk + l];
    const double sum = block_sum(t, sh);
    if (threadIdx.x == 0) {
      const double v = S[(size_t)c * mk + c] - sum;
      sd = (v > 0.0 && isfinite(v)) ? sqrt(v) : -1.0;
      if (sd > 0.0) S[(size_t)c * mk + c] = sd;
    }
    __syncthreads();
    const double d = sd;
    if (!(d > 0.0)) {
      if (threadIdx.x == 0) atomicExch(status, 2);
      return;
    }
    for (int rr = c + 1 + threadIdx.x; rr < mk; rr += blockDim.x) {
      double tt = S[(size_t)rr * mk + c];
      for (int l = 0; l < c; ++l) tt -= S[(size_t)rr * mk + l] * S[(size_t)c * mk + l];
      S[(size_t)rr * mk + c] = tt / d;
    }
    __syncthreads();
  }
  // L v = rhs
  for (int c = 0; c < mk; ++c) {
    double t = 0.0;
    for (int l = threadIdx.x; l < c; l += blockDim.x) t += S[(size_t)c * mk + l] * dy[l];
    const double sum = block_sum(t, sh);
    if (threadIdx.x == 0) dy[c] = (rhs[c] - sum) / S[(size_t)c * mk + c];
    __syncthreads();
  }
  // L^T dy = v
  for (int c = mk - 1; c >= 0; --c) {
    double t = 0.0;
    for (int l = c + 1 + threadIdx.x; l < mk; l += blockDim.x) t += S[(size_t)l * mk + c] * dy[l];
    const double sum = block_sum(t, sh);
    if (threadIdx.x == 0) dy[c] = (dy[c] - sum) / S[(size_t)c * mk + c];
    __syncthreads();
  }
}

// dx = P^-1 (u - W^T dy) = L_i^-T (u_i - (W^T dy)_i), one thread per row i
__global__ void ipm_dx(const double* W, const double* u, const double* dy, const double* L1, int n, int k, int mk,
                       long long nk, double* dx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v[KMAX];
  for (int a = 0; a < k; ++a) {
    const long long q = (long long)i * k + a;
    double t = u[q];
    for (int p1 = 0; p1 < mk; ++p1) t -= W[(size_t)p1 * nk + q] * dy[p1];
    v[a] = t;
  }
  const double* L = L1 + (size_t)i * k * k;
  for (int a = k - 1; a >= 0; --a) {
    double t = v[a];
    for (int l = a + 1; l < k; ++l) t -= L[l * k + a] * v[l];
    v[a] = t / L[a * k + a];
  }
  for (int a = 0; a < k; ++a) dx[(size_t)i * k + a] = v[a];
}

// the complementarity rows: Diag(r) dx + Diag(x) dr = mu e - Diag(r) x (and y, s)
__global__ void ipm_duals(const double* x, const double* r, const double* dx, long long nk, const double* y,
                          const double* s, const double* dy, long long mk, double mu, double* dr, double* ds) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nk + mk;
       q += (long long)gridDim.x * blockDim.x) {
    if (q < nk) dr[q] = mu / x[q] - r[q] - r[q] / x[q] * dx[q];
    else {
      const long long p = q - nk;
      ds[p] = mu / y[p] - s[p] - s[p] / y[p] * dy[p];
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Ipm {
  nmf_handle* h;
  HandleInfo hi{};
  Problem p{};
  cudaStream_t st = nullptr;
  int n = 0, m = 0, k = 0;
  long long nk = 0, mk = 0;
  std::vector<void*> bufs;
  double *x, *y, *r, *s, *gX, *gY, *dx, *dy, *dr, *ds, *xt, *yt, *frow, *YY, *XX, *L1, *u, *W, *S, *rhs, *red;
  int* status;
  double hred[4];
  cudaError_t err = cudaSuccess;

  template <typename T>
  T* alloc(size_t count) {
    void* ptr = nullptr;
    if (err == cudaSuccess) err = cudaMalloc(&ptr, sizeof(T) * std::max<size_t>(count, 1));
    if (ptr) bufs.push_back(ptr);
    return static_cast<T*>(ptr);
  }
  ~Ipm() {
    for (void* b : bufs) cudaFree(b);
  }
  int grid(long long N) const { return (int)std::max<long long>(1, std::min<long long>((N + 255) / 256, 4096)); }
  void fetch(int count) {
    if (err == cudaSuccess) err = cudaMemcpyAsync(hred, red, sizeof(double) * count, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  }
  template <typename F>
  void onM(F&& f) {
    if (hi.store_f32) f(static_cast<const float*>(p.M));
    else f(static_cast<const double*>(p.M));
  }
  // gradients at (x, y) and f
  double grad() {
    onM([&](auto M) {
      ipm_grad_rows<<<grid(n), 256, 0, st>>>(M, hi.ld, p.head, hi.mcap, n, m, k, x, y, gX, frow);
      ipm_grad_cols<<<grid(m), 256, 0, st>>>(M, hi.ld, p.head, hi.mcap, n, m, k, x, y, gY);
    });
    ipm_sum<<<1, RT, 0, st>>>(frow, n, red);
    fetch(1);
    return hred[0];
  }
  double objective(const double* xv, const double* yv) {
    onM([&](auto M) { ipm_obj_rows<<<grid(n), 256, 0, st>>>(M, hi.ld, p.head, hi.mcap, n, m, k, xv, yv, frow); });
    ipm_sum<<<1, RT, 0, st>>>(frow, n, red);
    fetch(1);
    return hred[0];
  }
  // E(.; mu) of eq. "error" at (x, y, r, s) with the current gradients
  double error(double mu) {
    ipm_err_terms<<<1, RT, 0, st>>>(x, gX, r, nk, mu, red, 0);
    ipm_err_terms<<<1, RT, 0, st>>>(y, gY, s, mk, mu, red, 1);
    fetch(2);
    return std::max(std::sqrt(hred[0]), std::sqrt(hred[1]));
  }
  // phi = f - mu (sum log x + sum log y); +inf outside x, y > 0
  double phi(const double* xv, const double* yv, double mu) {
    ipm_logs<<<1, RT, 0, st>>>(xv, nk, yv, mk, red + 2);
    const double f = objective(xv, yv);
    if (err == cudaSuccess) err = cudaMemcpyAsync(hred + 2, red + 2, sizeof(double) * 2, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (hred[3] > 0.0) return INFINITY;
    return f - mu * hred[2];
  }
  // the direction; returns 0, 1 (block not PD), 2 (Schur matrix not PD)
  int direction(double mu, double rho, int full) {
    if (err == cudaSuccess) err = cudaMemsetAsync(status, 0, sizeof(int), st);
    ipm_grams<<<1, 256, 0, st>>>(x, y, n, m, k, YY, XX);
    ipm_blocks<<<grid(n), 256, 0, st>>>(x, r, gX, YY, rho, mu, n, k, L1, u, status);
    onM([&](auto M) {
      ipm_W<<<grid((long long)n * m), 256, 0, st>>>(M, hi.ld, p.head, hi.mcap, x, y, L1, n, m, k, full, W);
    });
    ipm_schur<<<grid(mk * mk), 256, 0, st>>>(W, XX, y, s, rho, (int)mk, nk, k, S);
    ipm_rhs<<<grid(mk), 256, 0, st>>>(W, u, gY, y, mu, (int)mk, nk, rhs);
    ipm_chol_solve<<<1, RT, 0, st>>>(S, rhs, (int)mk, dy, status);
    ipm_dx<<<grid(n), 256, 0, st>>>(W, u, dy, L1, n, k, (int)mk, nk, dx);
    ipm_duals<<<grid(nk + mk), 256, 0, st>>>(x, r, dx, nk, y, s, dy, mk, mu, dr, ds);
    int hs = 0;
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    return hs;
  }
  double slope(double mu) {
    ipm_slope<<<1, RT, 0, st>>>(dx, gX, x, nk, dy, gY, y, mk, mu, red);
    fetch(1);
    return hred[0];
  }
  void frac(const double* v1, const double* d1, const double* v2, const double* d2, double tau, double* a) {
    ipm_frac2<<<1, RT, 0, st>>>(v1, d1, nk, v2, d2, mk, tau, red);
    fetch(2);
    *a = std::min(hred[0], hred[1]);
  }
};

bool ipm_sizes_ok(int n, int m, int k) {
  const long long nk = (long long)n * k, mk = (long long)m * k;
  return k >= 1 && k <= KMAX && mk <= 4096 && nk * mk <= (1ll << 27);
}

// Set up the work arrays and the current iterate (logical column order).
nmf_status ipm_setup(nmf_handle* h, Ipm& w) {
  w.h = h;
  if (!handle_info(h, &w.hi)) return NMF_EINVAL;
  if (!w.hi.factors_set) return handle_fail(h, NMF_ESTATE, "factors not set");
  nmf_status s = handle_sync_state(h);
  if (s != NMF_OK) return s;
  const int var = w.hi.store_f32 ? VAR_F32 : VAR_F64;
  if (!handle_problem(h, var, &w.p)) return NMF_EINVAL;
  w.st = w.hi.stream;
  w.n = w.hi.n;
  w.m = w.hi.m;
  w.k = w.hi.k;
  w.nk = (long long)w.n * w.k;
  w.mk = (long long)w.m * w.k;
  if (!ipm_sizes_ok(w.n, w.m, w.k)) return handle_fail(h, NMF_ECAPACITY, "stage 2: m k or n m k^2 too large");
  w.x = w.alloc<double>(w.nk);
  w.y = w.alloc<double>(w.mk);
  w.r = w.alloc<double>(w.nk);
  w.s = w.alloc<double>(w.mk);
  w.gX = w.alloc<double>(w.nk);
  w.gY = w.alloc<double>(w.mk);
  w.dx = w.alloc<double>(w.nk);
  w.dy = w.alloc<double>(w.mk);
  w.dr = w.alloc<double>(w.nk);
  w.ds = w.alloc<double>(w.mk);
  w.xt = w.alloc<double>(w.nk);
  w.yt = w.alloc<double>(w.mk);
  w.frow = w.alloc<double>(w.n);
  w.YY = w.alloc<double>(w.k * w.k);
  w.XX = w.alloc<double>(w.k * w.k);
  w.L1 = w.alloc<double>((size_t)w.n * w.k * w.k);
  w.u = w.alloc<double>(w.nk);
  w.W = w.alloc<double>((size_t)(w.mk * w.nk));
  w.S = w.alloc<double>((size_t)(w.mk * w.mk));
  w.rhs = w.alloc<double>(w.mk);
  w.red = w.alloc<double>(4);
  w.status = w.alloc<int>(1);
  if (w.err != cudaSuccess) return handle_fail(h, NMF_ENOMEM, "stage 2: device allocation failed");
  const int cur = w.hi.hSt->iter & 1;
  // the iterate in logical column order (the ring is read through head)
  cudaError_t e = cudaMemcpyAsync(w.x, w.p.X[cur], sizeof(double) * w.nk, cudaMemcpyDeviceToDevice, w.st);
  const int first = std::min(w.m, w.hi.mcap - w.p.head);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w.y, w.p.Y[cur] + (size_t)w.p.head * w.k, sizeof(double) * first * w.k,
                        cudaMemcpyDeviceToDevice, w.st);
  if (e == cudaSuccess && first < w.m)
    e = cudaMemcpyAsync(w.y + (size_t)first * w.k, w.p.Y[cur], sizeof(double) * (w.m - first) * w.k,
                        cudaMemcpyDeviceToDevice, w.st);
  if (e != cudaSuccess) return handle_fail(h, NMF_ECUDA, cudaGetErrorString(e));
  return NMF_OK;
}

}  // namespace

extern "C" {

nmf_status nmf_ipm_direction(nmf_handle* h, const double* r, const double* s, double mu, double rho,
                             int32_t full, double* dx, double* dy, double* dr, double* ds, int32_t on_device) {
  if (!h || !r || !s || !dx || !dy || !dr || !ds || !(mu >= 0.0) || !(rho >= 0.0)) return NMF_EINVAL;
  Ipm w;
  nmf_status st = ipm_setup(h, w);
  if (st != NMF_OK) return st;
  const cudaMemcpyKind in = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind out = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaMemcpyAsync(w.r, r, sizeof(double) * w.nk, in, w.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.s, s, sizeof(double) * w.mk, in, w.st);
  if (e != cudaSuccess) return handle_fail(h, NMF_ECUDA, cudaGetErrorString(e));
  w.grad();
  const int ds_ = w.direction(mu, rho, full ? 1 : 0);
  if (w.err != cudaSuccess) return handle_fail(h, NMF_ECUDA, cudaGetErrorString(w.err));
  if (ds_) return handle_fail(h, NMF_ENUMERIC, "stage 2: a Cholesky factorisation failed (not positive definite)");
  e = cudaMemcpyAsync(dx, w.dx, sizeof(double) * w.nk, out, w.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dy, w.dy, sizeof(double) * w.mk, out, w.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dr, w.dr, sizeof(double) * w.nk, out, w.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ds, w.ds, sizeof(double) * w.mk, out, w.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(w.st);
  if (e != cudaSuccess) return handle_fail(h, NMF_ECUDA, cudaGetErrorString(e));
  return NMF_OK;
}

nmf_status nmf_ipm(nmf_handle* h, double eps_tol, int32_t max_newton, double* stats) {
  if (!h || !(eps_tol > 0.0) || max_newton < 1) return NMF_EINVAL;
  Ipm w;
  nmf_status st = ipm_setup(h, w);
  if (st != NMF_OK) return st;
  const double tau = 0.9, eta = 0.5, sigma_c = 0.01;
  const long long nk = w.nk, mk = w.mk;
  // transition (Sec. 4): (x, y) := max{(x, y), rho0}, rho0 = 1e-6 max(x, y);
  // r = max|graX| e, s = max|graY| e; mu the mean complementarity; rho = eps_TOL
  ipm_maxes<<<1, RT, 0, w.st>>>(w.x, w.x, nk, w.red);
  w.fetch(2);
  double vmax = w.hred[1];
  ipm_maxes<<<1, RT, 0, w.st>>>(w.y, w.y, mk, w.red);
  w.fetch(2);
  vmax = std::max(vmax, w.hred[1]);
  const double rho0 = 1e-6 * vmax;
  ipm_floor<<<w.grid(nk), 256, 0, w.st>>>(w.x, nk, rho0);
  ipm_floor<<<w.grid(mk), 256, 0, w.st>>>(w.y, mk, rho0);
  w.grad();
  ipm_maxes<<<1, RT, 0, w.st>>>(w.gX, w.x, nk, w.red);
  w.fetch(2);
  double gxm = w.hred[0];
  ipm_maxes<<<1, RT, 0, w.st>>>(w.gY, w.y, mk, w.red);
  w.fetch(2);
  double gym = w.hred[0];
  if (!(gxm > 0.0)) gxm = 2.220446049250313e-16;
  if (!(gym > 0.0)) gym = 2.220446049250313e-16;
  ipm_fill<<<w.grid(nk), 256, 0, w.st>>>(w.r, nk, gxm);
  ipm_fill<<<w.grid(mk), 256, 0, w.st>>>(w.s, mk, gym);
  ipm_dot2<<<1, RT, 0, w.st>>>(w.x, w.r, nk, w.y, w.s, mk, w.red);
  w.fetch(2);
  double mu = (w.hred[0] + w.hred[1]) / (double)(nk + mk);
  const double rho = eps_tol;
  bool flag = false;
  double E0 = 0.0;
  int it = 0, outer = 0, nfull = 0, nfail = 0;
  nmf_status result = NMF_OK;
  for (outer = 0;; ++outer) {
    w.grad();
    E0 = w.error(0.0);
    if (E0 <= eps_tol) break;
    if (it >= max_newton || outer >= max_newton) {
      result = NMF_ENOTCONV;
      break;
    }
    const double eps_mu = mu;
    for (;;) {
      w.grad();
      const double e_mu = w.error(mu);
      if (e_mu <= eps_mu) break;
      if (it >= max_newton) {
        result = NMF_ENOTCONV;
        break;
      }
      bool used_full = false;
      double slope = 0.0;
      if (flag) {
        const int dst = w.direction(mu, rho, 1);
        if (dst == 0) slope = w.slope(mu);
        if (dst != 0 || !(slope < 0.0)) flag = false;
        else used_full = true;
      }
      if (!used_full) {
        if (w.direction(mu, rho, 0) != 0) {
          result = NMF_ENUMERIC;
          break;
        }
        slope = w.slope(mu);
      }
      double a1 = 1.0, a2 = 1.0;
      w.frac(w.x, w.dx, w.y, w.dy, tau, &a1);
      // dual step: r with dr over nk entries, s with ds over mk entries
      ipm_frac2<<<1, RT, 0, w.st>>>(w.r, w.dr, nk, w.s, w.ds, mk, tau, w.red);
      w.fetch(2);
      a2 = std::min(w.hred[0], w.hred[1]);
      const double phi0 = w.phi(w.x, w.y, mu);
      bool accepted = false;
      for (int bt = 0; bt < 60; ++bt, a1 *= 0.5) {
        ipm_axpy<<<w.grid(nk), 256, 0, w.st>>>(w.xt, w.x, a1, w.dx, nk);
        ipm_axpy<<<w.grid(mk), 256, 0, w.st>>>(w.yt, w.y, a1, w.dy, mk);
        const double phi1 = w.phi(w.xt, w.yt, mu);
        if (phi1 <= phi0 + eta * a1 * slope) {
          accepted = true;
          break;
        }
      }
      if (!accepted) {
        ++nfail;
        a1 = 0.0;
      }
      ipm_axpy<<<w.grid(nk), 256, 0, w.st>>>(w.x, w.x, a1, w.dx, nk);
      ipm_axpy<<<w.grid(mk), 256, 0, w.st>>>(w.y, w.y, a1, w.dy, mk);
      ipm_axpy<<<w.grid(nk), 256, 0, w.st>>>(w.r, w.r, a2, w.dr, nk);
      ipm_axpy<<<w.grid(mk), 256, 0, w.st>>>(w.s, w.s, a2, w.ds, mk);
      nfull += used_full ? 1 : 0;
      ++it;
      if (w.err != cudaSuccess) break;
    }
    if (result != NMF_OK || w.err != cudaSuccess) break;
    // predictor (affine-scaling) direction, mu = 0, Gauss-Newton Hessian
    if (w.direction(0.0, rho, 0) != 0) {
      result = NMF_ENUMERIC;
      break;
    }
    double a1 = 1.0;
    w.frac(w.x, w.dx, w.y, w.dy, 1.0, &a1);
    ipm_frac2<<<1, RT, 0, w.st>>>(w.r, w.dr, nk, w.s, w.ds, mk, 1.0, w.red);
    w.fetch(2);
    const double a2 = std::min(w.hred[0], w.hred[1]);
    ipm_mu_aff<<<1, RT, 0, w.st>>>(w.x, w.dx, w.r, w.dr, nk, w.y, w.dy, w.s, w.ds, mk, a1, a2, w.red);
    w.fetch(2);
    const double mu_aff = w.hred[0] / (double)(nk + mk), mu_cur = w.hred[1] / (double)(nk + mk);
    const double ratio = mu_aff / mu_cur;
    double sigma = ratio * ratio * ratio;
    if (!(sigma < 0.99)) sigma = 0.99;
    if (sigma < 0.0) sigma = 0.0;
    mu *= sigma;
    flag = sigma <= sigma_c;
  }
  if (w.err != cudaSuccess) return handle_fail(h, NMF_ECUDA, cudaGetErrorString(w.err));
  const double f = w.objective(w.x, w.y);
  if (stats) {
    stats[0] = E0;
    stats[1] = f;
    stats[2] = it;
    stats[3] = outer;
    stats[4] = mu;
    stats[5] = nfull;
    stats[6] = nfail;
  }
  // the stage-2 point becomes the handle's iterate (primed like nmf_set_factors)
  if (result == NMF_OK || result == NMF_ENOTCONV) {
    const nmf_status s2 = nmf_set_factors(h, w.x, w.y, 1);
    if (s2 != NMF_OK) return s2;
  }
  if (result == NMF_ENUMERIC) return handle_fail(h, NMF_ENUMERIC, "stage 2: a Cholesky factorisation failed");
  if (result == NMF_ENOTCONV) return handle_fail(h, NMF_ENOTCONV, "stage 2: Newton cap reached");
  return NMF_OK;
}

}  // extern "C"
