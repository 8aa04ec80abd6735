// fKK, fPEC and fSEC on the k basis vectors (Secs. 2.2-2.4), fp64, on the
// device.  Sizes are small (k <= 80 rows, |q| <= 2k rows, M <= 2048
// channels), so each step is a short kernel:
//   B = V^T / f;  H_B = H{B}                                   (fKK, Eq. fKK)
//   X = P_q;  Phi_ph = X H_B;  Phi_err = ALS baseline per row   (Eq. phi_err_USphi_b)
//   Phi_PEC^T = (X^T X + lambda_r I)^-1 X^T Phi_err            (Eq. PEC_Ridge)
//   H_Phi = H{Phi_PEC^T};  V_SEC^T = M{B + H_Phi}              (Eq. fSEC_VT)
//   C_amp = B + H_Phi - V_SEC^T;  C_ph = H_B - Phi_PEC^T       (Eq. fKKEC)
#include "common.cuh"
#include "df64.cuh"
#include "fft.cuh"
#include "fit.h"

namespace fkk {
namespace {

using dw::df;

// ------------------------------------------------------------------ q ---
__global__ void gather_q_kernel(const int64_t* __restrict__ qmax, const int64_t* __restrict__ qmin, int k,
                                int64_t n_rows, int64_t* __restrict__ q, int* __restrict__ nq, long long* status) {
  // the 2k extreme rows, sorted by rank (position = number of smaller values,
  // ties by index), then de-duplicated; one block
  __shared__ int64_t buf[160], srt[160];
  __shared__ int keep[160];
  const int n = 2 * k, t = threadIdx.x;
  if (t < n) {
    int64_t v = (t & 1) ? qmin[t >> 1] : qmax[t >> 1];
    // a column of P without a finite value has no extreme row: report it and
    // use row 0 rather than index past P
    if (v < 0 || v >= n_rows) {
      record_error(status, kErrNotConverged);
      v = 0;
    }
    buf[t] = v;
  }
  __syncthreads();
  if (t < n) {
    const int64_t v = buf[t];
    int rank = 0;
    for (int u = 0; u < n; ++u) rank += (buf[u] < v) || (buf[u] == v && u < t);
    srt[rank] = v;
  }
  __syncthreads();
  if (t < n) keep[t] = (t == 0 || srt[t] != srt[t - 1]);
  __syncthreads();
  if (t == 0) {
    int u = 0;
    for (int a = 0; a < n; ++a)
      if (keep[a]) q[u++] = srt[a];
    *nq = u;
  }
}

__global__ void gather_rows_kernel(const float* __restrict__ p, int k, const int64_t* __restrict__ q,
                                   const int* __restrict__ nq, double* __restrict__ x) {
  const int r = blockIdx.x;
  if (r >= *nq) return;
  for (int i = threadIdx.x; i < k; i += blockDim.x) x[(int64_t)r * k + i] = (double)p[q[r] * k + i];
}

// ------------------------------------------------------------- Hilbert ---
// One block per row: edge-replicated centred padding to L, FFT, -i sgn(m),
// inverse FFT, crop.  rows_dev (optional) bounds the live rows.
// e^{-2 pi i t / L} for t < L as double-word pairs (fp64 sincospi, split).
__global__ void twiddle_dz_kernel(dz* __restrict__ tw, int L) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L) return;
  double s, c;
  sincospi(-2.0 * (double)t / (double)L, &s, &c);
  const df cd = dw::from_double(c), sd = dw::from_double(s);
  tw[t] = {make_float2(cd.h, sd.h), make_float2(cd.l, sd.l)};
}

// H{x} of each row (the padded discrete Hilbert transform of Eq. KCARS) in
// double-word complex arithmetic: edge-replicated to L, forward FFT,
// multiplier -i sgn, inverse FFT, cropped and scaled by 1/L.
__global__ void hilbert_rows_kernel(const double* __restrict__ x, int m, int L, const dz* __restrict__ twg,
                                    double* __restrict__ h, const int* __restrict__ rows_dev) {
  extern __shared__ dz zsm[];
  const int row = blockIdx.x;
  if (rows_dev && row >= *rows_dev) return;
  dz* tw = zsm;
  dz* b0 = zsm + L;
  dz* b1 = b0 + L;
  const int left = (L - m) / 2;
  const double* xr = x + (int64_t)row * m;
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    tw[t] = twg[t];
    const int s = min(max(t - left, 0), m - 1);
    const df v = dw::from_double(xr[s]);
    b0[t] = {make_float2(v.h, 0.f), make_float2(v.l, 0.f)};
  }
  __syncthreads();
  int cur = fft_block_dz<-1>(b0, b1, L, tw, threadIdx.x, blockDim.x);
  dz* X = cur ? b1 : b0;
  dz* Y = cur ? b0 : b1;
  for (int t = threadIdx.x; t < L; t += blockDim.x) X[t] = hilbert_mult_dz(X[t], t, L);
  __syncthreads();
  int cur2 = fft_block_dz<+1>(X, Y, L, tw, threadIdx.x, blockDim.x);
  dz* H = cur2 ? Y : X;
  const double invL = 1.0 / (double)L;
  for (int j = threadIdx.x; j < m; j += blockDim.x)
    h[(int64_t)row * m + j] = dw::to_double(dw::make(H[left + j].h.x, H[left + j].l.x)) * invL;
}

// ---------------------------------------------------------- small ops ---
__global__ void b_from_v_kernel(const double* __restrict__ v, const double* __restrict__ f, int m, int k,
                                double* __restrict__ b) {
  const int i = blockIdx.x;
  for (int j = threadIdx.x; j < m; j += blockDim.x) b[(int64_t)i * m + j] = v[(int64_t)j * k + i] / (f ? f[j] : 1.0);
}

// out[r, j] = sum_i X[r, i] Y[i, j]   (X rows x k, Y k x m)
__global__ void small_gemm_kernel(const double* __restrict__ X, const double* __restrict__ Y, int k, int m,
                                  double* __restrict__ out, const int* __restrict__ rows_dev) {
  const int r = blockIdx.x;
  if (rows_dev && r >= *rows_dev) return;
  extern __shared__ double xs[];
  for (int i = threadIdx.x; i < k; i += blockDim.x) xs[i] = X[(int64_t)r * k + i];
  __syncthreads();
  for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < m; j += gridDim.y * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < k; ++i) acc = fma(xs[i], Y[(int64_t)i * m + j], acc);
    out[(int64_t)r * m + j] = acc;
  }
}

// ---------------------------------------------------------------- ALS ---
// Asymmetric least squares baseline of one row per block: repeat `iters`
// times: solve (W + lam D2^T D2) z = W y, then w_i = p if y_i > z_i else
// 1 - p (weights start at 1).  The pentadiagonal SPD system is solved as a
// block-tridiagonal system of 2 x 2 blocks (unknown pairs (z_2i, z_2i+1))
// by cyclic reduction: log2(P) levels of elimination and back-substitution
// with the block rows of each level in parallel.  P is the block count
// padded to a power of two with identity rows.  The arithmetic is
// double-word on the fp32 pipe (about 48 bits): the reduction's first
// levels are ~10^5 operations per row, which this part's fp64 rate (about
// 1.7 lane-operations per clock per SM) would make the bottleneck.

// Band entries of D2^T D2 (D2 = (M-2) x M second differences): diagonal at j
// and first off-diagonal (j, j+1); the second off-diagonal is 1 throughout.
__device__ __forceinline__ float band0(int j, int m) {
  float s = 0.f;
  if (j <= m - 3) s += 1.f;
  if (j >= 1 && j - 1 <= m - 3) s += 4.f;
  if (j >= 2 && j - 2 <= m - 3) s += 1.f;
  return s;
}
__device__ __forceinline__ float band1(int j, int m) {
  float s = 0.f;
  if (j >= 0 && j <= m - 3) s += -2.f;
  if (j >= 1 && j - 1 <= m - 3) s += -2.f;
  return s;
}

struct Blk {
  df a, b, c, d;  // [[a, b], [c, d]]
};
struct Vec2 {
  df x, y;
};
__device__ __forceinline__ df dot2(df p, df q, df r, df t) { return dw::add(dw::mul(p, q), dw::mul(r, t)); }
__device__ __forceinline__ Blk bmul(const Blk& x, const Blk& y) {
  return {dot2(x.a, y.a, x.b, y.c), dot2(x.a, y.b, x.b, y.d), dot2(x.c, y.a, x.d, y.c), dot2(x.c, y.b, x.d, y.d)};
}
__device__ __forceinline__ Blk badd(const Blk& x, const Blk& y) {
  return {dw::add(x.a, y.a), dw::add(x.b, y.b), dw::add(x.c, y.c), dw::add(x.d, y.d)};
}
__device__ __forceinline__ Blk bneg(const Blk& x) { return {dw::neg(x.a), dw::neg(x.b), dw::neg(x.c), dw::neg(x.d)}; }
__device__ __forceinline__ Blk binv(const Blk& x) {
  const df det = dw::sub(dw::mul(x.a, x.d), dw::mul(x.b, x.c));
  const df r = dw::rcp(det);
  return {dw::mul(x.d, r), dw::neg(dw::mul(x.b, r)), dw::neg(dw::mul(x.c, r)), dw::mul(x.a, r)};
}
__device__ __forceinline__ Vec2 bvec(const Blk& x, const Vec2& v) {
  return {dot2(x.a, v.x, x.b, v.y), dot2(x.c, v.x, x.d, v.y)};
}
__device__ __forceinline__ Vec2 vadd(const Vec2& u, const Vec2& v) { return {dw::add(u.x, v.x), dw::add(u.y, v.y)}; }
__device__ __forceinline__ Vec2 vsub(const Vec2& u, const Vec2& v) { return {dw::sub(u.x, v.x), dw::sub(u.y, v.y)}; }
// u > v for normalised double-words
__device__ __forceinline__ bool dgt(df u, df v) { return u.h > v.h || (u.h == v.h && u.l > v.l); }

__global__ void __launch_bounds__(256) als_kernel(const double* __restrict__ y_all, int m, int P, double lam_d,
                                                  double p_d, int iters, double* __restrict__ z_all,
                                                  const int* __restrict__ rows_dev) {
  extern __shared__ double als_sm[];
  const int row = blockIdx.x;
  if (rows_dev && row >= *rows_dev) return;
  Blk* A = reinterpret_cast<Blk*>(als_sm);
  Blk* B = A + P;
  Blk* C = B + P;
  Vec2* D = reinterpret_cast<Vec2*>(C + P);
  df* y = reinterpret_cast<df*>(D + P);
  df* w = y + 2 * P;
  df* z = w + 2 * P;
  const double* yr = y_all + (int64_t)row * m;
  const df lam = dw::from_double(lam_d);
  const df wp = dw::from_double(p_d), wq = dw::from_double(1.0 - p_d);
  const df one = dw::make(1.f), zero = dw::make(0.f);
  for (int j = threadIdx.x; j < 2 * P; j += blockDim.x) {
    y[j] = j < m ? dw::from_double(yr[j]) : zero;
    w[j] = one;
  }
  __syncthreads();
  // matrix entry a(j, l) for |j - l| <= 2 (identity outside the signal)
  auto ent = [&](int j, int l) -> df {
    if (j < 0 || l < 0 || j >= 2 * P || l >= 2 * P) return zero;
    if (j >= m || l >= m) return (j == l) ? one : zero;
    const int d = j - l;
    if (d == 0) return dw::add(w[j], dw::mul(lam, band0(j, m)));
    if (d == 1 || d == -1) return dw::mul(lam, band1(min(j, l), m));
    if (d == 2 || d == -2) return lam;
    return zero;
  };
  for (int it = 0; it < iters; ++it) {
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
      const int r0 = 2 * i, r1 = 2 * i + 1;
      B[i] = {ent(r0, r0), ent(r0, r1), ent(r1, r0), ent(r1, r1)};
      A[i] = {ent(r0, r0 - 2), ent(r0, r0 - 1), ent(r1, r0 - 2), ent(r1, r0 - 1)};
      C[i] = {ent(r0, r1 + 1), ent(r0, r1 + 2), ent(r1, r1 + 1), ent(r1, r1 + 2)};
      D[i] = {r0 < m ? dw::mul(w[r0], y[r0]) : zero, r1 < m ? dw::mul(w[r1], y[r1]) : zero};
    }
    __syncthreads();
    // forward reduction
    for (int s = 1; s < P; s *= 2) {
      for (int t = threadIdx.x; t < P / (2 * s); t += blockDim.x) {
        const int i = 2 * s * t + 2 * s - 1;
        const int im = i - s, ip = i + s;
        // alpha = -A_i B_im^-1, gamma = -C_i B_ip^-1
        const Blk alpha = bneg(bmul(A[i], binv(B[im])));
        Blk nb = badd(B[i], bmul(alpha, C[im]));
        Vec2 nd = vadd(D[i], bvec(alpha, D[im]));
        const Blk na = bmul(alpha, A[im]);
        Blk nc = {zero, zero, zero, zero};
        if (ip < P) {
          const Blk gamma = bneg(bmul(C[i], binv(B[ip])));
          nb = badd(nb, bmul(gamma, A[ip]));
          nd = vadd(nd, bvec(gamma, D[ip]));
          nc = bmul(gamma, C[ip]);
        }
        B[i] = nb;
        D[i] = nd;
        A[i] = na;
        C[i] = nc;
      }
      __syncthreads();
    }
    // back-substitution (solutions overwrite D)
    if (threadIdx.x == 0) D[P - 1] = bvec(binv(B[P - 1]), D[P - 1]);
    __syncthreads();
    for (int s = P / 2; s >= 1; s /= 2) {
      for (int t = threadIdx.x; t < P / (2 * s); t += blockDim.x) {
        const int i = 2 * s * t + s - 1;
        Vec2 rhs = D[i];
        if (i - s >= 0) rhs = vsub(rhs, bvec(A[i], D[i - s]));
        if (i + s < P) rhs = vsub(rhs, bvec(C[i], D[i + s]));
        D[i] = bvec(binv(B[i]), rhs);
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
      z[2 * i] = D[i].x;
      z[2 * i + 1] = D[i].y;
    }
    __syncthreads();
    // new weights; once they repeat, every further iteration reproduces the
    // same z, so the remaining iterations are skipped
    int changed = 0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const df nw = dgt(y[j], z[j]) ? wp : wq;
      changed |= (nw.h != w[j].h) || (nw.l != w[j].l);
      w[j] = nw;
    }
    if (!__syncthreads_or(changed)) break;
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x) z_all[(int64_t)row * m + j] = dw::to_double(z[j]);
}

// -------------------------------------------------------------- ridge ---
// Eq. PEC_Ridge as Phi_PEC^T = N Phi_err with N = (X^T X + lambda_r I)^-1 X^T
// (k x nq), lambda_r = rel * ||X||_F^2 / k.  ridge_n_kernel forms N in one
// block in double-word arithmetic (Cholesky with reciprocal pivots, then the
// two triangular solves on all nq right-hand sides at once); ridge_apply
// multiplies it out in fp64, one output per thread.
__global__ void ridge_n_kernel(const double* __restrict__ X, const int* __restrict__ nq_dev, int k, double rel,
                               double* __restrict__ n_out) {
  extern __shared__ dw::df rsm[];
  const int nq = *nq_dev;
  dw::df* C = rsm;            // [k][k], lower triangle used
  dw::df* B = C + k * k;      // [k][nq]: X^T, then the solution
  dw::df* rinv = B + k * nq;  // [k] reciprocal pivots
  __shared__ dw::df lam_s;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int x = tid; x < k * nq; x += nt) {
    const int i = x / nq, q = x % nq;
    B[x] = dw::from_double(X[(int64_t)q * k + i]);
  }
  __syncthreads();
  for (int x = tid; x < k * k; x += nt) {
    const int a = x / k, b = x % k;
    if (b > a) continue;
    dw::df acc = dw::make(0.f);
    for (int q = 0; q < nq; ++q) acc = dw::add(acc, dw::mul(B[a * nq + q], B[b * nq + q]));
    C[x] = acc;
  }
  __syncthreads();
  if (tid == 0) {
    dw::df tr = dw::make(0.f);
    for (int a = 0; a < k; ++a) tr = dw::add(tr, C[a * k + a]);
    lam_s = dw::mul(tr, dw::from_double(rel / k));
  }
  __syncthreads();
  for (int a = tid; a < k; a += nt) C[a * k + a] = dw::add(C[a * k + a], lam_s);
  __syncthreads();
  // Cholesky, lower, in place
  for (int c = 0; c < k; ++c) {
    if (tid == 0) {
      const dw::df d = dw::sqrt(C[c * k + c]);
      C[c * k + c] = d;
      rinv[c] = dw::rcp(d);
    }
    __syncthreads();
    for (int r = c + 1 + tid; r < k; r += nt) C[r * k + c] = dw::mul(C[r * k + c], rinv[c]);
    __syncthreads();
    const int w = k - c - 1;
    for (int x = tid; x < w * w; x += nt) {
      const int r = c + 1 + x / w, t = c + 1 + x % w;
      if (t <= r) C[r * k + t] = dw::sub(C[r * k + t], dw::mul(C[r * k + c], C[t * k + c]));
    }
    __syncthreads();
  }
  // L Y = X^T
  for (int i = 0; i < k; ++i) {
    for (int q = tid; q < nq; q += nt) B[i * nq + q] = dw::mul(B[i * nq + q], rinv[i]);
    __syncthreads();
    const int w = k - i - 1;
    for (int x = tid; x < w * nq; x += nt) {
      const int t = i + 1 + x / nq, q = x % nq;
      B[t * nq + q] = dw::sub(B[t * nq + q], dw::mul(C[t * k + i], B[i * nq + q]));
    }
    __syncthreads();
  }
  // L^T N = Y
  for (int i = k - 1; i >= 0; --i) {
    for (int q = tid; q < nq; q += nt) B[i * nq + q] = dw::mul(B[i * nq + q], rinv[i]);
    __syncthreads();
    for (int x = tid; x < i * nq; x += nt) {
      const int t = x / nq, q = x % nq;
      B[t * nq + q] = dw::sub(B[t * nq + q], dw::mul(C[i * k + t], B[i * nq + q]));
    }
    __syncthreads();
  }
  for (int x = tid; x < k * nq; x += nt) n_out[x] = dw::to_double(B[x]);
}

// Phi_PEC^T[i, j] = sum_q N[i, q] Phi_err[q, j].
__global__ void ridge_apply_kernel(const double* __restrict__ nmat, const double* __restrict__ perr,
                                   const int* __restrict__ nq_dev, int k, int m, double* __restrict__ out) {
  const int i = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int nq = *nq_dev;
  const double* nr = nmat + (int64_t)i * nq;
  double acc = 0.0;
  for (int q = 0; q < nq; ++q) acc = fma(nr[q], perr[(int64_t)q * m + j], acc);
  out[(int64_t)i * m + j] = acc;
}

// ---------------------------------------------------------------- SEC ---
// pinv of the window Vandermonde matrix V[t][p] = (t/h)^p, t = -h..h:
// pinv = (V^T V)^-1 V^T, (order+1) x window.  One block.
__global__ void sg_pinv_kernel(int window, int order, double* __restrict__ pinv) {
  __shared__ double A[8][16];
  __shared__ double part[8][8][32];
  const int h = window / 2;
  const int P = order + 1;
  // moments sum_t x^q, x = t/h, q = 0..2 order: per-warp partial sums
  double mom[15];
  for (int q = 0; q < 2 * P - 1; ++q) mom[q] = 0.0;
  for (int t = threadIdx.x; t < window; t += blockDim.x) {
    double x = (double)(t - h) / h, pw = 1.0;
    for (int q = 0; q < 2 * P - 1; ++q) {
      mom[q] += pw;
      pw *= x;
    }
  }
  for (int q = 0; q < 2 * P - 1; ++q) {
    double v = warp_sum(mom[q]);
    if ((threadIdx.x & 31) == 0) part[q / 8][q % 8][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double M_[15];
    for (int q = 0; q < 2 * P - 1; ++q) {
      double sum = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += part[q / 8][q % 8][w];
      M_[q] = sum;
    }
    for (int a = 0; a < P; ++a)
      for (int b = 0; b < P; ++b) {
        A[a][b] = M_[a + b];
        A[a][P + b] = (a == b) ? 1.0 : 0.0;
      }
    for (int c = 0; c < P; ++c) {  // Gauss-Jordan (SPD, no pivoting needed)
      double piv = A[c][c];
      for (int b = 0; b < 2 * P; ++b) A[c][b] /= piv;
      for (int a = 0; a < P; ++a)
        if (a != c) {
          double fct = A[a][c];
          for (int b = 0; b < 2 * P; ++b) A[a][b] -= fct * A[c][b];
        }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < window; t += blockDim.x) {
    double tt = (double)(t - h) / h;
    for (int a = 0; a < P; ++a) {
      double s = 0.0, pw = 1.0;
      for (int b = 0; b < P; ++b) {
        s += A[a][P + b] * pw;
        pw *= tt;
      }
      pinv[a * window + t] = s;
    }
  }
}

// Savitzky-Golay trendline of row r of x (k x m): interior points use the
// centre coefficients (row 0 of pinv).  grid = (k, chunks).
__global__ void sg_apply_kernel(const double* __restrict__ x, int m, int window, const double* __restrict__ pinv,
                                double* __restrict__ out) {
  const int r = blockIdx.x;
  const int h = window / 2;
  const double* xr = x + (int64_t)r * m;
  for (int j = h + blockIdx.y * blockDim.x + threadIdx.x; j < m - h; j += gridDim.y * blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < window; ++t) s = fma(pinv[t], xr[j - h + t], s);
    out[(int64_t)r * m + j] = s;
  }
}

// The h points at each edge of row r: the polynomial fitted to the first /
// last window (beta = pinv . window) evaluated there.  One block per row.
__global__ void sg_edges_kernel(const double* __restrict__ x, int m, int window, int order,
                                const double* __restrict__ pinv, double* __restrict__ out) {
  __shared__ double beta[2][8];
  __shared__ double red[8];
  const int r = blockIdx.x;
  const int h = window / 2;
  const double* xr = x + (int64_t)r * m;
  for (int side = 0; side < 2; ++side) {
    const double* seg = side ? xr + (m - window) : xr;
    for (int a = 0; a <= order; ++a) {
      double s = 0.0;
      for (int t = threadIdx.x; t < window; t += blockDim.x) s = fma(pinv[a * window + t], seg[t], s);
      s = warp_sum(s);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
      __syncthreads();
      if (threadIdx.x == 0) {
        double tsum = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tsum += red[q];
        beta[side][a] = tsum;
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < 2 * h; t += blockDim.x) {
    const int side = t >= h;
    const int j = side ? m - h + (t - h) : t;
    const double tt = side ? (double)(j - (m - 1 - h)) / h : (double)(j - h) / h;
    double s = 0.0, pw = 1.0;
    for (int a = 0; a <= order; ++a) {
      s += beta[side][a] * pw;
      pw *= tt;
    }
    out[(int64_t)r * m + j] = s;
  }
}

__global__ void mean_rows_kernel(const double* __restrict__ x, int m, double* __restrict__ out) {
  const int r = blockIdx.x;
  __shared__ double red[32];
  double s = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) s += x[(int64_t)r * m + j];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    red[0] = t / m;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) out[(int64_t)r * m + j] = red[0];
}

__global__ void axpy3_kernel(const double* __restrict__ a, const double* __restrict__ b, const double* __restrict__ c,
                             double sb, double sc, int64_t n, double* __restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  out[t] = a[t] + (b ? sb * b[t] : 0.0) + (c ? sc * c[t] : 0.0);
}

}  // namespace

fkk_status launch_gather_q(fkk_ctx* ctx, const int64_t* qmax, const int64_t* qmin, int k, const float* p,
                           int64_t n_rows, int64_t* q, int* nq_dev, double* x_rows, cudaStream_t st) {
  FKK_COUNT_LAUNCH(); gather_q_kernel<<<1, 160, 0, st>>>(qmax, qmin, k, n_rows, q, nq_dev, ctx->d_status);
  FKK_COUNT_LAUNCH(); gather_rows_kernel<<<2 * k, 32, 0, st>>>(p, k, q, nq_dev, x_rows);
  return cuda_check(ctx, cudaGetLastError(), "gather_q launch");
}

static fkk_status hilbert_rows(fkk_ctx* ctx, const double* x, int rows, int m, int L, double* h, const int* rows_dev,
                               cudaStream_t st) {
  fkk_status s;
  dz* tw = (dz*)workspace(ctx, "hilb_tw", (size_t)L * sizeof(dz), &s);
  if (!tw) return s;
  FKK_COUNT_LAUNCH(); twiddle_dz_kernel<<<(L + 255) / 256, 256, 0, st>>>(tw, L);
  size_t smem = (size_t)3 * L * sizeof(dz);
  FKK_CUDA(ctx, cudaFuncSetAttribute(hilbert_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  FKK_COUNT_LAUNCH(); hilbert_rows_kernel<<<rows, 256, smem, st>>>(x, m, L, tw, h, rows_dev);
  return cuda_check(ctx, cudaGetLastError(), "hilbert_rows launch");
}

fkk_status launch_basis_math(fkk_ctx* ctx, const BasisParams& bp, const double* v, const double* f,
                             const double* x_rows, int nq_max, BasisOut out, cudaStream_t st) {
  fkk_status s;
  const int m = bp.m, k = bp.k, L = bp.L;
  const size_t km = (size_t)k * m;
  double* b = out.b ? out.b : (double*)workspace(ctx, "bm_b", km * 8, &s);
  if (!b) return s;
  double* hb = out.h_b ? out.h_b : (double*)workspace(ctx, "bm_hb", km * 8, &s);
  if (!hb) return s;
  double* phit = out.phi_pec_t ? out.phi_pec_t : (double*)workspace(ctx, "bm_phit", km * 8, &s);
  if (!phit) return s;
  double* hphi = out.h_phi ? out.h_phi : (double*)workspace(ctx, "bm_hphi", km * 8, &s);
  if (!hphi) return s;
  double* vsec = out.v_sec_t ? out.v_sec_t : (double*)workspace(ctx, "bm_vsec", km * 8, &s);
  if (!vsec) return s;
  double* corr = (double*)workspace(ctx, "bm_corr", km * 8, &s);
  if (!corr) return s;

  // The ridge operator N = (X^T X + lambda I)^-1 X^T needs only the
  // sub-sampled rows X, and the Savitzky-Golay pseudo-inverse only the window:
  // both run on the context's side stream beside the Hilbert transform of B
  // and the ALS detrend, and the main stream waits before their first use.
  const bool sg = bp.sec && bp.sec_mode != 1;
  const int* nq_dev = nullptr;
  double* lc = nullptr;
  double* pinv = nullptr;
  if (bp.pec) {
    nq_dev = (const int*)workspace(ctx, "fit_nq", 64, &s);  // written by launch_gather_q
    if (!nq_dev) return s;
    lc = (double*)workspace(ctx, "bm_ridge_n", (size_t)k * nq_max * 8, &s);
    if (!lc) return s;
  }
  if (sg) {
    pinv = (double*)workspace(ctx, "bm_sgpinv", (size_t)(bp.sg_order + 1) * bp.sg_window * 8, &s);
    if (!pinv) return s;
  }
  cudaStream_t aux = nullptr;
  const bool side = bp.pec || sg;
  if (side) {
    FKK_TRY(side_stream(ctx, &aux));
    FKK_CUDA(ctx, cudaEventRecord(ctx->ev_fork, st));
    FKK_CUDA(ctx, cudaStreamWaitEvent(aux, ctx->ev_fork, 0));
    if (bp.pec) {
      const size_t rsm = (size_t)(k * k + k * nq_max + k) * sizeof(dw::df);
      FKK_CUDA(ctx, cudaFuncSetAttribute(ridge_n_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
      FKK_COUNT_LAUNCH(); ridge_n_kernel<<<1, 256, rsm, aux>>>(x_rows, nq_dev, k, bp.ridge_rel, lc);
    }
    if (sg) {
      FKK_COUNT_LAUNCH(); sg_pinv_kernel<<<1, 256, 0, aux>>>(bp.sg_window, bp.sg_order, pinv);
    }
    FKK_CUDA(ctx, cudaEventRecord(ctx->ev_join, aux));
  }
  bool joined = !side;
  auto join = [&]() -> fkk_status {
    if (!joined) {
      joined = true;
      return cuda_check(ctx, cudaStreamWaitEvent(st, ctx->ev_join, 0), "basis math join");
    }
    return FKK_OK;
  };

  FKK_COUNT_LAUNCH(); b_from_v_kernel<<<k, 256, 0, st>>>(v, f, m, k, b);
  FKK_TRY(hilbert_rows(ctx, b, k, m, L, hb, nullptr, st));
  const unsigned ek = (unsigned)((km + 255) / 256);
  if (bp.pec) {
    double* phph = (double*)workspace(ctx, "bm_phph", (size_t)nq_max * m * 8, &s);
    if (!phph) return s;
    double* perr = (double*)workspace(ctx, "bm_perr", (size_t)nq_max * m * 8, &s);
    if (!perr) return s;
    FKK_COUNT_LAUNCH(); small_gemm_kernel<<<dim3(nq_max, 4), 256, k * sizeof(double), st>>>(x_rows, hb, k, m, phph, nq_dev);
    int P = 1;
    while (P < (m + 1) / 2) P *= 2;
    size_t als_smem = (size_t)P * (3 * sizeof(Blk) + sizeof(Vec2)) + (size_t)6 * P * sizeof(df);
    FKK_CUDA(ctx, cudaFuncSetAttribute(als_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)als_smem));
    FKK_COUNT_LAUNCH(); als_kernel<<<nq_max, 256, als_smem, st>>>(phph, m, P, bp.als_lambda, bp.als_p, bp.als_iters, perr, nq_dev);
    FKK_TRY(join());
    FKK_COUNT_LAUNCH(); ridge_apply_kernel<<<dim3((m + 127) / 128, k), 128, 0, st>>>(lc, perr, nq_dev, k, m, phit);
    FKK_CUDA(ctx, cudaGetLastError());
    FKK_TRY(hilbert_rows(ctx, phit, k, m, L, hphi, nullptr, st));
  } else {
    FKK_CUDA(ctx, cudaMemsetAsync(phit, 0, km * 8, st));
    FKK_CUDA(ctx, cudaMemsetAsync(hphi, 0, km * 8, st));
  }
  FKK_COUNT_LAUNCH(); axpy3_kernel<<<ek, 256, 0, st>>>(b, hphi, nullptr, 1.0, 0.0, (int64_t)km, corr);  // B + H_Phi
  if (bp.sec) {
    if (bp.sec_mode == 1) {
      FKK_COUNT_LAUNCH(); mean_rows_kernel<<<k, 256, 0, st>>>(corr, m, vsec);
    } else {
      FKK_TRY(join());
      FKK_COUNT_LAUNCH(); sg_apply_kernel<<<dim3(k, (m + 255) / 256), 256, 0, st>>>(corr, m, bp.sg_window, pinv, vsec);
      FKK_COUNT_LAUNCH(); sg_edges_kernel<<<k, 256, 0, st>>>(corr, m, bp.sg_window, bp.sg_order, pinv, vsec);
    }
  } else {
    FKK_CUDA(ctx, cudaMemsetAsync(vsec, 0, km * 8, st));
  }
  FKK_TRY(join());
  FKK_COUNT_LAUNCH(); axpy3_kernel<<<ek, 256, 0, st>>>(corr, vsec, nullptr, -1.0, 0.0, (int64_t)km, out.c_amp);
  FKK_COUNT_LAUNCH(); axpy3_kernel<<<ek, 256, 0, st>>>(hb, phit, nullptr, -1.0, 0.0, (int64_t)km, out.c_ph);
  return cuda_check(ctx, cudaGetLastError(), "basis math launch");
}

}  // namespace fkk
