// Symmetric eigensolve of the Gram matrix (Sec. 2.2: the SVD of A through
// A^T A): a two-sided block Jacobi method in fp32 over the whole matrix,
// then a Rayleigh-Ritz refinement of the leading K' = k + 32 vectors in fp64
// whose small projected eigenproblem is solved by the same block Jacobi
// method in fp64.
//
// Block Jacobi: the working matrix Gw (mp x mp, zero-padded) is split into
// blocks of 8 indices.  A sweep visits every pair of blocks once in a
// round-robin (circle) schedule; in each round the mp/16 disjoint block
// pairs are processed in parallel, one CTA per pair:
//   phase 1  one cyclic scalar Jacobi sweep over the 16 x 16 principal
//            submatrix S of the pair (one warp) gives the rotation E; in fp32
//            E is re-orthonormalised by a Newton-Schulz step so that
//            accumulated rounding does not drift the basis;
//   phase 2a rows J of Gw and of V^T are multiplied by E^T;
//   phase 2b (after a grid barrier) columns J of Gw are multiplied by E.
// A rotation is applied when |S_pq| > tol sqrt(|S_pp S_qq|) (relative
// criterion); the sweep loop ends after a sweep in which no pair exceeded it.
// Grid barriers spin a bounded number of times and report FKK_ERR_TIMEOUT.
//
// Refinement: Q = orth(V_K') by Cholesky-QR in fp64, H = Q^T G Q, H = W
// diag(theta) W^T by fp64 block Jacobi, V_k = Q W[:, top k], lambda = theta.
#include <algorithm>

#include "common.cuh"
#include "fit.h"

namespace fkk {
namespace {

constexpr int kB = 8;        // block width
constexpr int kJ = 2 * kB;   // indices per block pair
constexpr int kThreads = 256;
constexpr int kExtra = 32;   // refinement subspace beyond k

// 16-byte vector type of T (float4 / double2)
template <typename T>
struct V4;
template <>
struct V4<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct V4<double> {
  using type = double2;
  static constexpr int n = 2;
};

template <typename T>
struct JacobiArgs {
  T* gw;
  T* vt;
  int mp;
  int nblk;
  T tol;
  int max_sweeps;
  unsigned* bar;
  int* abort_flag;
  int* sweep_rot;
  int* sweeps_done;
  long long* status;
};

// circle schedule of the 16 indices of a block pair: kPair16[r][i] = (p, q)
__constant__ unsigned char kPair16[kJ - 1][kJ / 2][2];

__device__ __forceinline__ void circle_pair(int i, int r, int n, int& P, int& Q) {
  const int n1 = n - 1;
  if (i == 0) {
    P = 0;
    Q = 1 + (r % n1);
  } else {
    P = 1 + ((i + r) % n1);
    Q = 1 + ((n1 - i + r) % n1);
  }
}

// Rotation (c, s), J = [[c, s], [-s, c]], with J^T [[app, apq], [apq, aqq]] J
// diagonal (symmetric 2 x 2 Schur decomposition).
template <typename T>
__device__ __forceinline__ void sym_schur2(T app, T aqq, T apq, T& c, T& s) {
  T tau = (aqq - app) / (T(2) * apq);
  T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
  c = T(1) / sqrt(T(1) + t * t);
  s = t * c;
}

template <typename T>
__device__ __forceinline__ bool significant(T app, T aqq, T apq, T tol) {
  return fabs(apq) > tol * sqrt(fabs(app) * fabs(aqq)) && fabs(apq) > T(1e-30);
}

// One cyclic Jacobi sweep on the 16x16 S (shared), accumulating E; all
// threads of the block take part (2 barriers per inner round).  Returns
// whether any pair was significant at the start (block-uniform).
template <typename T>
__device__ __forceinline__ bool inner_sweep(T (*S)[kJ + 1], T (*E)[kJ + 1], T* cs_c, T* cs_s, int* flag, T tol,
                                            int tid) {
  if (tid == 0) *flag = 0;
  {
    const int a = tid / kJ, b = tid % kJ;
    E[a][b] = (a == b) ? T(1) : T(0);
  }
  __syncthreads();
  {
    const int a = tid / kJ, b = tid % kJ;
    if (a < b && significant(S[a][a], S[b][b], S[a][b], tol)) *flag = 1;
  }
  __syncthreads();
  if (!*flag) return false;
  for (int r = 0; r < kJ - 1; ++r) {
    if (tid < kJ / 2) {
      const int p = kPair16[r][tid][0], q = kPair16[r][tid][1];
      T apq = S[p][q];
      T c = T(1), s = T(0);
      if (significant(S[p][p], S[q][q], apq, tol)) sym_schur2(S[p][p], S[q][q], apq, c, s);
      cs_c[tid] = c;
      cs_s[tid] = s;
    }
    __syncthreads();
    if (tid < (kJ / 2) * (kJ / 2)) {
      // S <- J^T S J on the 8 x 8 grid of 2 x 2 blocks
      const int a = tid / (kJ / 2), b = tid % (kJ / 2);
      const int pa = kPair16[r][a][0], qa = kPair16[r][a][1];
      const int pb = kPair16[r][b][0], qb = kPair16[r][b][1];
      T ca = cs_c[a], sa = cs_s[a], cb = cs_c[b], sb = cs_s[b];
      T b00 = S[pa][pb], b01 = S[pa][qb], b10 = S[qa][pb], b11 = S[qa][qb];
      T x00 = ca * b00 - sa * b10, x01 = ca * b01 - sa * b11;
      T x10 = sa * b00 + ca * b10, x11 = sa * b01 + ca * b11;
      S[pa][pb] = x00 * cb - x01 * sb;
      S[pa][qb] = x00 * sb + x01 * cb;
      S[qa][pb] = x10 * cb - x11 * sb;
      S[qa][qb] = x10 * sb + x11 * cb;
    } else if (tid < (kJ / 2) * (kJ / 2) + kJ * (kJ / 2)) {
      // E <- E J
      const int it = tid - (kJ / 2) * (kJ / 2);
      const int row = it / (kJ / 2), a = it % (kJ / 2);
      const int pa = kPair16[r][a][0], qa = kPair16[r][a][1];
      T c = cs_c[a], s = cs_s[a];
      T ep = E[row][pa], eq = E[row][qa];
      E[row][pa] = c * ep - s * eq;
      E[row][qa] = s * ep + c * eq;
    }
    __syncthreads();
  }
  return true;
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) block_jacobi_kernel(JacobiArgs<T> p) {
  __shared__ T S[kJ][kJ + 1];
  __shared__ T E[kJ][kJ + 1];
  __shared__ T F[kJ][kJ + 1];
  __shared__ T cs_c[kJ / 2], cs_s[kJ / 2];
  __shared__ int J[kJ];
  __shared__ int rot_s;
  extern __shared__ __align__(16) unsigned char stage_raw[];
  T* stage = reinterpret_cast<T*>(stage_raw);  // kJ x mp staging (rows or columns)
  const int tid = threadIdx.x;
  const int mp = p.mp;
  int sweep = 0;
  bool ok = true;
  for (; sweep < p.max_sweeps && ok; ++sweep) {
    for (int r = 0; r < p.nblk - 1 && ok; ++r) {
      int P, Q;
      circle_pair(blockIdx.x, r, p.nblk, P, Q);
      if (tid < kJ) J[tid] = (tid < kB) ? P * kB + tid : Q * kB + (tid - kB);
      __syncthreads();
      {
        int a = tid / kJ, b = tid % kJ;  // 256 threads = 16 x 16
        T x = p.gw[(int64_t)J[a] * mp + J[b]];
        T y = p.gw[(int64_t)J[b] * mp + J[a]];
        S[a][b] = T(0.5) * (x + y);
      }
      __syncthreads();
      const bool rot = inner_sweep<T>(S, E, cs_c, cs_s, &rot_s, p.tol, tid);
      if (rot && tid == 0) atomicAdd(&p.sweep_rot[sweep], 1);
      if (!rot) {
        // nothing significant in this pair (E = I): keep the barrier count
        ok = grid_sync(p.bar, gridDim.x, p.abort_flag, p.status);
        if (ok) ok = grid_sync(p.bar, gridDim.x, p.abort_flag, p.status);
        continue;
      }
      if (sizeof(T) == 4) {
        // Newton-Schulz: E <- E (3 I - E^T E) / 2
        const int a = tid / kJ, b = tid % kJ;
        T f = T(0);
#pragma unroll
        for (int q = 0; q < kJ; ++q) f += E[q][a] * E[q][b];
        F[a][b] = f;
        __syncthreads();
        T e = T(0);
#pragma unroll
        for (int q = 0; q < kJ; ++q) e += E[a][q] * ((q == b ? T(3) : T(0)) - F[q][b]);
        __syncthreads();
        E[a][b] = T(0.5) * e;
        __syncthreads();
      }
      // phase 2a: rows J of Gw and V^T <- E^T rows, staged through shared
      // memory (all loads in flight, then the 16x16 transform per column)
      for (int mat = 0; mat < 2; ++mat) {
        T* base = mat ? p.vt : p.gw;
        const int nv = mp / V4<T>::n;  // vectors per row
        for (int t = tid; t < kJ * nv; t += kThreads) {
          const int a = t / nv, cv = t % nv;
          reinterpret_cast<typename V4<T>::type*>(stage + a * mp)[cv] =
              reinterpret_cast<const typename V4<T>::type*>(base + (int64_t)J[a] * mp)[cv];
        }
        __syncthreads();
        for (int c = tid; c < mp; c += kThreads) {
          T g[kJ];
#pragma unroll
          for (int a = 0; a < kJ; ++a) g[a] = stage[a * mp + c];
#pragma unroll
          for (int b = 0; b < kJ; ++b) {
            T sg = T(0);
#pragma unroll
            for (int a = 0; a < kJ; ++a) sg = fma(E[a][b], g[a], sg);
            stage[b * mp + c] = sg;
          }
        }
        __syncthreads();
        for (int t = tid; t < kJ * nv; t += kThreads) {
          const int a = t / nv, cv = t % nv;
          reinterpret_cast<typename V4<T>::type*>(base + (int64_t)J[a] * mp)[cv] =
              reinterpret_cast<const typename V4<T>::type*>(stage + a * mp)[cv];
        }
        __syncthreads();
      }
      ok = grid_sync(p.bar, gridDim.x, p.abort_flag, p.status);
      if (!ok) break;
      // phase 2b: columns J of Gw <- columns E (two 8-wide segments per row)
      {
        constexpr int vpb = kB / V4<T>::n;  // vectors per 8-wide segment
        for (int t = tid; t < mp * 2 * vpb; t += kThreads) {
          const int rr = t / (2 * vpb), q = t % (2 * vpb);
          const int seg = q / vpb, v = q % vpb;
          const int col0 = (seg ? J[kB] : J[0]) + v * V4<T>::n;
          reinterpret_cast<typename V4<T>::type*>(stage + rr * kJ + seg * kB)[v] =
              *reinterpret_cast<const typename V4<T>::type*>(p.gw + (int64_t)rr * mp + col0);
        }
        __syncthreads();
        for (int rr = tid; rr < mp; rr += kThreads) {
          T h[kJ];
#pragma unroll
          for (int a = 0; a < kJ; ++a) h[a] = stage[rr * kJ + a];
#pragma unroll
          for (int b = 0; b < kJ; ++b) {
            T sg = T(0);
#pragma unroll
            for (int a = 0; a < kJ; ++a) sg = fma(h[a], E[a][b], sg);
            stage[rr * kJ + b] = sg;
          }
        }
        __syncthreads();
        for (int t = tid; t < mp * 2 * vpb; t += kThreads) {
          const int rr = t / (2 * vpb), q = t % (2 * vpb);
          const int seg = q / vpb, v = q % vpb;
          const int col0 = (seg ? J[kB] : J[0]) + v * V4<T>::n;
          *reinterpret_cast<typename V4<T>::type*>(p.gw + (int64_t)rr * mp + col0) =
              reinterpret_cast<const typename V4<T>::type*>(stage + rr * kJ + seg * kB)[v];
        }
      }
      ok = grid_sync(p.bar, gridDim.x, p.abort_flag, p.status);
    }
    if (!ok) break;
    if (*(volatile int*)&p.sweep_rot[sweep] == 0) {
      ++sweep;
      break;
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    *p.sweeps_done = sweep;
    if (ok && sweep >= p.max_sweeps && p.sweep_rot[p.max_sweeps - 1] != 0) record_error(p.status, kErrNotConverged);
  }
}

// Gw (mp x mp, zero padded) from G (fp64, m x m, leading dimension ldg); V^T = I.
template <typename T>
__global__ void jacobi_init_kernel(const double* __restrict__ g, int m, int ldg, int mp, T* __restrict__ gw,
                                   T* __restrict__ vt) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (c >= mp) return;
  double x = (r < m && c < m) ? g[(int64_t)r * ldg + c] : 0.0;
  gw[(int64_t)r * mp + c] = (T)x;
  vt[(int64_t)r * mp + c] = (r == c) ? T(1) : T(0);
}

// order[rank] = i for the `want` largest diagonal entries of Gw (ties to the lower index)
template <typename T>
__global__ void rank_kernel(const T* __restrict__ gw, int m, int mp, int* __restrict__ order, int want) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  T di = gw[(int64_t)i * mp + i];
  int rank = 0;
  for (int j = 0; j < m; ++j) {
    T dj = gw[(int64_t)j * mp + j];
    rank += (dj > di) || (dj == di && j < i);
  }
  if (rank < want) order[rank] = i;
}

// X[j, c] = (double) V^T[order[c], j]: m x kk, row-major
template <typename T>
__global__ void gather_vecs_kernel(const T* __restrict__ vt, int m, int mp, const int* __restrict__ order, int kk,
                                   double* __restrict__ x) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (j < m) x[(int64_t)j * kk + c] = (double)vt[(int64_t)order[c] * mp + j];
}

// Small fp64 GEMM, 16 x 16 output tiles: C[M x N] = op(A) op(B), op = transpose if flagged.
__global__ void gemm64_kernel(const double* __restrict__ A, int lda, int ta, const double* __restrict__ B, int ldb,
                              int tb, double* __restrict__ Cm, int ldc, int M, int N, int K) {
  __shared__ double As[16][17], Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    int ka = k0 + tx, kb = k0 + ty;
    int ar = blockIdx.y * 16 + ty;
    As[ty][tx] = (ar < M && ka < K) ? (ta ? A[(int64_t)ka * lda + ar] : A[(int64_t)ar * lda + ka]) : 0.0;
    int bc = blockIdx.x * 16 + tx;
    Bs[ty][tx] = (bc < N && kb < K) ? (tb ? B[(int64_t)bc * ldb + kb] : B[(int64_t)kb * ldb + bc]) : 0.0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) acc = fma(As[ty][q], Bs[q][tx], acc);
    __syncthreads();
  }
  if (row < M && col < N) Cm[(int64_t)row * ldc + col] = acc;
}

// Cyclic Jacobi on a small symmetric fp64 matrix H (n x n, n even, n <= 112)
// held in shared memory by one block, accumulating W (columns =
// eigenvectors).  Pairs whose |h_pq| <= tol sqrt(|h_pp h_qq|) are skipped,
// and so are the updates of blocks both of whose rotations are skipped.
// Ends after a sweep with no significant pair or 30 sweeps.
__global__ void __launch_bounds__(512) small_jacobi64_kernel(const double* __restrict__ h_in, int n_real, int n,
                                                             double tol, double* __restrict__ h_out,
                                                             double* __restrict__ w_out, long long* status) {
  extern __shared__ double sm[];
  double* H = sm;              // n x n
  double* W = H + n * n;       // n x n
  double* cs = W + n * n;      // n/2 pairs: c, s
  __shared__ int any;
  __shared__ int sig[64];
  const int tid = threadIdx.x;
  for (int t = tid; t < n * n; t += blockDim.x) {
    int r = t / n, c = t % n;
    H[t] = (r < n_real && c < n_real) ? h_in[r * n_real + c] : (r == c ? -1e300 : 0.0);
    W[t] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int np = n / 2;
  int sweep = 0;
  for (; sweep < 30; ++sweep) {
    if (tid == 0) any = 0;
    __syncthreads();
    for (int r = 0; r < n - 1; ++r) {
      if (tid < np) {
        int p, q;
        circle_pair(tid, r, n, p, q);
        double hp = H[p * n + p], hq = H[q * n + q], hpq = H[p * n + q];
        double c = 1.0, s = 0.0;
        int g = 0;
        if (significant(hp, hq, hpq, tol)) {
          sym_schur2(hp, hq, hpq, c, s);
          g = 1;
          any = 1;
        }
        cs[2 * tid] = c;
        cs[2 * tid + 1] = s;
        sig[tid] = g;
      }
      __syncthreads();
      for (int bi = tid; bi < np * np; bi += blockDim.x) {
        const int a = bi / np, b = bi % np;
        if (!sig[a] && !sig[b]) continue;
        int pa, qa, pb, qb;
        circle_pair(a, r, n, pa, qa);
        circle_pair(b, r, n, pb, qb);
        const double ca = cs[2 * a], sa = cs[2 * a + 1], cb = cs[2 * b], sb = cs[2 * b + 1];
        double b00 = H[pa * n + pb], b01 = H[pa * n + qb], b10 = H[qa * n + pb], b11 = H[qa * n + qb];
        double x00 = ca * b00 - sa * b10, x01 = ca * b01 - sa * b11;
        double x10 = sa * b00 + ca * b10, x11 = sa * b01 + ca * b11;
        H[pa * n + pb] = x00 * cb - x01 * sb;
        H[pa * n + qb] = x00 * sb + x01 * cb;
        H[qa * n + pb] = x10 * cb - x11 * sb;
        H[qa * n + qb] = x10 * sb + x11 * cb;
      }
      for (int it = tid; it < n * np; it += blockDim.x) {
        const int row = it / np, a = it % np;
        if (!sig[a]) continue;
        int pa, qa;
        circle_pair(a, r, n, pa, qa);
        const double c = cs[2 * a], s = cs[2 * a + 1];
        double ep = W[row * n + pa], eq = W[row * n + qa];
        W[row * n + pa] = c * ep - s * eq;
        W[row * n + qa] = s * ep + c * eq;
      }
      __syncthreads();
    }
    if (!any) {
      ++sweep;
      break;
    }
  }
  if (tid == 0) {
    status[3] = sweep;
    if (sweep >= 30 && any) record_error(status, kErrNotConverged);
  }
  for (int t = tid; t < n * n; t += blockDim.x) {
    h_out[t] = H[t];
    w_out[t] = W[t];
  }
}

// X <- X (3 I - C) / 2 with C = X^T X (kk x kk): one Newton-Schulz step
// toward the orthonormal polar factor.  One block per row of X.
__global__ void ns_apply_kernel(double* __restrict__ X, int m, int kk, const double* __restrict__ Cm) {
  extern __shared__ double xr[];
  const int j = blockIdx.x;
  for (int t = threadIdx.x; t < kk; t += blockDim.x) xr[t] = X[(int64_t)j * kk + t];
  __syncthreads();
  for (int c = threadIdx.x; c < kk; c += blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < kk; ++t) s = fma(xr[t], (t == c ? 3.0 : 0.0) - Cm[t * kk + c], s);
    X[(int64_t)j * kk + c] = 0.5 * s;
  }
}

// lam[c] = H[o,o], V[:, c] = sum_t Q[:, t] W[t, o] (o = order[c]), sign-fixed
// so the largest-magnitude component is positive.  One block per column.
__global__ void finish_kernel(const double* __restrict__ q, int m, int kk, const double* __restrict__ hw,
                              const double* __restrict__ wt, int mph, const int* __restrict__ order, int k,
                              double* __restrict__ lam, double* __restrict__ v) {
  __shared__ double best_v[32];
  __shared__ int best_i[32];
  const int c = blockIdx.x;
  const int o = order[c];
  double bv = -1.0;
  int bi = 0x7fffffff;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < kk; ++t) s = fma(q[(int64_t)j * kk + t], wt[(int64_t)t * mph + o], s);
    v[(int64_t)j * k + c] = s;
    double a = fabs(s);
    if (a > bv || (a == bv && j < bi)) { bv = a; bi = j; }
  }
  for (int off = 16; off > 0; off >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, bv, off);
    int oi = __shfl_xor_sync(0xffffffffu, bi, off);
    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
  }
  if ((threadIdx.x & 31) == 0) { best_v[threadIdx.x >> 5] = bv; best_i[threadIdx.x >> 5] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (best_v[w] > best_v[0] || (best_v[w] == best_v[0] && best_i[w] < best_i[0])) {
        best_v[0] = best_v[w];
        best_i[0] = best_i[w];
      }
    lam[c] = hw[(int64_t)o * mph + o];
  }
  __syncthreads();
  const double sgn = v[(int64_t)best_i[0] * k + c] < 0.0 ? -1.0 : 1.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) v[(int64_t)j * k + c] *= sgn;
}

template <typename T>
fkk_status run_block_jacobi(fkk_ctx* ctx, const char* tag, const double* g, int m, int ldg, T tol, int max_sweeps,
                            T** gw_out, T** vt_out, int* mp_out, int diag_word, cudaStream_t st) {
  fkk_status s;
  const int mp = ((m + kJ - 1) / kJ) * kJ;
  const int nblk = mp / kB;
  const int npairs = nblk / 2;
  char name[64];
  snprintf(name, sizeof name, "%s_gw", tag);
  T* gw = (T*)workspace(ctx, name, (size_t)mp * mp * sizeof(T), &s);
  if (!gw) return s;
  snprintf(name, sizeof name, "%s_vt", tag);
  T* vt = (T*)workspace(ctx, name, (size_t)mp * mp * sizeof(T), &s);
  if (!vt) return s;
  snprintf(name, sizeof name, "%s_scr", tag);
  uint8_t* scr = (uint8_t*)workspace(ctx, name, 64 + 4 * max_sweeps, &s);
  if (!scr) return s;
  unsigned* bar = (unsigned*)(scr + 16);
  int* abort_flag = (int*)(scr + 24);
  int* sweeps_done = (int*)(scr + 28);
  int* sweep_rot = (int*)(scr + 64);
  FKK_CUDA(ctx, cudaMemsetAsync(scr, 0, 64 + 4 * max_sweeps, st));
  FKK_COUNT_LAUNCH(); jacobi_init_kernel<T><<<dim3((mp + 255) / 256, mp), 256, 0, st>>>(g, m, ldg, mp, gw, vt);
  FKK_CUDA(ctx, cudaGetLastError());
  const size_t stage_bytes = (size_t)kJ * mp * sizeof(T);
  FKK_CUDA(ctx, cudaFuncSetAttribute(block_jacobi_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_bytes));
  int per_sm = 0;
  FKK_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, block_jacobi_kernel<T>, kThreads, stage_bytes));
  if ((int64_t)per_sm * ctx->sm_count < npairs)
    return fail(ctx, FKK_ERR_INVALID_ARG, "eigensolve: %d block pairs exceed co-resident capacity", npairs);
  JacobiArgs<T> a{gw, vt, mp, nblk, tol, max_sweeps, bar, abort_flag, sweep_rot, sweeps_done, ctx->d_status};
  void* args[] = {&a};
  FKK_COUNT_LAUNCH();
  FKK_CUDA(ctx, cudaLaunchCooperativeKernel((void*)block_jacobi_kernel<T>, dim3(npairs), dim3(kThreads), args,
                                            stage_bytes, st));
  // sweep count of this solve -> status word diag_word (diagnostic)
  FKK_CUDA(ctx, cudaMemcpyAsync(ctx->d_status + diag_word, sweeps_done, sizeof(int), cudaMemcpyDeviceToDevice, st));
  *gw_out = gw;
  *vt_out = vt;
  *mp_out = mp;
  return FKK_OK;
}

void gemm64(const double* A, int lda, int ta, const double* B, int ldb, int tb, double* C, int ldc, int M, int N,
            int K, cudaStream_t st) {
  dim3 grid((N + 15) / 16, (M + 15) / 16);
  FKK_COUNT_LAUNCH(); gemm64_kernel<<<grid, 256, 0, st>>>(A, lda, ta, B, ldb, tb, C, ldc, M, N, K);
}

}  // namespace

fkk_status launch_eig_topk(fkk_ctx* ctx, const double* g, int m, int k, double* lam, double* v, cudaStream_t st,
                           int* sweeps_out, double tol32, int max_sweeps32) {
  fkk_status s;
  static bool tables = false;
  if (!tables) {
    unsigned char t[kJ - 1][kJ / 2][2];
    for (int r = 0; r < kJ - 1; ++r)
      for (int i = 0; i < kJ / 2; ++i) {
        const int n1 = kJ - 1;
        int P = (i == 0) ? 0 : 1 + ((i + r) % n1);
        int Q = (i == 0) ? 1 + (r % n1) : 1 + ((n1 - i + r) % n1);
        t[r][i][0] = (unsigned char)P;
        t[r][i][1] = (unsigned char)Q;
      }
    FKK_CUDA(ctx, cudaMemcpyToSymbol(kPair16, t, sizeof t));
    tables = true;
  }
  // 1. fp32 block Jacobi over the whole matrix
  float* gw;
  float* vt;
  int mp;
  FKK_TRY(run_block_jacobi<float>(ctx, "eig32", g, m, m, (float)(tol32 > 0 ? tol32 : 1e-6),
                                          max_sweeps32 > 0 ? max_sweeps32 : 40, &gw, &vt, &mp, 2, st));
  if (sweeps_out) FKK_CUDA(ctx, cudaMemcpyAsync(sweeps_out, ctx->d_status + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
  // 2. leading K' vectors, orthonormalised in fp64 (two Newton-Schulz steps)
  const int kk = std::min(m, k + kExtra);
  const int nsm = kk + (kk % 2);  // even size for the small Jacobi
  int* order = (int*)workspace(ctx, "eig_order", (size_t)m * 4, &s);
  if (!order) return s;
  double* q = (double*)workspace(ctx, "eig_q", (size_t)m * kk * 8, &s);
  if (!q) return s;
  double* y = (double*)workspace(ctx, "eig_y", (size_t)m * kk * 8, &s);
  if (!y) return s;
  double* h = (double*)workspace(ctx, "eig_h", (size_t)kk * kk * 8, &s);
  if (!h) return s;
  double* hw = (double*)workspace(ctx, "eig_hw", (size_t)nsm * nsm * 8, &s);
  if (!hw) return s;
  double* ww = (double*)workspace(ctx, "eig_ww", (size_t)nsm * nsm * 8, &s);
  if (!ww) return s;
  FKK_COUNT_LAUNCH(); rank_kernel<float><<<(m + 127) / 128, 128, 0, st>>>(gw, m, mp, order, kk);
  FKK_COUNT_LAUNCH(); gather_vecs_kernel<float><<<dim3((m + 127) / 128, kk), 128, 0, st>>>(vt, m, mp, order, kk, q);
  for (int pass = 0; pass < 2; ++pass) {
    gemm64(q, kk, 1, q, kk, 0, h, kk, kk, kk, m, st);
    FKK_COUNT_LAUNCH(); ns_apply_kernel<<<m, 128, kk * sizeof(double), st>>>(q, m, kk, h);
  }
  // 3. H = Q^T G Q
  gemm64(g, m, 0, q, kk, 0, y, kk, m, kk, m, st);
  gemm64(q, kk, 1, y, kk, 0, h, kk, kk, kk, m, st);
  FKK_CUDA(ctx, cudaGetLastError());
  // 4. fp64 Jacobi on H (one block; a padded odd size gets a -inf diagonal
  //    entry that sorts last), then V_k = Q W
  const size_t ssm = (size_t)(2 * nsm * nsm + nsm) * sizeof(double);
  FKK_CUDA(ctx, cudaFuncSetAttribute(small_jacobi64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm));
  FKK_COUNT_LAUNCH(); small_jacobi64_kernel<<<1, 512, ssm, st>>>(h, kk, nsm, 1e-14, hw, ww, ctx->d_status);
  int* order2 = (int*)workspace(ctx, "eig_order2", (size_t)nsm * 4, &s);
  if (!order2) return s;
  FKK_COUNT_LAUNCH(); rank_kernel<double><<<(nsm + 127) / 128, 128, 0, st>>>(hw, nsm, nsm, order2, k);
  FKK_COUNT_LAUNCH(); finish_kernel<<<k, 256, 0, st>>>(q, m, kk, hw, ww, nsm, order2, k, lam, v);
  return cuda_check(ctx, cudaGetLastError(), "eig refinement");
}

}  // namespace fkk
