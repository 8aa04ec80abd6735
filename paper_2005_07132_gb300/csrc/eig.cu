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
// Before the sweeps, the dominant eigenpair (rho, x) is found by fp64 power
// iteration; when it has converged the sweeps run on G - rho x x^T, so their
// fp32 rounding is relative to the second eigenvalue rather than the first.
//
// Refinement: Q = orth([x, V_K'-1]) by Newton-Schulz steps in fp64,
// H = Q^T G Q with the original G, H = W diag(theta) W^T by a one-block fp64
// Jacobi method, V_k = Q W[:, top k], lambda = theta.
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
  int cpp;          // CTAs per block pair (phase 2 split)
  int inner_sweeps;
  long long* phase_cycles;  // optional: block 0 accumulates clock64 per phase (8 words)
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

// fp32 rotation with fast division / reciprocal square root: the resulting
// E is re-orthonormalised afterwards, so only the reduction of the
// off-diagonal entry matters here.
__device__ __forceinline__ void sym_schur2_fast(float app, float aqq, float apq, float& c, float& s) {
  float tau = __fdividef(aqq - app, 2.f * apq);
  float t = copysignf(1.f, tau) * __frcp_rn(fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
  c = rsqrtf(fmaf(t, t, 1.f));
  s = t * c;
}
__device__ __forceinline__ void rotation(float app, float aqq, float apq, float& c, float& s) {
  sym_schur2_fast(app, aqq, apq, c, s);
}
__device__ __forceinline__ void rotation(double app, double aqq, double apq, double& c, double& s) {
  sym_schur2(app, aqq, apq, c, s);
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
                                            int tid, int nsweeps) {
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
  for (int rr = 0; rr < nsweeps * (kJ - 1); ++rr) {
    const int r = rr % (kJ - 1);
    if (tid < kJ / 2) {
      const int p = kPair16[r][tid][0], q = kPair16[r][tid][1];
      T apq = S[p][q];
      T c = T(1), s = T(0);
      if (significant(S[p][p], S[q][q], apq, tol)) rotation(S[p][p], S[q][q], apq, c, s);
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
  // phase clock (block 0, thread 0) when p.phase_cycles is set:
  // 0 S load, 1 inner sweeps, 2 Newton-Schulz, 3 phase 2a, 4 barrier, 5 phase 2b, 6 barrier
  long long pc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long t_prev = 0;
  const bool prof = p.phase_cycles && blockIdx.x == 0 && threadIdx.x == 0;
#define FKK_PHASE(i)                         \
  if (prof) {                                \
    long long t_now = clock64();             \
    pc[i] += t_now - t_prev;                 \
    t_prev = t_now;                          \
  }
  __shared__ T S[kJ][kJ + 1];
  __shared__ T E[kJ][kJ + 1];
  __shared__ T F[kJ][kJ + 1];
  __shared__ __align__(16) T Ev[kJ][kJ];  // the (re-orthonormalised) rotation, row-major
  __shared__ T cs_c[kJ / 2], cs_s[kJ / 2];
  __shared__ int J[kJ];
  __shared__ int rot_s;
  extern __shared__ __align__(16) unsigned char stage_raw[];
  T* stage = reinterpret_cast<T*>(stage_raw);  // kJ x (mp / cpp) staging
  using V = typename V4<T>::type;
  constexpr int VN = V4<T>::n;
  const int tid = threadIdx.x;
  const int mp = p.mp;
  const int pair = blockIdx.x / p.cpp, part = blockIdx.x % p.cpp;
  const int span = mp / p.cpp;             // columns (2a) / rows (2b) of this CTA
  const int c0 = part * span;
  unsigned target = 0;
  int sweep = 0;
  bool ok = true;
  for (; sweep < p.max_sweeps && ok; ++sweep) {
    for (int r = 0; r < p.nblk - 1 && ok; ++r) {
      int P, Q;
      if (prof) t_prev = clock64();
      circle_pair(pair, r, p.nblk, P, Q);
      if (tid < kJ) J[tid] = (tid < kB) ? P * kB + tid : Q * kB + (tid - kB);
      __syncthreads();
      {
        int a = tid / kJ, b = tid % kJ;  // 256 threads = 16 x 16
        T x = p.gw[(int64_t)J[a] * mp + J[b]];
        T y = p.gw[(int64_t)J[b] * mp + J[a]];
        S[a][b] = T(0.5) * (x + y);
      }
      __syncthreads();
      FKK_PHASE(0);
      // phase 1 (every CTA of the pair computes the same E)
      const bool rot = inner_sweep<T>(S, E, cs_c, cs_s, &rot_s, p.tol, tid, p.inner_sweeps);
      FKK_PHASE(1);
      if (rot && part == 0 && tid == 0) atomicAdd(&p.sweep_rot[sweep], 1);
      if (!rot) {
        ok = grid_sync(p.bar, gridDim.x, target, p.abort_flag, p.status);
        if (ok) ok = grid_sync(p.bar, gridDim.x, target, p.abort_flag, p.status);
        continue;
      }
      {
        const int a = tid / kJ, b = tid % kJ;
        if (sizeof(T) == 4) {
          // Newton-Schulz: E <- E (3 I - E^T E) / 2
          T f = T(0);
#pragma unroll
          for (int q = 0; q < kJ; ++q) f += E[q][a] * E[q][b];
          F[a][b] = f;
          __syncthreads();
          T e = T(0);
#pragma unroll
          for (int q = 0; q < kJ; ++q) e += E[a][q] * ((q == b ? T(3) : T(0)) - F[q][b]);
          Ev[a][b] = T(0.5) * e;
        } else {
          Ev[a][b] = E[a][b];
        }
        __syncthreads();
      }
      FKK_PHASE(2);
      // phase 2a: rows J of Gw and V^T, columns [c0, c0 + span), <- E^T rows;
      // both matrices staged together (rows 0..15 Gw, 16..31 V^T)
      {
        const int nv = span / VN;
        const int total = 2 * kJ * nv;
        // all of a thread's loads are issued before any shared-memory store
        for (int base = 0; base < total; base += kThreads * 8) {
          V r8[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int idx = base + u * kThreads + tid;
            if (idx < total) {
              const int a = idx / nv, cv = idx - a * nv;
              r8[u] = reinterpret_cast<const V*>((a < kJ ? p.gw : p.vt) + (int64_t)J[a & (kJ - 1)] * mp + c0)[cv];
            }
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int idx = base + u * kThreads + tid;
            if (idx < total) reinterpret_cast<V*>(stage)[idx] = r8[u];
          }
        }
        __syncthreads();
        for (int c = tid; c < 2 * span; c += kThreads) {
          const int mat = c >= span;
          const int cc = c - mat * span;
          T* col = stage + mat * kJ * span + cc;
          asm volatile("" ::: "memory");  // keep the rotation reads inside the loop (no hoisting to registers)
          T acc[kJ];
#pragma unroll
          for (int b = 0; b < kJ; ++b) acc[b] = T(0);
#pragma unroll
          for (int a = 0; a < kJ; ++a) {
            const T ga = col[a * span];
#pragma unroll
            for (int b4 = 0; b4 < kJ; b4 += VN) {
              V e = *reinterpret_cast<const V*>(&Ev[a][b4]);
              if constexpr (VN == 4) {
                acc[b4] = fma(e.x, ga, acc[b4]);
                acc[b4 + 1] = fma(e.y, ga, acc[b4 + 1]);
                acc[b4 + 2] = fma(e.z, ga, acc[b4 + 2]);
                acc[b4 + 3] = fma(e.w, ga, acc[b4 + 3]);
              } else {
                acc[b4] = fma(e.x, ga, acc[b4]);
                acc[b4 + 1] = fma(e.y, ga, acc[b4 + 1]);
              }
            }
          }
#pragma unroll
          for (int b = 0; b < kJ; ++b) col[b * span] = acc[b];
        }
        __syncthreads();
        for (int a = 0; a < 2 * kJ; ++a) {
          T* dst = (a < kJ ? p.gw : p.vt) + (int64_t)J[a & (kJ - 1)] * mp + c0;
          for (int cv = tid; cv < nv; cv += kThreads)
            reinterpret_cast<V*>(dst)[cv] = reinterpret_cast<const V*>(stage + a * span)[cv];
        }
      }
      FKK_PHASE(3);
      ok = grid_sync(p.bar, gridDim.x, target, p.abort_flag, p.status);
      FKK_PHASE(4);
      if (!ok) break;
      // phase 2b: rows [c0, c0 + span) of columns J of Gw <- columns E
      {
        constexpr int vpb = kB / VN;  // vectors per 8-wide segment
        const int total = span * 2 * vpb;
        for (int base = 0; base < total; base += kThreads * 8) {
          V r8[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int t = base + u * kThreads + tid;
            if (t < total) {
              const int rr = t / (2 * vpb), q = t % (2 * vpb);
              const int seg = q / vpb, v = q % vpb;
              const int col0 = (seg ? J[kB] : J[0]) + v * VN;
              r8[u] = *reinterpret_cast<const V*>(p.gw + (int64_t)(c0 + rr) * mp + col0);
            }
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int t = base + u * kThreads + tid;
            if (t < total) {
              const int rr = t / (2 * vpb), q = t % (2 * vpb);
              const int seg = q / vpb, v = q % vpb;
              reinterpret_cast<V*>(stage + rr * kJ + seg * kB)[v] = r8[u];
            }
          }
        }
        __syncthreads();
        for (int rr = tid; rr < span; rr += kThreads) {
          T* row = stage + rr * kJ;
          asm volatile("" ::: "memory");
          T acc[kJ];
#pragma unroll
          for (int b = 0; b < kJ; ++b) acc[b] = T(0);
#pragma unroll
          for (int a = 0; a < kJ; ++a) {
            const T ha = row[a];
#pragma unroll
            for (int b4 = 0; b4 < kJ; b4 += VN) {
              V e = *reinterpret_cast<const V*>(&Ev[a][b4]);
              if constexpr (VN == 4) {
                acc[b4] = fma(ha, e.x, acc[b4]);
                acc[b4 + 1] = fma(ha, e.y, acc[b4 + 1]);
                acc[b4 + 2] = fma(ha, e.z, acc[b4 + 2]);
                acc[b4 + 3] = fma(ha, e.w, acc[b4 + 3]);
              } else {
                acc[b4] = fma(ha, e.x, acc[b4]);
                acc[b4 + 1] = fma(ha, e.y, acc[b4 + 1]);
              }
            }
          }
#pragma unroll
          for (int b = 0; b < kJ; ++b) row[b] = acc[b];
        }
        __syncthreads();
        for (int t = tid; t < span * 2 * vpb; t += kThreads) {
          const int rr = t / (2 * vpb), q = t % (2 * vpb);
          const int seg = q / vpb, v = q % vpb;
          const int col0 = (seg ? J[kB] : J[0]) + v * VN;
          *reinterpret_cast<V*>(p.gw + (int64_t)(c0 + rr) * mp + col0) =
              reinterpret_cast<const V*>(stage + rr * kJ + seg * kB)[v];
        }
      }
      FKK_PHASE(5);
      ok = grid_sync(p.bar, gridDim.x, target, p.abort_flag, p.status);
      FKK_PHASE(6);
    }
    if (!ok) break;
    if (*(volatile int*)&p.sweep_rot[sweep] == 0) {
      ++sweep;
      break;
    }
  }
#undef FKK_PHASE
  if (prof)
    for (int i = 0; i < 8; ++i) p.phase_cycles[i] = pc[i];
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

__global__ void diag_start_kernel(const double* __restrict__ g, int m, double* __restrict__ x) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) x[j] = sqrt(fabs(g[(int64_t)j * m + j])) + 1e-300;
}

// y = G x (fp64, m x m row-major): one warp per row.
__global__ void matvec64_kernel(const double* __restrict__ g, int m, const double* __restrict__ x,
                                double* __restrict__ y) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  double s = 0.0;
  for (int j = lane; j < m; j += 32) s = fma(g[(int64_t)row * m + j], x[j], s);
  s = warp_sum(s);
  if (lane == 0) y[row] = s;
}

// x <- y / ||y||; scal[0] = x^T y_prev-style Rayleigh quotient (y . x_old),
// scal[1] = ||y||.  One block.
__global__ void normalize64_kernel(double* __restrict__ x, const double* __restrict__ y, int m,
                                   double* __restrict__ scal) {
  __shared__ double red[2][32];
  double ss = 0.0, rq = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    ss = fma(y[j], y[j], ss);
    rq = fma(y[j], x[j], rq);
  }
  ss = warp_sum(ss);
  rq = warp_sum(rq);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = ss;
    red[1][threadIdx.x >> 5] = rq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    red[0][0] = sqrt(a);
    scal[0] = b;  // x^T G x for the unit x
    scal[1] = red[0][0];
  }
  __syncthreads();
  const double inv = red[0][0] > 0.0 ? 1.0 / red[0][0] : 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) x[j] = y[j] * inv;
}

// Deflation test: with the power-iteration pair (rho = x^T G x, y = G x),
// flag[0] = 1 when ||y - rho x|| <= 1e-9 rho.  One block.
__global__ void deflate_test_kernel(const double* __restrict__ x, const double* __restrict__ y, int m,
                                    const double* __restrict__ scal, int* __restrict__ flag) {
  __shared__ double red[32];
  const double rho = scal[0];
  double r2 = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    double d = y[j] - rho * x[j];
    r2 = fma(d, d, r2);
  }
  r2 = warp_sum(r2);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    flag[0] = (rho > 0.0 && sqrt(t) <= 1e-9 * rho) ? 1 : 0;
  }
}

// Gd = G - rho x x^T when flag[0], else Gd = G.  grid = (cols, m).
__global__ void deflate64_kernel(const double* __restrict__ g, int m, const double* __restrict__ x,
                                 const double* __restrict__ scal, const int* __restrict__ flag,
                                 double* __restrict__ gd) {
  const int r = blockIdx.y;
  const int use = flag[0];
  const double rho = scal[0];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
    double v = g[(int64_t)r * m + c];
    if (use) v -= rho * x[r] * x[c];
    gd[(int64_t)r * m + c] = v;
  }
}

// Leading refinement basis: column 0 = x (when deflated), then the largest
// Jacobi vectors of the deflated matrix.  X[j, c] row-major m x kk.
template <typename T>
__global__ void gather_defl_kernel(const T* __restrict__ vt, int m, int mp, const int* __restrict__ order, int kk,
                                   const double* __restrict__ x, const int* __restrict__ flag,
                                   double* __restrict__ out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (j >= m) return;
  const int use = flag[0];
  double v;
  if (use && c == 0) v = x[j];
  else v = (double)vt[(int64_t)order[use ? c - 1 : c] * mp + j];
  out[(int64_t)j * kk + c] = v;
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
  int cpp = 1;
  while (cpp < 4 && (int64_t)npairs * cpp * 2 <= ctx->sm_count && (mp / (cpp * 2)) % V4<T>::n == 0) cpp *= 2;
  const size_t stage_bytes = (size_t)2 * kJ * (mp / cpp) * sizeof(T);
  FKK_CUDA(ctx, cudaFuncSetAttribute(block_jacobi_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stage_bytes));
  int per_sm = 0;
  FKK_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, block_jacobi_kernel<T>, kThreads, stage_bytes));
  if ((int64_t)per_sm * ctx->sm_count < (int64_t)npairs * cpp)
    return fail(ctx, FKK_ERR_INVALID_ARG, "eigensolve: %d block pairs exceed co-resident capacity", npairs);
  long long* pcyc = nullptr;
  if (ctx->timing) {
    pcyc = (long long*)workspace(ctx, "eig_phase_cycles", 8 * sizeof(long long), &s);
    if (!pcyc) return s;
  }
  JacobiArgs<T> a{gw, vt, mp, nblk, tol, max_sweeps, bar, abort_flag, sweep_rot, sweeps_done, ctx->d_status,
                  cpp, 1, pcyc};
  void* args[] = {&a};
  FKK_COUNT_LAUNCH();
  FKK_CUDA(ctx, cudaLaunchCooperativeKernel((void*)block_jacobi_kernel<T>, dim3(npairs * cpp), dim3(kThreads), args,
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
  // 0. dominant eigenpair by fp64 power iteration; when it has converged
  //    (residual <= 1e-9 rho) the fp32 Jacobi works on G - rho x x^T, whose
  //    norm is the second eigenvalue, so its rounding is relative to that
  double* pw = (double*)workspace(ctx, "eig_pw", (size_t)(2 * m + 8) * 8, &s);
  if (!pw) return s;
  double* px = pw;
  double* py = pw + m;
  double* scal = pw + 2 * m;
  int* flag = (int*)workspace(ctx, "eig_flag", 64, &s);
  if (!flag) return s;
  double* gd = (double*)workspace(ctx, "eig_gd", (size_t)m * m * 8, &s);
  if (!gd) return s;
  {
    // start from the diagonal (all positive for a Gram matrix)
    FKK_COUNT_LAUNCH(); diag_start_kernel<<<(m + 255) / 256, 256, 0, st>>>(g, m, px);
    for (int it = 0; it < 60; ++it) {
      FKK_COUNT_LAUNCH(); matvec64_kernel<<<(m + 7) / 8, 256, 0, st>>>(g, m, px, py);
      FKK_COUNT_LAUNCH(); normalize64_kernel<<<1, 1024, 0, st>>>(px, py, m, scal);
    }
    FKK_COUNT_LAUNCH(); matvec64_kernel<<<(m + 7) / 8, 256, 0, st>>>(g, m, px, py);
    FKK_COUNT_LAUNCH(); deflate_test_kernel<<<1, 1024, 0, st>>>(px, py, m, scal, flag);
    FKK_COUNT_LAUNCH(); deflate64_kernel<<<dim3((m + 255) / 256, m), 256, 0, st>>>(g, m, px, scal, flag, gd);
    FKK_CUDA(ctx, cudaGetLastError());
  }
  // 1. fp32 block Jacobi over the whole (deflated) matrix
  float* gw;
  float* vt;
  int mp;
  FKK_TRY(run_block_jacobi<float>(ctx, "eig32", gd, m, m, (float)(tol32 > 0 ? tol32 : 1e-6),
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
  FKK_COUNT_LAUNCH(); gather_defl_kernel<float><<<dim3((m + 127) / 128, kk), 128, 0, st>>>(vt, m, mp, order, kk, px,
                                                                                            flag, q);
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
