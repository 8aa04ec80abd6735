// Symmetric eigensolve of the Gram matrix for its k largest eigenpairs
// (Sec. 2.2: V and S of the SVD of A follow from G = A^T A = V S^2 V^T):
//   1. Householder reduction Q^T G Q = T to symmetric tridiagonal form in one
//      persistent cooperative kernel with one tagged all-to-all exchange per
//      column (no grid barrier);
//   2. the k largest eigenvalues of T by Sturm-count multisection;
//   3. one eigenvector of T per eigenvalue from the twisted factorisation of
//      T - lambda I (the index where the eigenvector is largest is found
//      from the two one-sided factorisations, and the vector follows from
//      products of their ratios);
//   4. V = Q Z with the reflectors applied 32 at a time in the compact WY
//      form I - Y T Y^T, then a Cholesky-QR pass in fp64 and the sign
//      convention (largest-magnitude component positive).
// Steps 1-4 run in double-word arithmetic on the fp32 pipe (df64.cuh, about
// 48 significant bits) on G scaled by a power of two; fp64 is used only to
// read G and for the final Cholesky QR.
//
// Reduction, step j (reflector H_j = I - tau v v^T, v[j+1] = 1, zero above):
//   p = tau A v,  w = p - (tau/2)(p.v) v,  A <- A - v w^T - w v^T
// on the trailing rows/columns j+1..m-1.  Column c belongs to CTA c mod G and
// stays in its shared memory (global memory when the matrix is too large);
// warp s of a CTA updates its s-th column.  Every CTA forms the next
// reflector v' itself from the published pivot column and the full p.  The
// p of the next step is then taken from the columns before this step's
// update, corrected by the two scalars v.v' and w.v', and published; the
// update itself follows while the other CTAs publish theirs.  So the
// critical path of a step is the exchange, the reflector and one dot product
// per column; there is no grid barrier (the exchanged words carry their step
// in two tag bits).
#include <algorithm>

#include "common.cuh"
#include "df64.cuh"
#include "fit.h"

namespace fkk {
namespace {

using dw::df;

// The reduction runs 256 threads per CTA up to m = 1,024 (fewer warps to
// combine in each step's block reductions: 6.19 against 6.49 ms for the
// eigensolve at m = 1,000) and 512 beyond; every warp takes part in the
// length-m vector phases and owns at most one column: m <= warps * grid.
constexpr int kTrThreadsSmall = 256, kTrThreadsLarge = 512;
constexpr int kWY = 32;            // reflectors per block in the back-transformation
constexpr int kBisWarps = 4;       // warps per eigenvalue; multisection points per round: 64 * kBisWarps
constexpr float kEpsF = 5.9604645e-08f;  // 2^-24

// Reflector from alpha (first entry) and sigma = sum of squares of the rest
// (LAPACK dlarfg convention): H x = beta e_1, tau = (beta - alpha) / beta,
// v = x / (alpha - beta) below the first entry.  sc = {tau, beta, scal}.
__device__ __forceinline__ void reflector(df alp, df sig, df* sc) {
  if (sig.h == 0.f) {
    sc[0] = dw::make(0.f);
    sc[1] = alp;
    sc[2] = dw::make(0.f);
    return;
  }
  const df mu = dw::sqrt(dw::add(dw::mul(alp, alp), sig));
  const df beta = alp.h <= 0.f ? mu : dw::neg(mu);
  sc[0] = dw::div(dw::sub(beta, alp), beta);
  sc[1] = beta;
  sc[2] = dw::rcp(dw::sub(alp, beta));
}

// Words exchanged between CTAs: a double-word value with a 2-bit step tag in
// the two lowest bits of its low float, written and read as one 64-bit
// access, so a reader knows from the word itself whether it is current.
// Tags alternate 1, 2 between the consecutive uses of a double-buffered
// slot; 0 (the cleared buffer) is never current.
__device__ __forceinline__ unsigned step_tag(int s) { return 1u + ((s >> 1) & 1u); }
__device__ __forceinline__ unsigned long long pack_tag(df x, unsigned tag) {
  const unsigned lo = (__float_as_uint(x.l) & ~3u) | tag;
  return ((unsigned long long)__float_as_uint(x.h) << 32) | lo;
}
__device__ __forceinline__ df unpack_tag(unsigned long long w) {
  return {__uint_as_float((unsigned)(w >> 32)), __uint_as_float((unsigned)w & ~3u)};
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v));
}
constexpr int kMaxPer = 4;  // vector entries per vector thread: m <= kMaxPer * threads
constexpr int kRedA = 48;   // partials of p.v in red[48..64); the three sums of phase B use red[0..48)

// Loads the words at p[i] and q[i], i = i0 + r * stride (r < kMaxPer,
// lo <= i < m) -- the p words and the pivot column of a step -- all in flight
// at once, and re-polls those not yet carrying `tag` until every one does
// (bounded), so a column that is already published costs no round trip of
// its own after the p words arrive.  On timeout records FKK_ERR_TIMEOUT and
// raises the abort flag; returns false then, or when another CTA has aborted.
__device__ __forceinline__ bool gather_tagged(const unsigned long long* p, const unsigned long long* q, int i0,
                                               int stride, int lo, int m, unsigned tag,
                                               unsigned long long (&wp)[kMaxPer], unsigned long long (&wq)[kMaxPer],
                                               int* abort_flag, long long* status, unsigned limit) {
  unsigned pending = 0;  // bit r: wp[r]; bit kMaxPer + r: wq[r]
#pragma unroll
  for (int r = 0; r < kMaxPer; ++r) {
    const int i = i0 + r * stride;
    wp[r] = 0;
    wq[r] = 0;
    if (i >= lo && i < m) {
      wp[r] = ld_relaxed_u64(p + i);
      wq[r] = ld_relaxed_u64(q + i);
      pending |= (1u << r) | (1u << (kMaxPer + r));
    }
  }
  unsigned it = 0;
  for (;;) {
#pragma unroll
    for (int r = 0; r < kMaxPer; ++r) {
      if (((pending >> r) & 1u) && ((unsigned)wp[r] & 3u) == tag) pending &= ~(1u << r);
      if (((pending >> (kMaxPer + r)) & 1u) && ((unsigned)wq[r] & 3u) == tag) pending &= ~(1u << (kMaxPer + r));
    }
    if (!pending) return true;
    if ((++it & 63u) == 0) {
      if (*(volatile int*)abort_flag) return false;
      if (it > limit) {
        atomicExch(abort_flag, 1);
        record_error(status, kErrTimeout);
        return false;
      }
    }
#pragma unroll
    for (int r = 0; r < kMaxPer; ++r) {
      if ((pending >> r) & 1u) wp[r] = ld_relaxed_u64(p + i0 + r * stride);
      if ((pending >> (kMaxPer + r)) & 1u) wq[r] = ld_relaxed_u64(q + i0 + r * stride);
    }
  }
}

// Sum of one double-word per vector warp (red[0..kVecWarps)), formed by any
// warp: each group of kVecWarps lanes runs the same butterfly over the same
// partials (and dw::add is commutative bit for bit), so every lane of every
// warp gets the same value.
template <int kVecWarps>
__device__ __forceinline__ df sum_vec_partials(const df* red) {
  static_assert((kVecWarps & (kVecWarps - 1)) == 0 && kVecWarps <= 32, "power-of-two warp count");
  const int lane = threadIdx.x & 31;
  df t = red[lane & (kVecWarps - 1)];
#pragma unroll
  for (int o = kVecWarps / 2; o > 0; o >>= 1) t = dw::add(t, dw::shfl_xor(t, o));
  return t;
}

struct TridArgs {
  const double* g;  // m x m symmetric, row-major (row c = column c)
  int m;
  int ncol_max;     // ceil(m / grid)
  df* work;         // m x m working columns when they do not fit in shared memory
  unsigned long long* pbuf;  // [2][m] tagged p of the next step, by column (cleared by the host)
  unsigned long long* cbuf;  // [2][m] tagged next pivot column (cleared by the host)
  df* d;            // [m] diagonal of T (scaled)
  df* e;            // [m] sub-diagonal of T (scaled; e[m-1] = 0)
  df* tau;          // [m] reflector scalars
  df* u;            // [m][m] row j = reflector vector of step j
  unsigned* maxbits;  // max |G| as float bits (atomicMax), zeroed by the host
  int* ex_out;      // T = 2^ex Ts
  long long* cycles;  // optional [8]: SM clock cycles of CTA 0 per phase
  unsigned* bar;
  int* abort_flag;
  long long* status;
  unsigned wait_limit;  // polls before an exchange wait gives up (FKK_ERR_TIMEOUT)
  int stall;            // test knob: step 0 waits for tag 0, which no step publishes
};

template <bool kSmem, int kTrThreads>
__global__ void __launch_bounds__(kTrThreads, 1) tridiag_kernel(TridArgs a) {
  constexpr int kTrWarps = kTrThreads / 32;
  constexpr int kVecWarps = kTrWarps;  // warps that run the length-m vector phases
  constexpr int kVecThreads = kVecWarps * 32;
  static_assert(3 * kVecWarps <= kRedA && kRedA + kVecWarps <= 64, "partial slots overlap");
  extern __shared__ df smd[];
  const int m = a.m, nb = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const bool vecw = warp < kVecWarps;
  const int nloc = (m - b + nb - 1) / nb;  // own columns c = b + s * nb
  const int c_last = b + (nloc - 1) * nb;   // last own column
  // the owner of column m-1 takes part in every step and writes T and the
  // reflectors; a CTA whose columns are all reduced leaves (nobody waits on
  // it any more, so it must not read exchange buffers others may reuse)
  const bool writer = b == (m - 1) % nb;
  df* cols = smd;
  df* v = smd + (kSmem ? (size_t)a.ncol_max * m : 0);
  df* vn = v + m;
  df* w = vn + m;
  df* red = w + m;   // [64]
  df* sc = red + 64; // [8] scalars
  __shared__ float fmax_s[kTrWarps];
  __shared__ int ex_s;
  unsigned target = 0;
  auto colp = [&](int s) -> df* {
    return kSmem ? cols + (size_t)s * m : a.work + (size_t)(b + s * nb) * m;
  };
  const bool timed = a.cycles != nullptr && writer && tid == 0;
  long long cyc[5] = {0, 0, 0, 0, 0};
  long long t_prev = timed ? clock64() : 0;
  auto mark = [&](int ph) {
    if (timed) {
      const long long t = clock64();
      cyc[ph] += t - t_prev;
      t_prev = t;
    }
  };

  // own columns in double-word, and max |G| over the whole matrix
  float mx = 0.f;
  for (int s = 0; s < nloc; ++s) {
    const double* src = a.g + (size_t)(b + s * nb) * m;
    df* dst = colp(s);
    for (int i = tid; i < m; i += kTrThreads) {
      const df x = dw::from_double(src[i]);
      dst[i] = x;
      mx = fmaxf(mx, fabsf(x.h));
    }
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) fmax_s[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int q = 0; q < kTrWarps; ++q) t = fmaxf(t, fmax_s[q]);
    atomicMax(a.maxbits, __float_as_uint(t));
  }
  if (!grid_sync(a.bar, nb, target, a.abort_flag, a.status)) return;
  mark(0);
  if (tid == 0) {
    const float t = __uint_as_float(__ldcg(a.maxbits));
    ex_s = t > 0.f ? ilogbf(t) : 0;
    if (b == 0) *a.ex_out = ex_s;
  }
  __syncthreads();
  const int ex = ex_s;
  for (int s = 0; s < nloc; ++s) {
    df* col = colp(s);
    for (int i = tid; i < m; i += kTrThreads) col[i] = dw::ldexp(col[i], -ex);
  }
  if (m <= 2) {
    if (writer && tid == 0) {
      a.d[0] = dw::ldexp(dw::from_double(a.g[0]), -ex);
      a.e[0] = dw::make(0.f);
      if (m == 2) {
        a.d[1] = dw::ldexp(dw::from_double(a.g[3]), -ex);
        a.e[0] = dw::ldexp(dw::from_double(a.g[2]), -ex);
      }
    }
    return;
  }

  // reflector of step 0 from column 0
  {
    df sig = dw::make(0.f);
    if (vecw)
      for (int i = tid; i < m; i += kVecThreads) {
        const df x = i >= 1 ? dw::ldexp(dw::from_double(a.g[i]), -ex) : dw::make(0.f);
        vn[i] = x;
        if (i >= 2) sig = dw::add(sig, dw::mul(x, x));
      }
    if (vecw) {
      sig = dw::warp_sum(sig);
      if (lane == 0) red[warp] = sig;
    }
    __syncthreads();
    if (warp == 0) {
      const df t = sum_vec_partials<kVecWarps>(red);
      if (lane == 0) {
        reflector(vn[1], t, sc);
        if (writer) {
          a.d[0] = dw::ldexp(dw::from_double(a.g[0]), -ex);
          a.e[0] = sc[1];
          a.tau[0] = sc[0];
        }
      }
    }
    __syncthreads();
    const df scal = sc[2];
    if (vecw)
      for (int i = tid; i < m; i += kVecThreads) {
        const df x = i < 1 ? dw::make(0.f) : (i == 1 ? dw::make(1.f) : dw::mul(vn[i], scal));
        v[i] = x;
        if (writer) a.u[i] = x;
      }
    __syncthreads();
    // p of step 0 and the copy of column 1: warp s takes own column s
    const df tau0 = sc[0];
    const unsigned tag0 = step_tag(0);
    if (warp < nloc) {
      const int c = b + warp * nb;
      const df* col = colp(warp);
      df acc = dw::make(0.f);
      if (c >= 1)
        for (int i = 1 + lane; i < m; i += 32) {
          const df x = col[i];
          acc = dw::add(acc, dw::mul(x, v[i]));
          if (c == 1) st_relaxed_u64(a.cbuf + i, pack_tag(x, tag0));
        }
      acc = dw::warp_sum(acc);
      if (lane == 0 && c >= 1) st_relaxed_u64(a.pbuf + c, pack_tag(dw::mul(tau0, acc), tag0));
    }
  }
  df tau_cur = sc[0];
  df scal_cur = sc[2];  // v of step 0 is already scaled
  mark(0);

  const int nsteps = m - 2;
  for (int j = 0; j < nsteps; ++j) {
    if (c_last < j + 2) break;  // nothing of this CTA's is read from step j on
    const int buf = j & 1, nxt = buf ^ 1;
    const unsigned want = (a.stall && j == 0) ? 0u : step_tag(j);
    const unsigned long long* pb = a.pbuf + (size_t)buf * m;
    const unsigned long long* cb = a.cbuf + (size_t)buf * m;
    const bool last = (j + 1 > m - 3);
    // A. v of this step from the raw pivot column the previous step kept
    //    (each vector thread scales its own entries); gather p and the pivot
    //    column (rows >= j+1) as they arrive; p.v
    df cbr[kMaxPer];
    bool ok = true;
    df dot = dw::make(0.f);
    if (vecw) {
      if (j > 0) {
#pragma unroll
        for (int r = 0; r < kMaxPer; ++r) {
          const int i = tid + r * kVecThreads;
          if (i < m) {
            const df x = i <= j ? dw::make(0.f) : (i == j + 1 ? dw::make(1.f) : dw::mul(v[i], scal_cur));
            v[i] = x;
            if (writer) a.u[(size_t)j * m + i] = x;
          }
        }
      }
      unsigned long long wp[kMaxPer], wcb[kMaxPer];
      ok = gather_tagged(pb, cb, tid, kVecThreads, j + 1, m, want, wp, wcb, a.abort_flag, a.status, a.wait_limit);
#pragma unroll
      for (int r = 0; r < kMaxPer; ++r) {
        const int i = tid + r * kVecThreads;
        cbr[r] = dw::make(0.f);
        if (i < m) {
          df p = dw::make(0.f);
          if (i >= j + 1) {
            p = unpack_tag(wp[r]);
            cbr[r] = unpack_tag(wcb[r]);
            dot = dw::add(dot, dw::mul(p, v[i]));
          }
          w[i] = p;
        }
      }
      dot = dw::warp_sum(dot);
      if (lane == 0) red[kRedA + warp] = dot;
    }
    if (!__syncthreads_and(ok)) return;
    // every warp sums the partials itself (the same butterfly, so the same
    // value in every warp) instead of one warp and a second barrier
    const df halfk = dw::mul(dw::mul(tau_cur, sum_vec_partials<kVecWarps>(red + kRedA)), 0.5f);
    const df wj1 = dw::sub(w[j + 1], halfk);  // w_{j+1} = p_{j+1} - halfk v_{j+1}, v_{j+1} = 1
    mark(1);
    // B. w = p - halfk v; pivot column x = c - v w_{j+1} - w after this
    //    step's update, kept raw; the next reflector from x, with
    //    alpha = v.v' and beta = w.v' (v' = e_{j+2} + scal x below row j+2)
    df sig = dw::make(0.f), vx = dw::make(0.f), wx = dw::make(0.f);
    if (vecw) {
#pragma unroll
      for (int r = 0; r < kMaxPer; ++r) {
        const int i = tid + r * kVecThreads;
        if (i < m && i >= j + 1) {
          const df vi = v[i];
          const df wi = dw::fnma(halfk, vi, w[i]);
          if (i != j + 1) w[i] = wi;  // every warp read w[j+1] above; no one reads it after
          const df x = dw::sub(dw::fnma(vi, wj1, cbr[r]), wi);
          vn[i] = x;
          if (i == j + 1 && writer) a.d[j + 1] = x;
          if (last) {
            if (i == m - 1 && writer) a.e[m - 2] = x;
          } else if (i >= j + 3) {
            sig = dw::add(sig, dw::mul(x, x));
            vx = dw::add(vx, dw::mul(vi, x));
            wx = dw::add(wx, dw::mul(wi, x));
          }
        }
      }
    }
    df tau_nxt = dw::make(0.f), scal = dw::make(0.f);
    df s6 = dw::make(0.f), s7 = dw::make(0.f);  // v.v' and w.v' of the next reflector
    if (!last) {
      if (vecw) {
        sig = dw::warp_sum(sig);
        vx = dw::warp_sum(vx);
        wx = dw::warp_sum(wx);
        if (lane == 0) {
          red[warp] = sig;
          red[kVecWarps + warp] = vx;
          red[2 * kVecWarps + warp] = wx;
        }
      }
      __syncthreads();
      // the next reflector, formed by every warp from the same partials
      const df ts = sum_vec_partials<kVecWarps>(red);
      const df tv = sum_vec_partials<kVecWarps>(red + kVecWarps);
      const df tw = sum_vec_partials<kVecWarps>(red + 2 * kVecWarps);
      df rf[3];
      reflector(vn[j + 2], ts, rf);
      s6 = dw::add(v[j + 2], dw::mul(rf[2], tv));
      s7 = dw::add(w[j + 2], dw::mul(rf[2], tw));
      if (writer && tid == 0) {
        a.e[j + 1] = rf[1];
        a.tau[j + 1] = rf[0];
      }
      tau_nxt = rf[0];
      scal = rf[2];
    } else {
      __syncthreads();
    }
    mark(2);
    // C1. p of the next step from the owned columns as they are before this
    //     step's update:  A'v' = A v' - v (w.v') - w (v.v')  column by column,
    //     A v' = A[j+2, c] + scal (A[j+3.., c] . x); published at once.  The
    //     owner of column j+2 also publishes that column after the update.
    if (warp < nloc) {
      const int c = b + warp * nb;
      if (c >= j + 2) {
        const df* col = colp(warp);
        const df wc = w[c], vc = v[c];
        if (last) {
          // c == m - 1: the last diagonal entry
          if (lane == 0) a.d[m - 1] = dw::sub(col[m - 1], dw::add(dw::mul(v[m - 1], wc), dw::mul(w[m - 1], vc)));
        } else {
          const unsigned tagn = step_tag(j + 1);
          df acc = dw::make(0.f);
          if (c == j + 2) {
            unsigned long long* cnext = a.cbuf + (size_t)nxt * m;
            for (int i = j + 2 + lane; i < m; i += 32) {
              const df y = col[i];
              st_relaxed_u64(cnext + i, pack_tag(dw::sub(y, dw::add(dw::mul(v[i], wc), dw::mul(w[i], vc))), tagn));
              if (i > j + 2) acc = dw::add(acc, dw::mul(y, vn[i]));
            }
          } else {
            for (int i = j + 3 + lane; i < m; i += 32) acc = dw::add(acc, dw::mul(col[i], vn[i]));
          }
          acc = dw::warp_sum(acc);
          if (lane == 0) {
            const df av = dw::add(col[j + 2], dw::mul(scal, acc));
            const df pc = dw::mul(tau_nxt, dw::sub(av, dw::add(dw::mul(wc, s6), dw::mul(vc, s7))));
            st_relaxed_u64(a.pbuf + (size_t)nxt * m + c, pack_tag(pc, tagn));
          }
        }
      }
    }
    mark(3);
    if (last) break;
    // C2. this step's update of the owned columns c >= j+3 on rows >= j+3
    //     (the rows the next steps read), while the other CTAs publish
    if (warp < nloc) {
      const int c = b + warp * nb;
      if (c >= j + 3) {
        df* col = colp(warp);
        const df wc = w[c], vc = v[c];
        for (int i = j + 3 + lane; i < m; i += 32)
          col[i] = dw::sub(col[i], dw::add(dw::mul(v[i], wc), dw::mul(w[i], vc)));
      }
    }
    mark(4);
    df* tmp = v;
    v = vn;
    vn = tmp;
    tau_cur = tau_nxt;
    scal_cur = scal;
    __syncthreads();  // the column passes read v, w, vn; the next step rewrites them
  }
  if (timed)
    for (int q = 0; q < 5; ++q) a.cycles[q] = cyc[q];
}

// ---------------------------------------------------------------------------
// Tridiagonal eigenvalues and eigenvectors on Ts (largest entry below 2).
// Off-diagonals below 2^-46 sqrt(|d_i d_{i+1}|) are set to zero (the matrix
// splits there).

struct TriBounds {
  float gl, gu;  // Gershgorin bounds, widened
};

// Loads ds, es (es[m-1] = 0) and eb[i] = es[i-1]^2 (eb[0] = 0) into shared
// memory; any number of warps.
__device__ TriBounds load_tri(const df* __restrict__ d, const df* __restrict__ e, int m, df* ds, df* es, df* eb,
                              float* redf) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) ds[i] = d[i];
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    df x = dw::make(0.f);
    if (i < m - 1) {
      x = e[i];
      if (fabsf(x.h) <= 1.4210855e-14f * sqrtf(fabsf(ds[i].h) * fabsf(ds[i + 1].h))) x = dw::make(0.f);
    }
    es[i] = x;
  }
  __syncthreads();
  float lo = 3e38f, hi = -3e38f;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const df el = i > 0 ? es[i - 1] : dw::make(0.f);
    eb[i] = dw::mul(el, el);
    const float r = fabsf(el.h) + fabsf(es[i].h);
    lo = fminf(lo, ds[i].h - r);
    hi = fmaxf(hi, ds[i].h + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    redf[warp] = lo;
    redf[32 + warp] = hi;
  }
  __syncthreads();
  TriBounds t;
  t.gl = 3e38f;
  t.gu = -3e38f;
  for (int q = 0; q < nw; ++q) {
    t.gl = fminf(t.gl, redf[q]);
    t.gu = fmaxf(t.gu, redf[32 + q]);
  }
  const float wid = (fabsf(t.gl) + fabsf(t.gu)) * 1e-5f + 1e-30f;
  t.gl -= wid;
  t.gu += wid;
  __syncthreads();
  return t;
}

// Power of two bringing the larger of two floats' exponents to zero, when
// that exponent has left [-32, 32] (else 1): exact rescaling by exponent bits.
__device__ __forceinline__ float rescale_factor(float a, float b) {
  const int ea = (__float_as_int(a) >> 23) & 0xff, eb = (__float_as_int(b) >> 23) & 0xff;
  const int e = max(ea, eb);
  if (e > 127 + 32 || e < 127 - 32) return __int_as_float(max(1, min(254, 254 - e)) << 23);
  return 1.f;
}

// Number of eigenvalues of Ts below x: sign changes of the leading principal
// minors of Ts - x I (three-term recurrence; an exact zero minor counts as a
// tiny negative pivot).  The minors can shrink by the ratio of the smallest
// to the largest diagonal entry at every step, so the pair is rescaled by a
// power of two whenever the larger leaves [2^-32, 2^32]: the float exponent
// of a double-word would otherwise underflow within a few steps.
// Two counts at once: the two recurrences run side by side on the paired
// fp32 instructions (dw2), which also hides the dependent latency of each.
// Bit-identical to two separate double-word counts.
__device__ __forceinline__ void sturm_count2(const df* ds, const df* eb, int m, df x, df y, int& nx, int& ny) {
  const dw2::df2 xy = dw2::pack(x, y);
  dw2::df2 pq2 = dw2::pack(dw::make(1.f), dw::make(1.f));
  dw2::df2 pq1 = dw2::sub(dw2::splat(ds[0]), xy);
  if (pq1.h.x == 0.f) {
    pq1.h.x = -0x1p-60f;
    pq1.l.x = 0.f;
  }
  if (pq1.h.y == 0.f) {
    pq1.h.y = -0x1p-60f;
    pq1.l.y = 0.f;
  }
  int cx = pq1.h.x < 0.f, cy = pq1.h.y < 0.f;
#pragma unroll 4
  for (int i = 1; i < m; ++i) {
    const dw2::df2 d2 = dw2::splat(ds[i]), e2 = dw2::splat(eb[i]);
    dw2::df2 pq = dw2::sub(dw2::mul(dw2::sub(d2, xy), pq1), dw2::mul(e2, pq2));
    // branch-free: an exact zero becomes a tiny negative multiple of the
    // previous minor; the rescale factor is 1 when none is needed (exact)
    const bool pz = pq.h.x == 0.f, qz = pq.h.y == 0.f;
    pq.h.x = pz ? -0x1p-60f * pq1.h.x : pq.h.x;
    pq.l.x = pz ? 0.f : pq.l.x;
    pq.h.y = qz ? -0x1p-60f * pq1.h.y : pq.h.y;
    pq.l.y = qz ? 0.f : pq.l.y;
    cx += (pq.h.x < 0.f) != (pq1.h.x < 0.f);
    cy += (pq.h.y < 0.f) != (pq1.h.y < 0.f);
    const float2 fg = make_float2(rescale_factor(pq.h.x, pq1.h.x), rescale_factor(pq.h.y, pq1.h.y));
    pq2 = {__fmul2_rn(pq1.h, fg), __fmul2_rn(pq1.l, fg)};
    pq1 = {__fmul2_rn(pq.h, fg), __fmul2_rn(pq.l, fg)};
  }
  nx = cx;
  ny = cy;
}

// The same pair of counts in plain fp32 on the leading words: exact for a
// matrix within a few float roundings of Ts, used to bracket before the
// double-word rounds.
__device__ __forceinline__ void sturm_count2_f32(const df* ds, const df* eb, int m, float x, float y, int& nx,
                                                 int& ny) {
  const float2 nxy = make_float2(-x, -y);
  float2 p2 = make_float2(1.f, 1.f);
  float2 p1 = __fadd2_rn(make_float2(ds[0].h, ds[0].h), nxy);
  if (p1.x == 0.f) p1.x = -0x1p-60f;
  if (p1.y == 0.f) p1.y = -0x1p-60f;
  int cx = p1.x < 0.f, cy = p1.y < 0.f;
#pragma unroll 4
  for (int i = 1; i < m; ++i) {
    const float d = ds[i].h, e = eb[i].h;
    float2 p = __ffma2_rn(__fadd2_rn(make_float2(d, d), nxy), p1, __fmul2_rn(make_float2(-e, -e), p2));
    if (p.x == 0.f) p.x = -0x1p-60f * p1.x;
    if (p.y == 0.f) p.y = -0x1p-60f * p1.y;
    cx += (p.x < 0.f) != (p1.x < 0.f);
    cy += (p.y < 0.f) != (p1.y < 0.f);
    const float2 fg = make_float2(rescale_factor(p.x, p1.x), rescale_factor(p.y, p1.y));
    p2 = __fmul2_rn(p1, fg);
    p1 = __fmul2_rn(p, fg);
  }
  nx = cx;
  ny = cy;
}

// First of the 2 x blockDim points (thread t holds points 2t and 2t + 1)
// whose count exceeds r; 2 x blockDim if none.
__device__ __forceinline__ int first_above2(int n0, int n1, int r, int* first_s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // bit pattern over the warp's 64 points, in point order
  const unsigned a0 = __ballot_sync(0xffffffffu, n0 > r), a1 = __ballot_sync(0xffffffffu, n1 > r);
  if (lane == 0) {
    int f = 64;
    const unsigned any = a0 | a1;
    if (any) {
      const int t = __ffs(any) - 1;  // first thread with a crossing
      f = 2 * t + (((a0 >> t) & 1u) ? 0 : 1);
    }
    first_s[warp] = f;
  }
  __syncthreads();
  int first = 2 * (int)blockDim.x;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
    if (first_s[q] < 64) {
      first = q * 64 + first_s[q];
      break;
    }
  return first;
}

// One CTA per eigenvalue: rank r = m-1-c (c = 0 the largest).  Rounds of
// multisection evaluate P = 2 x blockDim points of the bracket [lo, hi]
// (N(lo) <= r < N(hi)) and keep the sub-interval where the count crosses r:
// first in fp32 down to the float resolution, then, from that bracket
// widened by the fp32 count's error bound, in double-word.  The first
// double-word round includes the bracket ends and falls back to the
// Gershgorin interval if they do not bracket rank r.
__global__ void __launch_bounds__(kBisWarps * 32) tri_bisect_kernel(const df* __restrict__ d,
                                                                    const df* __restrict__ e, int m,
                                                                    df* __restrict__ lam) {
  extern __shared__ df smd[];
  df* ds = smd;
  df* es = ds + m;
  df* eb = es + m;
  __shared__ float redf[64];
  __shared__ int first_s[kBisWarps];
  __shared__ df lohi[2];
  __shared__ float flh[2];
  const int P = 2 * kBisWarps * 32;
  const int tid = threadIdx.x;
  const int c = blockIdx.x;
  const int r = m - 1 - c;
  const TriBounds t = load_tri(d, e, m, ds, es, eb, redf);
  const float gmax = fmaxf(fabsf(t.gl), fabsf(t.gu));
  // fp32 rounds
  float flo = t.gl, fhi = t.gu;
  for (int round = 0; round < 8 && fhi - flo > 64.f * kEpsF * gmax; ++round) {
    const float x0 = flo + (fhi - flo) * ((float)(2 * tid + 1) / (float)(P + 1));
    const float x1 = flo + (fhi - flo) * ((float)(2 * tid + 2) / (float)(P + 1));
    int n0, n1;
    sturm_count2_f32(ds, eb, m, x0, x1, n0, n1);
    const int first = first_above2(n0, n1, r, first_s);
    if (first - 1 == 2 * tid) flh[0] = x0;
    if (first - 1 == 2 * tid + 1) flh[0] = x1;
    if (first == 2 * tid) flh[1] = x0;
    if (first == 2 * tid + 1) flh[1] = x1;
    __syncthreads();
    if (first > 0) flo = flh[0];
    if (first < P) fhi = flh[1];
    __syncthreads();
  }
  // double-word rounds
  const float widen = 64.f * kEpsF * gmax;
  df lo = dw::make(flo - widen), hi = dw::make(fhi + widen);
  const float tol = 8.f * kEpsF * kEpsF * gmax;
  bool first_round = true;
  for (int round = 0; round < 24; ++round) {
    const df wid = dw::sub(hi, lo);
    if (wid.h <= tol) break;
    df x0, x1;
    if (first_round) {  // ends included
      x0 = dw::add(lo, dw::mul(wid, (float)(2 * tid) / (float)(P - 1)));
      x1 = dw::add(lo, dw::mul(wid, (float)(2 * tid + 1) / (float)(P - 1)));
    } else {
      x0 = dw::add(lo, dw::mul(wid, (float)(2 * tid + 1) / (float)(P + 1)));
      x1 = dw::add(lo, dw::mul(wid, (float)(2 * tid + 2) / (float)(P + 1)));
    }
    int n0, n1;
    sturm_count2(ds, eb, m, x0, x1, n0, n1);
    const int first = first_above2(n0, n1, r, first_s);
    if (first_round && (first == 0 || first == P)) {
      // the widened fp32 bracket does not hold rank r: start over from the
      // Gershgorin interval
      __syncthreads();
      lo = dw::make(t.gl);
      hi = dw::make(t.gu);
      first_round = false;
      continue;
    }
    first_round = false;
    if (first - 1 == 2 * tid) lohi[0] = x0;
    if (first - 1 == 2 * tid + 1) lohi[0] = x1;
    if (first == 2 * tid) lohi[1] = x0;
    if (first == 2 * tid + 1) lohi[1] = x1;
    __syncthreads();
    if (first > 0) lo = lohi[0];
    if (first < P) hi = lohi[1];
    __syncthreads();
  }
  if (tid == 0) lam[c] = dw::mul(dw::add(lo, hi), 0.5f);
}

// One warp per eigenvalue: eigenvector of Ts from the twisted factorisation
// of Ts - lambda I.  D+ (top-down) and D- (bottom-up) pivots; the twist index
// r minimises |gamma_r| = |D+_r + D-_r - (ds_r - lambda)|; then z_r = 1,
// z_i = -(es_i / D+_i) z_{i+1} above r and z_i = -(es_{i-1} / D-_i) z_{i-1}
// below.  Equal eigenvalues of a split matrix take the blocks in order of
// their smallest |gamma|.
__global__ void __launch_bounds__(32) tri_vec_kernel(const df* __restrict__ d, const df* __restrict__ e, int m,
                                                     int k, const df* __restrict__ lam, df* __restrict__ z_out,
                                                     long long* status) {
  extern __shared__ df smd[];
  df* ds = smd;
  df* es = ds + m;
  df* eb = es + m;
  df* dp = eb + m;
  df* dm = dp + m;
  df* z = dm + m;
  int* ez = reinterpret_cast<int*>(z + m);  // z_i = z[i] * 2^ez[i]
  __shared__ float redf[64];
  const int lane = threadIdx.x;
  const int c = blockIdx.x;
  const TriBounds t = load_tri(d, e, m, ds, es, eb, redf);
  // eigenvalues equal to within the bisection tolerance form a group; every
  // member computes with the group's first value, so all rank the blocks of
  // a split matrix alike and member t takes the t-th
  const float dup_tol = 16.f * kEpsF * kEpsF * fmaxf(fabsf(t.gl), fabsf(t.gu));
  int q0 = c;
  while (q0 > 0 && fabsf(dw::sub(lam[q0 - 1], lam[c]).h) <= dup_tol) --q0;
  const df ls = lam[q0];
  const int dup = c - q0;
  const float tiny = 0x1p-90f;
  if (lane == 0) {
    df x = dw::sub(ds[0], ls);
    if (fabsf(x.h) < tiny) x = dw::make(-tiny);
    dp[0] = x;
#pragma unroll 4
    for (int i = 1; i < m; ++i) {
      x = dw::sub(dw::sub(ds[i], ls), dw::div(eb[i], x));
      if (fabsf(x.h) < tiny) x = dw::make(-tiny);
      dp[i] = x;
    }
  } else if (lane == 1) {
    df x = dw::sub(ds[m - 1], ls);
    if (fabsf(x.h) < tiny) x = dw::make(-tiny);
    dm[m - 1] = x;
#pragma unroll 4
    for (int i = m - 2; i >= 0; --i) {
      x = dw::sub(dw::sub(ds[i], ls), dw::div(eb[i + 1], x));
      if (fabsf(x.h) < tiny) x = dw::make(-tiny);
      dm[i] = x;
    }
  }
  __syncwarp();
  auto gamma_abs = [&](int i) -> float {
    return fabsf(dw::sub(dw::add(dp[i], dm[i]), dw::sub(ds[i], ls)).h);
  };
  float best = 3e38f;
  int bi = 0x7fffffff;
  for (int i = lane; i < m; i += 32) {
    const float gam = gamma_abs(i);
    if (gam < best) { best = gam; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov < best || (ov == best && oi < bi)) { best = ov; bi = oi; }
  }
  int r = bi;
  if (dup > 0) {
    // blocks of the split matrix ranked by their smallest |gamma|; take the
    // (dup)-th
    int chosen = r;
    if (lane == 0) {
      float prev_v = -1.f;
      int prev_i = -1;
      for (int pick = 0; pick <= dup; ++pick) {
        float bv = 3e38f;
        int bidx = -1;
        int s0 = 0;
        while (s0 < m) {
          int s1 = s0;
          while (s1 < m - 1 && es[s1].h != 0.f) ++s1;
          float mv = 3e38f;
          int mi = s0;
          for (int i = s0; i <= s1; ++i) {
            const float gam = gamma_abs(i);
            if (gam < mv) { mv = gam; mi = i; }
          }
          const bool after_prev = mv > prev_v || (mv == prev_v && mi > prev_i);
          if (after_prev && (mv < bv || (mv == bv && mi < bidx))) { bv = mv; bidx = mi; }
          s0 = s1 + 1;
        }
        if (bidx < 0) break;
        chosen = bidx;
        prev_v = bv;
        prev_i = bidx;
      }
    }
    r = __shfl_sync(0xffffffffu, chosen, 0);
  }
  if (r < 0 || r >= m) {  // no finite |gamma|: report, fall back to index 0
    if (lane == 0) record_error(status, kErrNotConverged);
    r = 0;
  }
  // ratios (in place), then the two product chains; a pivot at the floor
  // gives a ratio near 2^90, so each chain keeps its running value in
  // [2^-40, 2^40] and carries the power of two separately
  for (int i = lane; i < m; i += 32) {
    if (i < r) dp[i] = dw::neg(dw::div(es[i], dp[i]));
    else if (i > r) dm[i] = dw::neg(dw::div(es[i - 1], dm[i]));
  }
  __syncwarp();
  auto chain_step = [&](df ratio, df& x, int& ex) {
    x = dw::mul(ratio, x);
    const int be = ((__float_as_int(x.h) >> 23) & 0xff) - 127;
    if (x.h == 0.f) {
      ex = -100000;
    } else if (be > 40 || be < -40) {
      x = dw::mul(x, __int_as_float((127 - be) << 23));
      ex += be;
    }
  };
  if (lane == 0) {
    z[r] = dw::make(1.f);
    ez[r] = 0;
    df x = dw::make(1.f);
    int ex = 0;
#pragma unroll 4
    for (int i = r - 1; i >= 0; --i) {
      if (ex > -100000) chain_step(dp[i], x, ex);
      z[i] = ex > -100000 ? x : dw::make(0.f);
      ez[i] = ex;
    }
  } else if (lane == 1) {
    df x = dw::make(1.f);
    int ex = 0;
#pragma unroll 4
    for (int i = r + 1; i < m; ++i) {
      if (ex > -100000) chain_step(dm[i], x, ex);
      z[i] = ex > -100000 ? x : dw::make(0.f);
      ez[i] = ex;
    }
  }
  __syncwarp();
  // common scale: the largest power of two carried, entries far below it vanish
  int emax = -1000000;
  for (int i = lane; i < m; i += 32)
    if (z[i].h != 0.f) emax = max(emax, ez[i] + (((__float_as_int(z[i].h) >> 23) & 0xff) - 127));
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  df nrm = dw::make(0.f);
  for (int i = lane; i < m; i += 32) {
    const int sh = ez[i] - emax;
    const df zi = (z[i].h == 0.f || sh < -120) ? dw::make(0.f) : dw::ldexp(z[i], sh);
    z[i] = zi;
    nrm = dw::add(nrm, dw::mul(zi, zi));
  }
  nrm = dw::warp_sum(nrm);
  if (!(nrm.h >= 1e-6f && nrm.h < 1e6f)) {  // the largest entry is in [1, 2): nrm >= 1
    if (lane == 0) record_error(status, kErrNotConverged);
    for (int i = lane; i < m; i += 32) z_out[(size_t)i * k + c] = dw::make(i == r ? 1.f : 0.f);
    return;
  }
  const df inv = dw::rcp(dw::sqrt(nrm));
  for (int i = lane; i < m; i += 32) z_out[(size_t)i * k + c] = dw::mul(z[i], inv);
}

// ---------------------------------------------------------------------------
// Back-transformation V = Q Z, Q = H_0 H_1 ... H_{m-3}, in blocks of 32
// reflectors B_b = I - Y_b T_b Y_b^T (T_b upper triangular) applied from the
// last block to the first.  wy_gram_kernel forms slices of Y_b^T Y_b,
// wy_t_kernel the factors T_b, and wy_apply_kernel applies all blocks to one
// column of Z per CTA (the columns are independent, so no grid-wide step).

constexpr int kWyThreads = 256;

// gpart[b][part] = (Y_b^T Y_b restricted to a slice of rows), upper triangle.
__global__ void __launch_bounds__(kWyThreads) wy_gram_kernel(const df* __restrict__ u, int m, int nrefl, int S,
                                                             df* __restrict__ gpart) {
  __shared__ df ys[32 * kWY];
  const int b = blockIdx.x, part = blockIdx.y, tid = threadIdx.x;
  const int j0 = b * kWY, nr = min(kWY, nrefl - j0);
  const int rbeg = j0 + 1, rows = m - rbeg;
  const int per = (rows + S - 1) / S;
  const int i0 = rbeg + part * per, i1 = min(m, i0 + per);
  constexpr int np = kWY * (kWY + 1) / 2;
  constexpr int kPer = (np + kWyThreads - 1) / kWyThreads;
  int pp[kPer], qq[kPer];
  df acc[kPer];
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int idx = tid + t * kWyThreads;
    pp[t] = -1;
    qq[t] = -1;
    acc[t] = dw::make(0.f);
    if (idx < np) {
      int pr = 0, rem = idx;
      while (rem >= kWY - pr) { rem -= kWY - pr; ++pr; }
      pp[t] = pr;
      qq[t] = pr + rem;
    }
  }
  for (int base = i0; base < i1; base += 32) {
    __syncthreads();
    for (int x = tid; x < 32 * kWY; x += kWyThreads) {
      const int rr = x / kWY, pr = x % kWY, i = base + rr;
      ys[rr * kWY + pr] = (i < i1 && pr < nr) ? u[(size_t)(j0 + pr) * m + i] : dw::make(0.f);
    }
    __syncthreads();
    const int nrr = min(32, i1 - base);
    for (int rr = 0; rr < nrr; ++rr)
#pragma unroll
      for (int t = 0; t < kPer; ++t)
        if (pp[t] >= 0) acc[t] = dw::add(acc[t], dw::mul(ys[rr * kWY + pp[t]], ys[rr * kWY + qq[t]]));
  }
  df* gp = gpart + ((size_t)b * S + part) * kWY * kWY;
#pragma unroll
  for (int t = 0; t < kPer; ++t)
    if (pp[t] >= 0) gp[pp[t] * kWY + qq[t]] = acc[t];
}

// T_b by the forward recurrence T[0:i, i] = -tau_i T[0:i, 0:i] (Y^T y_i),
// T[i, i] = tau_i.  One warp per block.
__global__ void __launch_bounds__(32) wy_t_kernel(const df* __restrict__ gpart, const df* __restrict__ tau,
                                                  int nrefl, int S, df* __restrict__ tblk) {
  __shared__ df gs[kWY * kWY];
  __shared__ df ts[kWY * kWY];
  __shared__ df tmp[kWY];
  const int b = blockIdx.x, lane = threadIdx.x;
  const int j0 = b * kWY, nr = min(kWY, nrefl - j0);
  for (int x = lane; x < kWY * kWY; x += 32) {
    const int pr = x / kWY, q = x % kWY;
    df v = dw::make(0.f);
    if (pr <= q)
      for (int part = 0; part < S; ++part) v = dw::add(v, gpart[((size_t)b * S + part) * kWY * kWY + x]);
    gs[x] = v;
    ts[x] = dw::make(0.f);
  }
  __syncwarp();
  for (int i = 0; i < nr; ++i) {
    const df ti = tau[j0 + i];
    if (lane < i) tmp[lane] = dw::neg(dw::mul(ti, gs[lane * kWY + i]));
    __syncwarp();
    df v = dw::make(0.f);
    if (lane < i)
      for (int q = lane; q < i; ++q) v = dw::add(v, dw::mul(ts[lane * kWY + q], tmp[q]));
    __syncwarp();
    if (lane < i) ts[lane * kWY + i] = v;
    if (lane == 0) ts[i * kWY + i] = ti;
    __syncwarp();
  }
  for (int x = lane; x < kWY * kWY; x += 32) tblk[(size_t)b * kWY * kWY + x] = ts[x];
}

// Two columns of Z per CTA: z <- B_b z for b = nbk-1 .. 0, with
// B_b z = z - Y_b (T_b (Y_b^T z)); writes V[:, c] in fp64.  Each thread
// carries four independent double-word accumulations (two reflectors or
// two rows, times two columns) to hide their dependent latency.
constexpr int kApThreads = 512;
__global__ void __launch_bounds__(kApThreads, 1) wy_apply_kernel(const df* __restrict__ u, const df* __restrict__ tblk,
                                                              int m, int nrefl, int k, const df* __restrict__ z,
                                                              double* __restrict__ v) {
  extern __shared__ df smd[];
  df* zc = smd;            // [m] this CTA's column
  df* ts = zc + m;         // [32 x 32]
  df* wv = ts + kWY * kWY; // [32]
  df* tv = wv + kWY;       // [32]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kApThreads / 32;
  const int c = blockIdx.x;
  for (int i = tid; i < m; i += kApThreads) zc[i] = z[(size_t)i * k + c];
  __syncthreads();  // every warp reads rows other warps loaded
  const int nbk = (nrefl + kWY - 1) / kWY;
  for (int b = nbk - 1; b >= 0; --b) {
    const int j0 = b * kWY, nr = min(kWY, nrefl - j0);
    for (int x = tid; x < kWY * kWY; x += kApThreads) ts[x] = tblk[(size_t)b * kWY * kWY + x];
    // w = Y^T z over rows >= j0 + 1: warp takes reflectors warp and warp + 16,
    // the two sums side by side (dw2)
    {
      const int pa = warp, pb = warp + kWarps;
      const df* ya = u + (size_t)(j0 + pa) * m;
      const df* yb = u + (size_t)(j0 + pb) * m;
      const bool va = pa < nr, vb = pb < nr;
      dw2::df2 acc = dw2::pack(dw::make(0.f), dw::make(0.f));
      // four rows per lane per iteration, their loads issued together
      for (int i = j0 + 1 + lane; i < m; i += 128) {
        df ra[4], rb[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int ii = i + 32 * t;
          const bool in = ii < m;
          ra[t] = (va && in) ? ya[ii] : dw::make(0.f);
          rb[t] = (vb && in) ? yb[ii] : dw::make(0.f);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int ii = i + 32 * t;
          if (ii < m) acc = dw2::add(acc, dw2::mul(dw2::pack(ra[t], rb[t]), dw2::splat(zc[ii])));
        }
      }
      const df a0 = dw::warp_sum(dw::make(acc.h.x, acc.l.x));
      const df b0 = dw::warp_sum(dw::make(acc.h.y, acc.l.y));
      if (lane == 0) {
        if (va) wv[pa] = a0;
        if (vb) wv[pb] = b0;
      }
    }
    __syncthreads();
    // t = T w (upper triangular)
    if (warp == 0) {
      df acc = dw::make(0.f);
      if (lane < nr)
        for (int q = lane; q < nr; ++q) acc = dw::add(acc, dw::mul(ts[lane * kWY + q], wv[q]));
      tv[lane] = acc;
    }
    __syncthreads();
    // z -= Y t: thread takes rows i and i + kApThreads, side by side (dw2)
    for (int i = j0 + 1 + tid; i < m; i += 2 * kApThreads) {
      const int i2 = i + kApThreads;
      const bool v2 = i2 < m;
      dw2::df2 sr = dw2::pack(dw::make(0.f), dw::make(0.f));
      // eight reflectors per iteration, their loads issued together
      for (int p0 = 0; p0 < nr; p0 += 8) {
        df ya[8], yb[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int pr = p0 + t;
          const df* y = u + (size_t)(j0 + pr) * m;
          ya[t] = pr < nr ? y[i] : dw::make(0.f);
          yb[t] = (pr < nr && v2) ? y[i2] : dw::make(0.f);
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int pr = p0 + t;
          if (pr < nr) sr = dw2::add(sr, dw2::mul(dw2::pack(ya[t], yb[t]), dw2::splat(tv[pr])));
        }
      }
      zc[i] = dw::sub(zc[i], dw::make(sr.h.x, sr.l.x));
      if (v2) zc[i2] = dw::sub(zc[i2], dw::make(sr.h.y, sr.l.y));
    }
    __syncthreads();
  }
  for (int i = tid; i < m; i += kApThreads) v[(size_t)i * k + c] = dw::to_double(zc[i]);
}

// Z (double-word) to fp64, for m <= 2 (no reflectors).
__global__ void df_to_double_kernel(const df* __restrict__ z, int n, double* __restrict__ v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = dw::to_double(z[i]);
}

// lam = 2^ex * lam_s in fp64.
__global__ void lam_out_kernel(const df* __restrict__ lam_s, const int* __restrict__ ex, int k,
                               double* __restrict__ lam) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < k) lam[c] = ldexp(dw::to_double(lam_s[c]), *ex);
}

// Cholesky QR: W = Z^T Z, W = R^T R, Z <- Z R^-1.

__global__ void ztz_kernel(const double* __restrict__ z, int m, int k, double* __restrict__ w) {
  const int p = blockIdx.y, q = blockIdx.x;
  if (q < p) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s = fma(z[(size_t)i * k + p], z[(size_t)i * k + q], s);
  __shared__ double red[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int x = 0; x < (int)(blockDim.x >> 5); ++x) t += red[x];
    w[p * k + q] = t;
    w[q * k + p] = t;
  }
}

// One block: R (upper) with W = R^T R, then Rinv.  A pivot that has lost all
// but drop_tol of its column's squared norm (a linearly dependent vector):
// strict -- reported as FKK_ERR_NOT_CONVERGED (pivot 1); otherwise the
// column is dropped (its column and row of Rinv are 0).  The pivots are kept
// as reciprocals (no division in the loops), and each entry of Rinv, formed
// a row at a time from the bottom, has its dot product split over 8 threads.
constexpr int kCholSplit = 8;
__global__ void __launch_bounds__(256) chol_inv_kernel(const double* __restrict__ w, int k, double* __restrict__ rinv,
                                                       long long* status, double drop_tol, int strict) {
  extern __shared__ double sm[];
  double* r = sm;              // [k][k]
  double* ri = r + k * k;      // [k][k]
  double* dinv = ri + k * k;   // [k]: 1 / R[j][j], 0 for a dropped column
  for (int x = threadIdx.x; x < k * k; x += blockDim.x) {
    r[x] = w[x];
    ri[x] = 0.0;
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      const double dj = r[j * k + j];
      double inv;
      if (dj > drop_tol * w[j * k + j] && dj < 1e300) {
        inv = rsqrt(dj);
      } else if (strict) {
        record_error(status, kErrNotConverged);
        inv = 1.0;
      } else {
        inv = 0.0;  // drop: the row of R below is zeroed, and so is its Rinv
      }
      dinv[j] = inv;
    }
    __syncthreads();
    const double inv = dinv[j];
    for (int q = j + 1 + threadIdx.x; q < k; q += blockDim.x) r[j * k + q] *= inv;
    __syncthreads();
    // trailing update, a (16 x 16)-thread grid over (q1, q2), q2 >= q1
    for (int q1 = j + 1 + (threadIdx.x >> 4); q1 < k; q1 += 16) {
      const double a = r[j * k + q1];
      for (int q2 = q1 + (threadIdx.x & 15); q2 < k; q2 += 16) r[q1 * k + q2] -= a * r[j * k + q2];
    }
    __syncthreads();
  }
  // Rinv[p][c] = dinv[p] (delta_pc - sum_{p < q <= c} R[p][q] Rinv[q][c]),
  // R[p][q] (q > p) = R scaled row p -- rows from the bottom up
  const int lane8 = threadIdx.x % kCholSplit, grp = threadIdx.x / kCholSplit;
  const int ngrp = blockDim.x / kCholSplit;
  for (int p = k - 1; p >= 0; --p) {
    for (int c0 = p; c0 < k; c0 += ngrp) {
      const int c = c0 + grp;
      double sacc = 0.0;
      if (c < k)
        for (int q = p + 1 + lane8; q <= c; q += kCholSplit) sacc = fma(r[p * k + q], ri[q * k + c], sacc);
#pragma unroll
      for (int o = kCholSplit / 2; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o, kCholSplit);
      if (c < k && lane8 == 0) ri[p * k + c] = dinv[p] * ((p == c ? 1.0 : 0.0) - sacc);
    }
    __syncthreads();
  }
  for (int x = threadIdx.x; x < k * k; x += blockDim.x) rinv[x] = ri[x];
}

// V = Z Rinv (row by row; one warp per row).
__global__ void apply_rinv_kernel(const double* __restrict__ z, int m, int k, const double* __restrict__ rinv,
                                  double* __restrict__ v) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  const double* zr = z + (size_t)row * k;
  for (int c = lane; c < k; c += 32) {
    double s = 0.0;
    for (int p = 0; p <= c; ++p) s = fma(zr[p], rinv[p * k + c], s);
    v[(size_t)row * k + c] = s;
  }
}

// Sign convention: the largest-magnitude component of each column positive
// (ties to the lowest row).  One block per column.
__global__ void sign_fix_kernel(double* __restrict__ v, int m, int k, long long* status) {
  __shared__ double bvs[32];
  __shared__ int bis[32];
  const int c = blockIdx.x;
  double bv = -1.0;
  int bi = 0x7fffffff;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double x = fabs(v[(size_t)j * k + c]);
    if (x > bv || (x == bv && j < bi)) { bv = x; bi = j; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
  }
  if ((threadIdx.x & 31) == 0) { bvs[threadIdx.x >> 5] = bv; bis[threadIdx.x >> 5] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int x = 1; x < (int)(blockDim.x >> 5); ++x)
      if (bvs[x] > bvs[0] || (bvs[x] == bvs[0] && bis[x] < bis[0])) { bvs[0] = bvs[x]; bis[0] = bis[x]; }
  }
  __syncthreads();
  if (bis[0] < 0 || bis[0] >= m) {  // no finite entry in the column
    if (threadIdx.x == 0) record_error(status, kErrNotConverged);
    return;
  }
  const double sgn = v[(size_t)bis[0] * k + c] < 0.0 ? -1.0 : 1.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) v[(size_t)j * k + c] *= sgn;
}

}  // namespace

fkk_status launch_eig_topk(fkk_ctx* ctx, const double* g, int m, int k, double* lam, double* v,
                           cudaStream_t st) {
  fkk_status s;
  const int nsm = ctx->sm_count;
  // 1. tridiagonal reduction
  int nb = std::min(nsm, m);
  if (nb < 1) nb = 1;
  const int ncol_max = (m + nb - 1) / nb;
  const int thr = (m <= kMaxPer * kTrThreadsSmall && ncol_max <= kTrThreadsSmall / 32) ? kTrThreadsSmall
                                                                                      : kTrThreadsLarge;
  if (ncol_max > thr / 32 || m > kMaxPer * thr)
    return fail(ctx, FKK_ERR_INVALID_ARG, "eigensolve: m = %d too large", m);
  const size_t vec_bytes = (size_t)(3 * m + 64 + 8) * sizeof(df);
  const size_t smem_cols = (size_t)ncol_max * m * sizeof(df) + vec_bytes;
  const bool in_smem = smem_cols <= 200 * 1024;
  const size_t smem_tr = in_smem ? smem_cols : vec_bytes;
  df* wsd = (df*)workspace(ctx, "tri_vecs", (size_t)(4 * m + 3 * m + 2 * k + 64) * sizeof(df), &s);
  if (!wsd) return s;
  unsigned long long* pbuf = reinterpret_cast<unsigned long long*>(wsd);
  unsigned long long* cbuf = pbuf + 2 * m;
  df* dd = wsd + 4 * m;
  df* ee = dd + m;
  df* tau = ee + m;
  df* lam_s = tau + m;
  unsigned* scr = (unsigned*)workspace(ctx, "tri_bar", 256, &s);
  if (!scr) return s;
  df* u = (df*)workspace(ctx, "tri_u", (size_t)m * m * sizeof(df), &s);
  if (!u) return s;
  df* work = nullptr;
  if (!in_smem) {
    work = (df*)workspace(ctx, "tri_work", (size_t)m * m * sizeof(df), &s);
    if (!work) return s;
  }
  FKK_CUDA(ctx, cudaMemsetAsync(scr, 0, 256, st));
  // tagged exchange buffers start cleared (tag 0 is never current), and e
  // at zero (e[m-1] stays 0)
  FKK_CUDA(ctx, cudaMemsetAsync(wsd, 0, (size_t)(4 * m + 2 * m) * sizeof(df), st));
  int* ex_dev = (int*)(scr + 48);
  {
    long long* cycles = nullptr;
    if (ctx->timing >= 2) {
      cycles = (long long*)workspace(ctx, "eig_phase_cycles", 8 * sizeof(long long), &s);
      if (!cycles) return s;
    }
    // the test knob of fkk_test_stall_next_eigensolve: one eigensolve whose
    // first exchange waits for a tag nobody publishes, with a short bound
    const int stall = ctx->stall_next_eig;
    ctx->stall_next_eig = 0;
    TridArgs ta{g,     m,         ncol_max,      work,          pbuf,   cbuf,  dd, ee, tau, u, scr + 40, ex_dev,
                cycles, scr,      (int*)(scr + 16), ctx->d_status, stall ? (1u << 14) : (1u << 20), stall};
    void* args[] = {&ta};
    const bool small = thr == kTrThreadsSmall;
    const void* fn = in_smem ? (small ? (const void*)tridiag_kernel<true, kTrThreadsSmall>
                                      : (const void*)tridiag_kernel<true, kTrThreadsLarge>)
                             : (small ? (const void*)tridiag_kernel<false, kTrThreadsSmall>
                                      : (const void*)tridiag_kernel<false, kTrThreadsLarge>);
    FKK_CUDA(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_tr));
    int per_sm = 0;
    FKK_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, thr, smem_tr));
    if (per_sm < 1) return fail(ctx, FKK_ERR_INVALID_ARG, "eigensolve: reduction kernel cannot be resident");
    FKK_COUNT_LAUNCH();
    FKK_CUDA(ctx, cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(thr), args, smem_tr, st));
  }
  // 4a. the WY block factors of the reflectors depend on nothing else, so
  // they run on the context's side stream beside steps 2-3
  const int nrefl = std::max(0, m - 2);
  df* tblk = nullptr;
  if (nrefl > 0) {
    const int nbk = (nrefl + kWY - 1) / kWY;
    const int S = std::max(1, std::min(8, nsm / nbk));
    df* gpart = (df*)workspace(ctx, "tri_gpart", (size_t)nbk * S * kWY * kWY * sizeof(df), &s);
    if (!gpart) return s;
    tblk = (df*)workspace(ctx, "tri_tblk", (size_t)nbk * kWY * kWY * sizeof(df), &s);
    if (!tblk) return s;
    cudaStream_t aux = nullptr;
    FKK_TRY(side_stream(ctx, &aux));
    FKK_CUDA(ctx, cudaEventRecord(ctx->ev_fork, st));
    FKK_CUDA(ctx, cudaStreamWaitEvent(aux, ctx->ev_fork, 0));
    FKK_COUNT_LAUNCH();
    wy_gram_kernel<<<dim3(nbk, S), kWyThreads, 0, aux>>>(u, m, nrefl, S, gpart);
    FKK_COUNT_LAUNCH();
    wy_t_kernel<<<nbk, 32, 0, aux>>>(gpart, tau, nrefl, S, tblk);
    FKK_CUDA(ctx, cudaEventRecord(ctx->ev_join, aux));
  }
  // 2-3. eigenvalues and tridiagonal eigenvectors
  df* z = (df*)workspace(ctx, "tri_z", (size_t)m * k * sizeof(df), &s);
  if (!z) return s;
  double* vz = (double*)workspace(ctx, "tri_vz", (size_t)m * k * sizeof(double), &s);
  if (!vz) return s;
  {
    const size_t sb = (size_t)3 * m * sizeof(df);
    FKK_CUDA(ctx, cudaFuncSetAttribute(tri_bisect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
    FKK_COUNT_LAUNCH();
    tri_bisect_kernel<<<k, kBisWarps * 32, sb, st>>>(dd, ee, m, lam_s);
    const size_t sv = (size_t)6 * m * sizeof(df) + (size_t)m * sizeof(int);
    FKK_CUDA(ctx, cudaFuncSetAttribute(tri_vec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sv));
    FKK_COUNT_LAUNCH();
    tri_vec_kernel<<<k, 32, sv, st>>>(dd, ee, m, k, lam_s, z, ctx->d_status);
    FKK_COUNT_LAUNCH();
    lam_out_kernel<<<(k + 127) / 128, 128, 0, st>>>(lam_s, ex_dev, k, lam);
    FKK_CUDA(ctx, cudaGetLastError());
  }
  // 4b. back-transformation of the eigenvectors
  if (nrefl > 0) {
    FKK_CUDA(ctx, cudaStreamWaitEvent(st, ctx->ev_join, 0));
    const size_t sa = ((size_t)m + kWY * kWY + 2 * kWY) * sizeof(df);
    FKK_CUDA(ctx, cudaFuncSetAttribute(wy_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sa));
    FKK_COUNT_LAUNCH();
    wy_apply_kernel<<<k, kApThreads, sa, st>>>(u, tblk, m, nrefl, k, z, vz);
    FKK_CUDA(ctx, cudaGetLastError());
  } else {
    FKK_COUNT_LAUNCH();
    df_to_double_kernel<<<(m * k + 255) / 256, 256, 0, st>>>(z, m * k, vz);
  }
  // 5. Cholesky QR, sign convention
  double* wk = (double*)workspace(ctx, "tri_wk", (size_t)2 * k * k * sizeof(double), &s);
  if (!wk) return s;
  FKK_COUNT_LAUNCH();
  ztz_kernel<<<dim3(k, k), 128, 0, st>>>(vz, m, k, wk);
  const size_t sc = ((size_t)2 * k * k + k) * sizeof(double);
  FKK_CUDA(ctx, cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc));
  FKK_COUNT_LAUNCH();
  chol_inv_kernel<<<1, 256, sc, st>>>(wk, k, wk + k * k, ctx->d_status, 1e-20, 1);
  FKK_COUNT_LAUNCH();
  apply_rinv_kernel<<<(m + 7) / 8, 256, 0, st>>>(vz, m, k, wk + k * k, v);
  FKK_COUNT_LAUNCH();
  sign_fix_kernel<<<k, 256, 0, st>>>(v, m, k, ctx->d_status);
  return cuda_check(ctx, cudaGetLastError(), "eigensolve");
}

// The fp64 Cholesky-QR pieces above, for other small m x k matrices.
fkk_status launch_ztz(fkk_ctx* ctx, const double* z, int m, int k, double* w, cudaStream_t st) {
  FKK_COUNT_LAUNCH();
  ztz_kernel<<<dim3(k, k), 128, 0, st>>>(z, m, k, w);
  return cuda_check(ctx, cudaGetLastError(), "ztz");
}

fkk_status launch_chol_inv(fkk_ctx* ctx, const double* w, int k, double* rinv, cudaStream_t st, double drop_tol,
                           bool strict) {
  const size_t sc = ((size_t)2 * k * k + k) * sizeof(double);
  if (sc > 227 * 1024) return fail(ctx, FKK_ERR_INVALID_ARG, "Cholesky of %d x %d does not fit shared memory", k, k);
  FKK_CUDA(ctx, cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc));
  FKK_COUNT_LAUNCH();
  chol_inv_kernel<<<1, 256, sc, st>>>(w, k, rinv, ctx->d_status, drop_tol, strict ? 1 : 0);
  return cuda_check(ctx, cudaGetLastError(), "chol_inv");
}

fkk_status launch_apply_rinv(fkk_ctx* ctx, const double* z, int m, int k, const double* rinv, double* v,
                             cudaStream_t st) {
  FKK_COUNT_LAUNCH();
  apply_rinv_kernel<<<(m + 7) / 8, 256, 0, st>>>(z, m, k, rinv, v);
  return cuda_check(ctx, cudaGetLastError(), "apply_rinv");
}

fkk_status launch_sign_fix(fkk_ctx* ctx, double* v, int m, int k, cudaStream_t st) {
  FKK_COUNT_LAUNCH();
  sign_fix_kernel<<<k, 256, 0, st>>>(v, m, k, ctx->d_status);
  return cuda_check(ctx, cudaGetLastError(), "sign_fix");
}

}  // namespace fkk
