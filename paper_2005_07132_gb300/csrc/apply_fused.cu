// ML:fKK-EC apply (Sec. 2.6) in one persistent launch: for new spectra,
//   a    = 1/2 ln(max(I / I_ref, floor)) - o          (Sec. 2.1; o the basis' offset)
//   dP   = a (f W),  W = V diag(s^2 / (s^2 + lambda))  (Eq. ML_Unew: U_new S = dP + o (f W))
//   Im K = exp((U_new S) C_amp) sin((U_new S) C_ph)    (Eq. fKKEC; Re K with cos)
// I is read from HBM once and Im written once; P never leaves the SM.  The
// offset o (the training mean of the log ratios) shrinks the values that are
// rounded to bf16; its contribution (o f W) C is added back exactly through
// two extra K columns of the reconstruction (P column k = 1 against the bf16
// hi part of the bias, and a column that carries its lo part).
//
// One CTA per SM, 16 warps, each 128-spectrum row tile flowing through a
// warp-specialised pipeline:
//   warp 0   TMA producer of 64-channel chunks of I (two 32-channel fp32
//            boxes, 128-byte swizzle), of f W (bf16 hi / lo, K-major) and
//            of the chunk's channel constants (1 / I_ref, offset), through a
//            3-4 stage ring;
//   warp 1   issues the projection MMAs into one of two TMEM accumulators;
//   warp 2   TMA producer of 64-column tiles of the interleaved coefficients;
//   warp 3   issues the reconstruction MMAs into four TMEM accumulators;
//   warps 4-11 (one spectrum and one 32-channel box per thread) turn each
//            fp32 chunk into the bf16 A operand in place, then move the
//            finished projection from TMEM into the reconstruction's A
//            operand in shared memory;
//   warps 12-15 evaluate exp / sin (/ cos) of each accumulator for 32
//            channels into a 128-byte-swizzled staging tile that TMA stores
//            to Im (and Re), clipping rows and channels outside the arrays.
// The projection of one tile overlaps the reconstruction of the previous.
// Products: FKK_PREC_BF16X3 -- hi.hi + hi.lo + lo.hi in both GEMMs;
// FKK_PREC_BF16 -- hi.hi in the projection, hi.hi + lo.hi in the
// reconstruction.  Every mbarrier wait is bounded: on expiry the CTA records
// FKK_ERR_TIMEOUT, its roles stop issuing and the kernel drains and returns.
#include <cmath>

#include "basis_internal.h"
#include "common.cuh"
#include "fit.h"
#include "tc.cuh"

namespace fkk {
namespace {

constexpr int kTM = 128;      // spectra per row tile (TMEM lanes)
constexpr int kCh = 64;       // channels per projection chunk
constexpr int kNT = 64;       // interleaved output columns per reconstruction tile (32 channels)
constexpr int kKp = 64;       // K per 128-byte atom of the P and coefficient operands (one or two atoms)
constexpr int kThreads = 512;  // warps 0-3 control, 4-11 transform, 12-15 epilogue
constexpr int kTW = 8;         // transform warps
constexpr uint32_t kConstBytes = 2 * 64 * 4;  // per chunk: 1 / I_ref, offset (64 channels each)
constexpr int kD2 = 4;        // reconstruction accumulators
constexpr uint32_t kIBytes = kTM * kCh * 4;   // one fp32 I chunk (two boxes)
constexpr uint32_t kStg = 32 * 32 * 4;        // one 32 x 32 fp32 staging tile
constexpr uint32_t kPopAtom = kTM * kKp * 2;  // P operand, one K atom of one plane
constexpr uint32_t kCAtom = kNT * kKp * 2;    // coefficient tile, one K atom of one plane
constexpr uint32_t kTmemCols = 512;           // D1 at d * 64 katoms; D2 at 128 katoms + 64 b
constexpr int kMaxStages = 4;

struct FusedArgs {
  int64_t n;
  int m;
  int k;
  int kp1;       // N of the projection GEMM, K extent of the reconstruction: ceil16(k + 2) <= 128
  int katoms;    // 64-wide K atoms of the P and coefficient operands: ceil(kp1 / 64)
  int rows_c;    // rows of one K atom of the packed coefficients
  int n_chunks;  // ceil(m / 64)
  int n_ct;      // ceil(2m / 64)
  int n_tiles;   // ceil(n / 128)
  int x3;        // 1: FKK_PREC_BF16X3, 0: FKK_PREC_BF16
  int stages;
  float floor_;
  const float* consts;   // [n_chunks][2][64] floats: 1 / I_ref and the offset o, 0 beyond m
  long long* status;
  uint32_t stage_bytes;
  uint32_t w_bytes;  // one W plane of a stage: kp1 rows x 128 B
};

// 16-byte chunk q of row r of a 128-byte-swizzled tile
__device__ __forceinline__ uint32_t sw128(int r, int q) { return (uint32_t)(r * 128 + ((q ^ (r & 7)) << 4)); }

__device__ __forceinline__ uint32_t bf2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// bf16 hi (and lo = bf16(v - hi)) of 8 consecutive floats
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
    const float2 hf = __bfloat1622float2(hb);
    h[e] = *reinterpret_cast<const uint32_t*>(&hb);
    l[e] = bf2(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Named barrier 1 over the 256 transform threads that ORs a flag across them.
__device__ __forceinline__ bool bar_t_any(bool flag) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, 1, 256, q;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)flag)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// bounded wait by every lane of a warp, made warp-uniform
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity) {
  const bool ok = tc::mbar_wait(bar, parity);
  return __all_sync(0xffffffffu, ok);
}

template <bool kRe>
__global__ void __launch_bounds__(kThreads, 1)
    apply_fused_kernel(const __grid_constant__ CUtensorMap tm_i, const __grid_constant__ CUtensorMap tm_whi,
                       const __grid_constant__ CUtensorMap tm_wlo, const __grid_constant__ CUtensorMap tm_chi,
                       const __grid_constant__ CUtensorMap tm_clo, const __grid_constant__ CUtensorMap tm_im,
                       const __grid_constant__ CUtensorMap tm_re, FusedArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const bool x3 = p.x3 != 0;
  const int S = p.stages;
  // layout: ring [S] | P operand (hi, lo; katoms K atoms each) | coefficient ring [2] (hi[, lo]; katoms
  // atoms each) | staging [4 warps] | barriers
  const int na = p.katoms;
  const uint32_t pop_plane = na * kPopAtom, c_plane = na * kCAtom;
  const uint32_t d1s = 64 * na;  // TMEM columns per projection accumulator
  uint8_t* ring = smem;
  uint8_t* pop = ring + S * p.stage_bytes;
  const uint32_t c_stage = (x3 ? 2 : 1) * c_plane;
  uint8_t* cring = pop + 2 * pop_plane;
  uint8_t* stg = cring + 2 * c_stage;
  const uint32_t stg_warp = kRe ? 2 * kStg : kStg;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg + 4 * stg_warp);
  uint64_t* full = bars;                   // [kMaxStages] ring stage landed (TMA bytes)
  uint64_t* aready = full + kMaxStages;    // [kMaxStages] A operand written (8 transform warps)
  uint64_t* empty = aready + kMaxStages;   // [kMaxStages] ring stage consumed (projection MMAs)
  uint64_t* d1full = empty + kMaxStages;   // [2] projection accumulator complete
  uint64_t* d1empty = d1full + 2;          // [2] projection accumulator read (8 transform warps)
  uint64_t* popfull = d1empty + 2;         // P operand written (8 transform warps)
  uint64_t* popempty = popfull + 1;        // P operand consumed (reconstruction MMAs)
  uint64_t* cfull = popempty + 1;          // [2] coefficient tile landed
  uint64_t* cempty = cfull + 2;            // [2] coefficient tile consumed
  uint64_t* d2full = cempty + 2;           // [kD2] reconstruction accumulator complete
  uint64_t* d2empty = d2full + kD2;        // [kD2] reconstruction accumulator read (4 epilogue warps)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(d2empty + kD2);
  __shared__ volatile int fail_s;  // set by any role whose bounded wait ran out

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    fail_s = 0;
    for (int s = 0; s < kMaxStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&aready[s], kTW);
      tc::mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&d1full[s], 1);
      tc::mbar_init(&d1empty[s], kTW);
      tc::mbar_init(&cfull[s], 1);
      tc::mbar_init(&cempty[s], 1);
    }
    tc::mbar_init(popfull, kTW);
    tc::mbar_init(popempty, 1);
    for (int s = 0; s < kD2; ++s) {
      tc::mbar_init(&d2full[s], 1);
      tc::mbar_init(&d2empty[s], 4);
    }
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tm_i);
    tc::prefetch_tmap(&tm_whi);
    tc::prefetch_tmap(&tm_chi);
    tc::prefetch_tmap(&tm_im);
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = *tmem_slot;
  const int ksteps = p.kp1 / 16;
  long long clamped = 0;

  if (warp == 0) {
    // ------------------------------------------------ I / W producer
    if (lane == 0) {
      const uint32_t wpl = (x3 ? 2 : 1) * p.w_bytes;
      const uint32_t tx = kIBytes + wpl + kConstBytes;
      uint32_t it = 0;
      for (int tile = blockIdx.x; tile < p.n_tiles && !fail_s; tile += gridDim.x) {
        const int row0 = tile * kTM;
        for (int c = 0; c < p.n_chunks; ++c, ++it) {
          const int s = it % S;
          if (!tc::mbar_wait(&empty[s], ((it / S) & 1) ^ 1)) { fail_s = 1; break; }
          uint8_t* st = ring + s * p.stage_bytes;
          tc::mbar_arrive_expect_tx(&full[s], tx);
          tc::tma_load_2d(st, &tm_i, &full[s], c * kCh, row0);
          tc::tma_load_2d(st + kIBytes / 2, &tm_i, &full[s], c * kCh + 32, row0);
          tc::tma_load_2d(st + kIBytes, &tm_whi, &full[s], c * kCh, 0);
          if (x3) tc::tma_load_2d(st + kIBytes + p.w_bytes, &tm_wlo, &full[s], c * kCh, 0);
          tc::bulk_load(st + kIBytes + wpl, p.consts + (size_t)c * 128, kConstBytes, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ projection MMAs
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(kTM, p.kp1);
      uint32_t it = 0, lt = 0;
      for (int tile = blockIdx.x; tile < p.n_tiles && !fail_s; tile += gridDim.x, ++lt) {
        const int d = lt & 1;
        if (!tc::mbar_wait(&d1empty[d], ((lt >> 1) & 1) ^ 1)) { fail_s = 1; break; }
        tc::tc_fence_after();
        const uint32_t dacc = tbase + d * d1s;
        bool ok = true;
        for (int c = 0; c < p.n_chunks; ++c, ++it) {
          const int s = it % S;
          if (!tc::mbar_wait(&aready[s], (it / S) & 1)) { ok = false; break; }
          tc::tc_fence_after();
          const uint32_t a_hi = tc::smem_u32(ring + s * p.stage_bytes);
          const uint32_t a_lo = a_hi + kIBytes / 2;
          const uint32_t w_hi = a_hi + kIBytes, w_lo = w_hi + p.w_bytes;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t o = ks * 32;
            tc::mma_bf16(dacc, tc::sdesc_kmajor_sw128(a_hi + o), tc::sdesc_kmajor_sw128(w_hi + o), idesc,
                         (c > 0 || ks > 0) ? 1u : 0u);
            if (x3) {
              tc::mma_bf16(dacc, tc::sdesc_kmajor_sw128(a_hi + o), tc::sdesc_kmajor_sw128(w_lo + o), idesc, 1u);
              tc::mma_bf16(dacc, tc::sdesc_kmajor_sw128(a_lo + o), tc::sdesc_kmajor_sw128(w_hi + o), idesc, 1u);
            }
          }
          tc::mma_commit(&empty[s]);
        }
        if (!ok) { fail_s = 1; break; }
        tc::mma_commit(&d1full[d]);
      }
    }
  } else if (warp == 2) {
    // ------------------------------------------------ coefficient producer
    if (lane == 0) {
      uint32_t it = 0;
      for (int tile = blockIdx.x; tile < p.n_tiles && !fail_s; tile += gridDim.x) {
        for (int ct = 0; ct < p.n_ct; ++ct, ++it) {
          const int s = it & 1;
          if (!tc::mbar_wait(&cempty[s], ((it >> 1) & 1) ^ 1)) { fail_s = 1; break; }
          uint8_t* cs = cring + s * c_stage;
          tc::mbar_arrive_expect_tx(&cfull[s], c_stage);
          for (int at = 0; at < na; ++at) {
            tc::tma_load_2d(cs + at * kCAtom, &tm_chi, &cfull[s], 0, at * p.rows_c + ct * kNT);
            if (x3) tc::tma_load_2d(cs + c_plane + at * kCAtom, &tm_clo, &cfull[s], 0, at * p.rows_c + ct * kNT);
          }
        }
      }
    }
  } else if (warp == 3) {
    // ------------------------------------------------ reconstruction MMAs
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(kTM, kNT);
      const uint32_t p_hi = tc::smem_u32(pop), p_lo = p_hi + pop_plane;
      uint32_t it = 0, lt = 0;
      for (int tile = blockIdx.x; tile < p.n_tiles && !fail_s; tile += gridDim.x, ++lt) {
        if (!tc::mbar_wait(popfull, lt & 1)) { fail_s = 1; break; }
        tc::tc_fence_after();
        bool ok = true;
        for (int ct = 0; ct < p.n_ct; ++ct, ++it) {
          const int s = it & 1;
          const int b = it % kD2;
          if (!tc::mbar_wait(&d2empty[b], ((it / kD2) & 1) ^ 1)) { ok = false; break; }
          if (!tc::mbar_wait(&cfull[s], (it >> 1) & 1)) { ok = false; break; }
          tc::tc_fence_after();
          const uint32_t c_hi = tc::smem_u32(cring + s * c_stage), c_lo = c_hi + c_plane;
          const uint32_t dacc = tbase + 2 * d1s + b * kNT;
          for (int ks = 0; ks < ksteps; ++ks) {
            // K step ks: atom ks / 4, 32-byte column group ks % 4 of its rows
            const uint32_t op = (ks >> 2) * kPopAtom + (ks & 3) * 32, oc = (ks >> 2) * kCAtom + (ks & 3) * 32;
            tc::mma_bf16(dacc, tc::sdesc_kmajor_sw128(p_hi + op), tc::sdesc_kmajor_sw128(c_hi + oc), idesc,
                         ks > 0 ? 1u : 0u);
            if (x3) tc::mma_bf16(dacc, tc::sdesc_kmajor_sw128(p_hi + op), tc::sdesc_kmajor_sw128(c_lo + oc), idesc, 1u);
            tc::mma_bf16(dacc, tc::sdesc_kmajor_sw128(p_lo + op), tc::sdesc_kmajor_sw128(c_hi + oc), idesc, 1u);
          }
          tc::mma_commit(&cempty[s]);
          tc::mma_commit(&d2full[b]);
        }
        if (!ok) { fail_s = 1; break; }
        tc::mma_commit(popempty);
      }
    }
  } else if (warp < 4 + kTW) {
    // ------------------------------------------------ transform + P operand
    const int q4 = warp & 3;
    const int h = (warp - 4) >> 2;  // the 32-channel box of the chunk (and half of the P row)
    const int r = q4 * 32 + lane;
    const uint32_t wpl = (x3 ? 2 : 1) * p.w_bytes;
    uint32_t it = 0, lt = 0;
    int clamped32 = 0;
    bool failed = false;
    for (int tile = blockIdx.x; tile < p.n_tiles && !failed; tile += gridDim.x, ++lt) {
      const bool row_ok = (int64_t)tile * kTM + r < p.n;
      for (int c = 0; c < p.n_chunks; ++c, ++it) {
        const int s = it % S;
        uint8_t* st = ring + s * p.stage_bytes;
        const float* cst = reinterpret_cast<const float*>(st + kIBytes + wpl);
        const int jlim = row_ok ? p.m - c * kCh - 32 * h : 0;  // channels of the box that count
        const bool ok = warp_wait(&full[s], (it / S) & 1);
        float a[32];
        if (ok) {
          const uint8_t* box = st + h * (kIBytes / 2);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 v = *reinterpret_cast<const float4*>(box + sw128(r, q));
            const float4 ir = *reinterpret_cast<const float4*>(cst + 32 * h + 4 * q);
            const float4 of = *reinterpret_cast<const float4*>(cst + 64 + 32 * h + 4 * q);
            const float xv[4] = {v.x * ir.x, v.y * ir.y, v.z * ir.z, v.w * ir.w};
            const float ov[4] = {of.x, of.y, of.z, of.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              clamped32 += (!(xv[e] >= p.floor_) && 4 * q + e < jlim) ? 1 : 0;
              // (ln 2 / 2) log2(max(x, floor)) - o; fmaxf takes the floor for NaN
              a[4 * q + e] = fmaf(0.34657359027997264f, __log2f(fmaxf(xv[e], p.floor_)), -ov[e]);
            }
          }
        }
        // every transform thread has read the fp32 chunk: overwrite it with A
        failed = bar_t_any(!ok);
        if (!failed) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint4 hi, lo;
            split8(a + 8 * q, hi, lo);
            *reinterpret_cast<uint4*>(st + sw128(r, 4 * h + q)) = hi;
            if (x3) *reinterpret_cast<uint4*>(st + kIBytes / 2 + sw128(r, 4 * h + q)) = lo;
          }
          tc::fence_proxy_async();
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&aready[s]);
        if (failed) break;
      }
      if (failed) break;
      // the finished projection -> the reconstruction's A operand (this
      // warp: columns 32 h .. 32 h + 31 of the row)
      const int d = lt & 1;
      bool ok = warp_wait(&d1full[d], (lt >> 1) & 1);
      ok = ok && warp_wait(popempty, (lt & 1) ^ 1);
      failed = bar_t_any(!ok);
      if (failed) break;
      tc::tc_fence_after();
      for (int at = 0; at < na; ++at) {
        // columns 64 at + 32 h .. + 31 of the row, into K atom `at`
        const uint32_t taddr = tbase + ((uint32_t)(q4 * 32) << 16) + d * d1s + 64 * at + 32 * h;
        float pv[32];
#pragma unroll
        for (int c16 = 0; c16 < 2; ++c16) {
          if (4 * at + 2 * h + c16 < ksteps) {
            tc::tmem_ld16(taddr + c16 * 16, pv + c16 * 16);
          } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) pv[c16 * 16 + e] = 0.f;
          }
        }
        uint8_t* pa = pop + at * kPopAtom;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint4 hi, lo;
          split8(pv + 8 * q, hi, lo);
          // columns k, k+1 carry the offset's contribution: P_hi[k] = 1 and
          // (reduced form) P_lo[k+1] = 1, the rest 0
          uint32_t hw[4] = {hi.x, hi.y, hi.z, hi.w}, lw[4] = {lo.x, lo.y, lo.z, lo.w};
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int col = 64 * at + 32 * h + 8 * q + e;
            const uint32_t sh = (e & 1) * 16;
            if (col >= p.k) {
              const uint32_t one = 0x3F80u;  // bf16 1.0
              const uint32_t hv = col == p.k ? one : 0u;
              const uint32_t lv = (!x3 && col == p.k + 1) ? one : 0u;
              hw[e >> 1] = (hw[e >> 1] & ~(0xFFFFu << sh)) | (hv << sh);
              lw[e >> 1] = (lw[e >> 1] & ~(0xFFFFu << sh)) | (lv << sh);
            }
          }
          *reinterpret_cast<uint4*>(pa + sw128(r, 4 * h + q)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4*>(pa + pop_plane + sw128(r, 4 * h + q)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
      }
      tc::tc_fence_before();
      tc::fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(&d1empty[d]);
        tc::mbar_arrive(popfull);
      }
    }
    clamped = clamped32;
    if (failed) fail_s = 1;
  } else {
    // ------------------------------------------------ exp / sin epilogue
    const int q4 = warp & 3;
    uint8_t* my_stg = stg + (warp - 4 - kTW) * stg_warp;
    uint32_t it = 0;
    bool failed = false;
    for (int tile = blockIdx.x; tile < p.n_tiles && !failed; tile += gridDim.x) {
      const int y = tile * kTM + q4 * 32;
      for (int ct = 0; ct < p.n_ct; ++ct, ++it) {
        const int b = it % kD2;
        if (!warp_wait(&d2full[b], (it / kD2) & 1)) { failed = true; break; }
        tc::tc_fence_after();
        const uint32_t taddr = tbase + ((uint32_t)(q4 * 32) << 16) + 2 * d1s + b * kNT;
        float v[64];
        tc::tmem_ld32(taddr, v);
        tc::tmem_ld32(taddr + 32, v + 32);
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          tc::mbar_arrive(&d2empty[b]);
          tc::bulk_wait_read0();  // the previous stores have read the staging tile(s)
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          float im4[4], re4[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int t = 4 * q + e;
            const float ex = ex2_approx(v[2 * t]);  // the amplitude column is prescaled by log2(e)
            im4[e] = ex * __sinf(v[2 * t + 1]);
            if (kRe) re4[e] = ex * __cosf(v[2 * t + 1]);
          }
          *reinterpret_cast<float4*>(my_stg + sw128(lane, q)) = make_float4(im4[0], im4[1], im4[2], im4[3]);
          if (kRe) *reinterpret_cast<float4*>(my_stg + kStg + sw128(lane, q)) = make_float4(re4[0], re4[1], re4[2], re4[3]);
        }
        tc::fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
          tc::tma_store_2d(&tm_im, my_stg, ct * 32, y);
          if (kRe) tc::tma_store_2d(&tm_re, my_stg + kStg, ct * 32, y);
          tc::bulk_commit();
        }
      }
    }
    if (lane == 0) tc::bulk_wait0();
    if (failed) fail_s = 1;
  }
  if (warp >= 4 && warp < 4 + kTW) {
    for (int o = 16; o > 0; o >>= 1) clamped += __shfl_xor_sync(0xffffffffu, clamped, o);
    if (lane == 0 && clamped)
      atomicAdd(reinterpret_cast<unsigned long long*>(p.status + 1), (unsigned long long)clamped);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (fail_s && threadIdx.x == 0) record_error(p.status, kErrTimeout);
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc(tbase, kTmemCols);
}

// f W (m x k fp64, row-major) -> bf16 hi / lo [kp1][mp], zero padded
__global__ void pack_w_kernel(const double* __restrict__ w, const double* __restrict__ f, int m, int k, int kp1,
                              int mp, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)kp1 * mp) return;
  const int i = (int)(t / mp), j = (int)(t % mp);
  const float v = (i < k && j < m) ? (float)(f[j] * w[(int64_t)j * k + i]) : 0.f;
  split_bf16(v, hi[t], lo[t]);
}

// pbar = o^T (f W) (k), fp64
__global__ void pbar_kernel(const double* __restrict__ w, const double* __restrict__ f,
                            const double* __restrict__ off, int m, int k, double* __restrict__ pbar) {
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) acc += off[j] * f[j] * w[(int64_t)j * k + i];
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) pbar[i] = red[0];
}

// Interleaved coefficients: row 2j = log2(e) C_amp[:, j], row 2j + 1 =
// C_ph[:, j], as bf16 hi / lo in K atoms of 64 columns, atom-major
// [katoms][rows_c][64]; column k holds the bias b = pbar^T C of the row (hi
// part in the hi plane, its lo part in the lo plane), column k + 1 the lo
// part of the bias in the hi plane.
__global__ void pack_c_kernel(const double* __restrict__ camp, const double* __restrict__ cph,
                              const double* __restrict__ pbar, int k, int m, int rows_c, int katoms,
                              __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)katoms * rows_c * kKp) return;
  const int at = (int)(t / ((int64_t)rows_c * kKp));
  const int64_t u = t - (int64_t)at * rows_c * kKp;
  const int r = (int)(u / kKp), c = at * kKp + (int)(u % kKp);
  const int j = r >> 1;
  const double sc = (r & 1) ? 1.0 : 1.4426950408889634;
  const double* cm = (r & 1) ? cph : camp;
  float v = 0.f;
  __nv_bfloat16 h, l;
  if (j < m && c < k) {
    v = (float)(sc * cm[(int64_t)c * m + j]);
    split_bf16(v, h, l);
  } else if (j < m && (c == k || c == k + 1)) {
    double b = 0.0;
    for (int i = 0; i < k; ++i) b += pbar[i] * cm[(int64_t)i * m + j];
    __nv_bfloat16 bh, bl;
    split_bf16((float)(sc * b), bh, bl);
    h = c == k ? bh : bl;
    l = c == k ? bl : __float2bfloat16_rn(0.f);
  } else {
    h = l = __float2bfloat16_rn(0.f);
  }
  hi[t] = h;
  lo[t] = l;
}

// [mp / 64][2][64]: per 64-channel chunk, 1 / I_ref then the offset (0 beyond m)
__global__ void chan_consts_kernel(const float* __restrict__ i_ref, const double* __restrict__ off, int m, int mp,
                                   float* __restrict__ consts) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= mp) return;
  float* cc = consts + (size_t)(j / 64) * 128 + (j % 64);
  cc[0] = j < m ? 1.0f / i_ref[j] : 0.f;
  cc[64] = j < m ? (float)off[j] : 0.f;
}

// Shared memory of the kernel with the deepest ring (2..4 stages, or `want`)
// that fits; above the 227 KB limit when not even two stages do.
size_t fused_smem(int kp1, bool x3, bool re, int want, int* stages, uint32_t* stage_bytes, uint32_t* w_bytes) {
  const int katoms = (kp1 + kKp - 1) / kKp;
  const uint32_t wb = (uint32_t)kp1 * 128;
  uint32_t st = kIBytes + (x3 ? 2 : 1) * wb + kConstBytes;
  st = (st + 1023) & ~1023u;
  const size_t fixed =
      1024 + 2 * katoms * kPopAtom + 2 * (x3 ? 2 : 1) * katoms * kCAtom + 4 * (re ? 2 : 1) * kStg + 512;
  const size_t cap = 227 * 1024;
  int s = (want >= 2 && want <= kMaxStages) ? want : kMaxStages;
  while (s > 2 && fixed + (size_t)s * st > cap) --s;
  *stages = s;
  *stage_bytes = st;
  *w_bytes = wb;
  return fixed + (size_t)s * st;
}

}  // namespace

fkk_status apply_pack(fkk_ctx* ctx, const fkk_basis* Bc, cudaStream_t st) {
  fkk_basis* B = const_cast<fkk_basis*>(Bc);
  std::lock_guard<std::mutex> lk(B->pack_mu);
  if (B->pack) return FKK_OK;
  const int m = B->m, k = B->k;
  const int kp1 = ((k + 2 + 15) / 16) * 16;
  const int katoms = (kp1 + kKp - 1) / kKp;
  const int mp = ((m + 63) / 64) * 64;
  const int rows_c = ((2 * m + kNT - 1) / kNT) * kNT;
  const size_t wbytes = (size_t)kp1 * mp * 2, cbytes = (size_t)katoms * rows_c * kKp * 2;
  const size_t bytes = 2 * wbytes + 2 * cbytes + 2 * (size_t)mp * 4 + (size_t)k * 8 + 2048;
  void* mem = nullptr;
  FKK_CUDA(ctx, cudaMalloc(&mem, bytes));
  uint8_t* q = static_cast<uint8_t*>(mem);
  auto take = [&](size_t nb) {
    uint8_t* r = q;
    q += (nb + 255) & ~size_t(255);
    return r;
  };
  B->w_hi = take(wbytes);
  B->w_lo = take(wbytes);
  B->c_hi = take(cbytes);
  B->c_lo = take(cbytes);
  B->consts = reinterpret_cast<float*>(take((size_t)mp * 8));
  double* pbar = reinterpret_cast<double*>(take((size_t)k * 8));
  FKK_COUNT_LAUNCH();
  pack_w_kernel<<<(unsigned)(((int64_t)kp1 * mp + 255) / 256), 256, 0, st>>>(
      B->w, B->f, m, k, kp1, mp, (__nv_bfloat16*)B->w_hi, (__nv_bfloat16*)B->w_lo);
  FKK_COUNT_LAUNCH();
  pbar_kernel<<<k, 256, 0, st>>>(B->w, B->f, B->a_off, m, k, pbar);
  FKK_COUNT_LAUNCH();
  pack_c_kernel<<<(unsigned)(((int64_t)katoms * rows_c * kKp + 255) / 256), 256, 0, st>>>(
      B->c_amp, B->c_ph, pbar, k, m, rows_c, katoms, (__nv_bfloat16*)B->c_hi, (__nv_bfloat16*)B->c_lo);
  FKK_COUNT_LAUNCH();
  chan_consts_kernel<<<(mp + 255) / 256, 256, 0, st>>>(B->i_ref, B->a_off, m, mp, B->consts);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(mem);
    return cuda_check(ctx, e, "apply operand packing");
  }
  B->pack_kp1 = kp1;
  B->pack_mp = mp;
  B->pack_rows_c = rows_c;
  B->pack = mem;
  return FKK_OK;
}

fkk_status launch_apply_fused(fkk_ctx* ctx, const fkk_basis* B, const float* i_cars, int64_t n, int64_t ld,
                              float* im, float* re, int64_t ld_out, cudaStream_t st, bool* handled) {
  *handled = false;
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  // the TMA boxes need 16-byte aligned rows; the output rows must also end
  // on a 16-byte boundary (a store clipped at the last channel still writes
  // the rest of its 16-byte granule, which would reach into a padded stride)
  if (ld % 4 || ld_out % 4 || B->m % 4 || !al16(i_cars) || !al16(im) || (re && !al16(re))) return FKK_OK;
  if (n > ((int64_t)1 << 31) - kTM) return FKK_OK;
  if (is_host_ptr(i_cars) || is_host_ptr(im) || (re && is_host_ptr(re))) return FKK_OK;
  const bool x3 = B->params.precision != FKK_PREC_BF16;
  FusedArgs a{};
  a.kp1 = ((B->k + 2 + 15) / 16) * 16;
  const size_t smem = fused_smem(a.kp1, x3, re != nullptr, ctx->apply_stages, &a.stages, &a.stage_bytes, &a.w_bytes);
  // two K atoms at k > 62 fit only the single-product form; the rest takes the two-kernel path
  if (smem > 227 * 1024) return FKK_OK;
  *handled = true;
  FKK_TRY(apply_pack(ctx, B, st));
  const int m = B->m;
  a.n = n;
  a.m = m;
  a.k = B->k;
  a.katoms = (a.kp1 + kKp - 1) / kKp;
  a.rows_c = B->pack_rows_c;
  a.n_chunks = (m + kCh - 1) / kCh;
  a.n_ct = (2 * m + kNT - 1) / kNT;
  a.n_tiles = (int)((n + kTM - 1) / kTM);
  a.x3 = x3 ? 1 : 0;
  a.floor_ = B->params.ratio_floor;
  a.consts = B->consts;
  a.status = ctx->d_status;
  CUtensorMap ti, twh, twl, tch, tcl, tim, tre;
  FKK_TRY(make_tmap_2d(ctx, &ti, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, const_cast<float*>(i_cars), (uint64_t)m,
                       (uint64_t)n, (uint64_t)ld * 4, 32, kTM, CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &twh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B->w_hi, (uint64_t)B->pack_mp,
                       (uint64_t)a.kp1, (uint64_t)B->pack_mp * 2, 64, (uint32_t)a.kp1, CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &twl, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B->w_lo, (uint64_t)B->pack_mp,
                       (uint64_t)a.kp1, (uint64_t)B->pack_mp * 2, 64, (uint32_t)a.kp1, CU_TENSOR_MAP_SWIZZLE_128B));
  const uint64_t crows = (uint64_t)a.katoms * B->pack_rows_c;
  FKK_TRY(make_tmap_2d(ctx, &tch, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B->c_hi, (uint64_t)kKp, crows, (uint64_t)kKp * 2,
                       64, kNT, CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &tcl, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B->c_lo, (uint64_t)kKp, crows, (uint64_t)kKp * 2,
                       64, kNT, CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &tim, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, im, (uint64_t)m, (uint64_t)n,
                       (uint64_t)ld_out * 4, 32, 32, CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &tre, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, re ? re : im, (uint64_t)m, (uint64_t)n,
                       (uint64_t)ld_out * 4, 32, 32, CU_TENSOR_MAP_SWIZZLE_128B));
  const void* fn = re ? (const void*)apply_fused_kernel<true> : (const void*)apply_fused_kernel<false>;
  FKK_CUDA(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = (int)std::min<int64_t>(ctx->sm_count, a.n_tiles);
  FKK_COUNT_LAUNCH();
  if (re)
    apply_fused_kernel<true><<<grid, kThreads, smem, st>>>(ti, twh, twl, tch, tcl, tim, tre, a);
  else
    apply_fused_kernel<false><<<grid, kThreads, smem, st>>>(ti, twh, twl, tch, tcl, tim, tre, a);
  return cuda_check(ctx, cudaGetLastError(), "apply_fused_kernel launch");
}

}  // namespace fkk
