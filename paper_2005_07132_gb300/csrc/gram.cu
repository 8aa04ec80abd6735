// Gram matrix of the transformed cube on the 5th-generation tensor cores.
//
// G_d = D^T D over all spectra, D = hi + lo (two bf16 terms), computed as
// hi.hi + hi.lo + lo.hi with fp32 accumulation in TMEM: every product of
// two bf16 values is exact in fp32, so the errors left are the rounding of d
// to hi + lo (2^-18 |d|, unbiased), the fp32 accumulation (kept short by the
// split-K) and the dropped lo.lo term.  Off the diagonal, sum_n lo_i lo_j is a
// sum of products of rounding residuals, 2^-16 below the other terms and of
// either sign; on the diagonal it would be a positive bias of ~2^-18 sum d^2,
// so the diagonal is taken instead from the exact sum_n d_j^2 of the
// transform (fp32 within a 64-row tile, double-word across tiles).  On the test
// cubes this leaves the spectral-norm error of G where four products put it
// (1e-7 of ||G||).  The rectangular A^T Q of the randomised SVD keeps all
// four products.  Output tiles are
// 128 (rows i) x 256 (columns j) covering the upper triangle (i-block 128*ib
// < 256*(jb+1)); the contraction over spectra is split into `splits`
// contiguous ranges, one CTA per (tile, split), and the fp32 partial tiles
// are summed in a fixed order, in double-word arithmetic, by the assemble
// kernel, which also adds the shift terms and the f(w) scaling.
//
// CTA = 4 warps.  Warp 0 lane 0 issues TMA loads of 64-spectrum K-blocks
// (A: 128 channels, B: 256 channels, hi and lo) into a 2-stage ring; warp 1
// lane 0 issues tcgen05.mma (M=128, N=256, K=16) from shared memory into a
// 256-column TMEM accumulator; after the last K-block all 4 warps read the
// accumulator (one TMEM lane per row) and store the partial tile.
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "df64.cuh"
#include "fit.h"
#include "tc.cuh"

namespace fkk {

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

fkk_status make_tmap_2d(fkk_ctx* ctx, CUtensorMap* map, CUtensorMapDataType dt, void* base, uint64_t inner,
                        uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer,
                        CUtensorMapSwizzle swz) {
  std::call_once(g_encode_once, [] {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!g_encode) return fail(ctx, FKK_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = g_encode(map, dt, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, FKK_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return FKK_OK;
}

namespace {

constexpr int kBK = 64;                       // spectra per K-block (128 bytes of bf16)
constexpr int kTileM = 128, kTileN = 256;
constexpr int kStages = 2;
constexpr int kAccBlocks = 96;                // K-blocks per fp32 accumulation (6,144 spectra)
constexpr uint32_t kABytes = kTileM * kBK * 2;  // 16 KB per term
template <int TN>
constexpr uint32_t stage_bytes() { return 2 * kABytes + 2 * (uint32_t)TN * kBK * 2; }
template <int TN>
constexpr size_t gram_smem() { return kStages * stage_bytes<TN>() + 1024 /*align*/ + 256 /*barriers*/; }

struct GramArgs {
  int mb;        // row blocks of 128
  int ntiles;
  int64_t nkb;   // K-blocks of 64 spectra
  int splits;
  float* partial;  // [splits][ntiles][128][TN]
  long long* status;
};

// tile t -> (ib, jb) enumerating jb = 0, 1, ... and ib < min(2 (jb + 1), mb)
__host__ __device__ inline void gram_tile(int t, int mb, int& ib, int& jb) {
  jb = 0;
  for (;;) {
    int cnt = 2 * (jb + 1) < mb ? 2 * (jb + 1) : mb;
    if (t < cnt) { ib = t; return; }
    t -= cnt;
    ++jb;
  }
}

// TN: columns of an output tile (the B operand's rows per K-block).  RECT:
// the tiles are the mb row blocks of one column block (A^T Q, Q with at most
// TN columns) instead of the upper triangle of A^T A.
template <int TN, bool RECT>
__global__ void __launch_bounds__(128, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap tm_a_hi, const __grid_constant__ CUtensorMap tm_a_lo,
                   const __grid_constant__ CUtensorMap tm_b_hi, const __grid_constant__ CUtensorMap tm_b_lo,
                   GramArgs p) {
  constexpr uint32_t kBBytes = (uint32_t)TN * kBK * 2;
  constexpr uint32_t kStageBytes = stage_bytes<TN>();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int fail_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ib, jb;
  if (RECT) {
    ib = blockIdx.x;
    jb = 0;
  } else {
    gram_tile(blockIdx.x, p.mb, ib, jb);
  }
  const int split = blockIdx.y;
  const int64_t kb0 = p.nkb * split / p.splits;
  const int64_t kb1 = p.nkb * (split + 1) / p.splits;
  const int nk = (int)(kb1 - kb0);

  if (threadIdx.x == 0) {
    fail_s = 0;
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tm_a_hi);
    tc::prefetch_tmap(&tm_a_lo);
    tc::prefetch_tmap(&tm_b_hi);
    tc::prefetch_tmap(&tm_b_lo);
  }
  if (warp == 2) tc::tmem_alloc(tmem_slot, TN);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t taddr = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer
    for (int i = 0; i < nk; ++i) {
      const int s = i % kStages;
      const uint32_t ph = (i / kStages) & 1;
      if (!tc::mbar_wait(&empty[s], ph ^ 1)) { fail_s = 1; break; }
      uint8_t* st = smem + s * kStageBytes;
      tc::mbar_arrive_expect_tx(&full[s], kStageBytes);
      const int x = (int)((kb0 + i) * kBK);
      tc::tma_load_2d(st, &tm_a_hi, &full[s], x, ib * kTileM);
      tc::tma_load_2d(st + kABytes, &tm_a_lo, &full[s], x, ib * kTileM);
      tc::tma_load_2d(st + 2 * kABytes, &tm_b_hi, &full[s], x, jb * TN);
      tc::tma_load_2d(st + 2 * kABytes + kBBytes, &tm_b_lo, &full[s], x, jb * TN);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTileM, TN);
    bool ok = true;
    for (int i = 0; i < nk; ++i) {
      const int s = i % kStages;
      const uint32_t ph = (i / kStages) & 1;
      if (!tc::mbar_wait(&full[s], ph)) { ok = false; fail_s = 1; break; }
      tc::tc_fence_after();
      const uint32_t a_hi = tc::smem_u32(smem + s * kStageBytes);
      const uint32_t a_lo = a_hi + kABytes;
      const uint32_t b_hi = a_hi + 2 * kABytes;
      const uint32_t b_lo = b_hi + kBBytes;
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        const uint32_t off = kk * 32;  // 16 bf16 along K
        tc::mma_bf16(taddr, tc::sdesc_kmajor_sw128(a_hi + off), tc::sdesc_kmajor_sw128(b_hi + off), idesc,
                     (i > 0 || kk > 0) ? 1u : 0u);
        tc::mma_bf16(taddr, tc::sdesc_kmajor_sw128(a_hi + off), tc::sdesc_kmajor_sw128(b_lo + off), idesc, 1u);
        tc::mma_bf16(taddr, tc::sdesc_kmajor_sw128(a_lo + off), tc::sdesc_kmajor_sw128(b_hi + off), idesc, 1u);
        if (RECT)
          tc::mma_bf16(taddr, tc::sdesc_kmajor_sw128(a_lo + off), tc::sdesc_kmajor_sw128(b_lo + off), idesc, 1u);
      }
      tc::mma_commit(&empty[s]);
    }
    if (ok) tc::mma_commit(done);
  }
  __syncthreads();  // fail_s written by the producer / MMA lanes is visible below

  // epilogue: every warp reads its 32 TMEM lanes (rows) x 256 columns
  bool have = (nk > 0);
  if (have) {
    if (!tc::mbar_wait(done, 0)) {
      have = false;
      fail_s = 1;
    }
  }
  tc::tc_fence_after();
  const int row = warp * 32 + lane;
  float* out = p.partial + (((int64_t)split * p.ntiles + blockIdx.x) * kTileM + row) * TN;
  const bool failed = fail_s != 0;
  for (int c = 0; c < TN / 32; ++c) {
    float v[32];
    if (have && !failed) {
      tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + c * 32, v);
    } else {
#pragma unroll
      for (int q = 0; q < 32; ++q) v[q] = 0.f;
    }
    float4* o4 = reinterpret_cast<float4*>(out + c * 32);
#pragma unroll
    for (int q = 0; q < 8; ++q) o4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  }
  if (failed && threadIdx.x == 0) record_error(p.status, kErrTimeout);
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 2) tc::tmem_dealloc(taddr, TN);
}

// Sum partial tiles (fixed split order, fp64), add the shift terms, scale by
// f, write both triangles of the m x m matrix.
__global__ void gram_assemble_kernel(const float* __restrict__ partial, int splits, int ntiles, int mb, int m,
                                     int64_t n, const float* __restrict__ c, const double* __restrict__ sd,
                                     const double* __restrict__ sd2, const double* __restrict__ f,
                                     double* __restrict__ g) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (j >= m || j < i) return;
  const int ib = i / kTileM, jb = j / kTileN;
  int base = 0;
  for (int q = 0; q < jb; ++q) base += (2 * (q + 1) < mb ? 2 * (q + 1) : mb);
  const int tile = base + ib;
  const int64_t off = ((int64_t)tile * kTileM + (i - ib * kTileM)) * kTileN + (j - jb * kTileN);
  const int64_t tstride = (int64_t)ntiles * kTileM * kTileN;
  double acc = 0.0;
  if (i == j) {
    acc = sd2[i];  // exact sum of d^2 (the tiles lack lo.lo)
  } else {
    // the fp32 partials summed in double-word arithmetic on the fp32 pipe
    // (about 48 bits; GB300's fp64 rate would make this the bottleneck):
    // four chains for loads in flight, combined in a fixed order
    dw::df a4[4] = {dw::make(0.f), dw::make(0.f), dw::make(0.f), dw::make(0.f)};
    int s = 0;
    for (; s + 4 <= splits; s += 4) {
#pragma unroll
      for (int q = 0; q < 4; ++q) a4[q] = dw::add(a4[q], partial[(int64_t)(s + q) * tstride + off]);
    }
    for (int q = 0; s < splits; ++s, ++q) a4[q] = dw::add(a4[q], partial[(int64_t)s * tstride + off]);
    acc = dw::to_double(dw::add(dw::add(a4[0], a4[1]), dw::add(a4[2], a4[3])));
  }
  const double ci = c[i], cj = c[j];
  acc += sd[i] * cj + ci * sd[j] + (double)n * ci * cj;
  if (f) acc *= f[i] * f[j];
  g[(int64_t)i * m + j] = acc;
  g[(int64_t)j * m + i] = acc;
}

__global__ void noise_scale_kernel(const double* __restrict__ sum_i, int64_t n, int m, double alpha,
                                   double sigma_g, double* __restrict__ f) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double mean = sum_i[j] / (double)n;
  f[j] = 2.0 * mean / sqrt(alpha * mean + sigma_g * sigma_g);
}

}  // namespace

fkk_status launch_noise_scale(fkk_ctx* ctx, const double* sum_i, int64_t n, int m, double alpha,
                              double sigma_g, double* f, cudaStream_t st) {
  FKK_COUNT_LAUNCH(); noise_scale_kernel<<<(m + 127) / 128, 128, 0, st>>>(sum_i, n, m, alpha, sigma_g, f);
  return cuda_check(ctx, cudaGetLastError(), "noise_scale launch");
}

// Z = A^T Q for A = f (d + c) (the transformed cube with its shift) and Q
// (n x l) given as Q^T in bf16 hi / lo, [tn][np] K-major (rows >= l and
// spectra >= n zero), with colsum[i] = sum_n Q[n, i]:
//   Z[j, i] = f_j (sum_n d[n, j] Q[n, i] + c_j colsum[i]).
__global__ void atq_assemble_kernel(const float* __restrict__ partial, int splits, int mb, int tn, int m, int l,
                                    const float* __restrict__ c, const double* __restrict__ colsum,
                                    const double* __restrict__ f, double* __restrict__ z) {
  const int j = blockIdx.x, i = threadIdx.x;
  if (j >= m || i >= l) return;
  const int ib = j / kTileM;
  const int64_t off = ((int64_t)ib * kTileM + (j - ib * kTileM)) * tn + i;
  const int64_t sstride = (int64_t)mb * kTileM * tn;
  dw::df a = dw::make(0.f);  // double-word sum on the fp32 pipe, in split order
  for (int s = 0; s < splits; ++s) a = dw::add(a, partial[(int64_t)s * sstride + off]);
  double acc = dw::to_double(a);
  acc += (double)c[j] * colsum[i];
  z[(int64_t)j * l + i] = f ? acc * f[j] : acc;
}

fkk_status launch_atq(fkk_ctx* ctx, const DtLayout& L, const __nv_bfloat16* qt_hi, const __nv_bfloat16* qt_lo,
                      int tn, int l, const double* colsum, const double* f, double* z, cudaStream_t st) {
  if (tn != 64 && tn != 128) return fail(ctx, FKK_ERR_INVALID_ARG, "A^T Q: %d columns per tile", tn);
  fkk_status s;
  const int mb = L.mg / kTileM;
  const int64_t nkb = L.np / kBK;
  int64_t splits = ((int64_t)ctx->sm_count * 4 + mb - 1) / mb;
  if (splits < (nkb + kAccBlocks - 1) / kAccBlocks) splits = (nkb + kAccBlocks - 1) / kAccBlocks;
  if (splits > nkb) splits = nkb;
  if (splits < 1) splits = 1;
  float* partial = (float*)workspace(ctx, "atq_partial", (size_t)splits * mb * kTileM * tn * sizeof(float), &s);
  if (!partial) return s;
  CUtensorMap ta_hi, ta_lo, tb_hi, tb_lo;
  const uint64_t row_bytes = (uint64_t)L.np * 2;
  FKK_TRY(make_tmap_2d(ctx, &ta_hi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, L.dt_hi, L.np, L.mg, row_bytes, kBK, kTileM,
                       CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &ta_lo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, L.dt_lo, L.np, L.mg, row_bytes, kBK, kTileM,
                       CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &tb_hi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (void*)qt_hi, L.np, tn, row_bytes, kBK, tn,
                       CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &tb_lo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (void*)qt_lo, L.np, tn, row_bytes, kBK, tn,
                       CU_TENSOR_MAP_SWIZZLE_128B));
  GramArgs a{mb, mb, nkb, (int)splits, partial, ctx->d_status};
  if (tn == 64) {
    auto kern = gram_tc_kernel<64, true>;
    FKK_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_smem<64>()));
    FKK_COUNT_LAUNCH(); kern<<<dim3(mb, (unsigned)splits), 128, gram_smem<64>(), st>>>(ta_hi, ta_lo, tb_hi, tb_lo, a);
  } else {
    auto kern = gram_tc_kernel<128, true>;
    FKK_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_smem<128>()));
    FKK_COUNT_LAUNCH(); kern<<<dim3(mb, (unsigned)splits), 128, gram_smem<128>(), st>>>(ta_hi, ta_lo, tb_hi, tb_lo, a);
  }
  FKK_CUDA(ctx, cudaGetLastError());
  FKK_COUNT_LAUNCH();
  atq_assemble_kernel<<<L.m, ((l + 31) / 32) * 32, 0, st>>>(partial, (int)splits, mb, tn, L.m, l, L.c, colsum, f, z);
  return cuda_check(ctx, cudaGetLastError(), "A^T Q assemble launch");
}

fkk_status launch_gram(fkk_ctx* ctx, const DtLayout& L, const double* f, double* g, cudaStream_t st) {
  fkk_status s;
  const int mb = L.mg / kTileM;
  const int jbs = L.mg / kTileN;
  int ntiles = 0;
  for (int q = 0; q < jbs; ++q) ntiles += (2 * (q + 1) < mb ? 2 * (q + 1) : mb);
  const int64_t nkb = L.np / kBK;
  // enough CTAs for several waves, at least 8 and at most kAccBlocks
  // K-blocks each (the fp32 TMEM accumulation length per partial tile)
  int64_t splits = ((int64_t)ctx->sm_count * 5 + ntiles - 1) / ntiles;
  if (splits < (nkb + kAccBlocks - 1) / kAccBlocks) splits = (nkb + kAccBlocks - 1) / kAccBlocks;
  if (splits > nkb / 8) splits = nkb / 8;
  if (splits < 1) splits = 1;
  float* partial =
      (float*)workspace(ctx, "gram_partial", (size_t)splits * ntiles * kTileM * kTileN * sizeof(float), &s);
  if (!partial) return s;
  CUtensorMap ta_hi, ta_lo, tb_hi, tb_lo;
  const uint64_t row_bytes = (uint64_t)L.np * 2;
  FKK_TRY(make_tmap_2d(ctx, &ta_hi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, L.dt_hi, L.np, L.mg, row_bytes, kBK, kTileM,
                       CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &ta_lo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, L.dt_lo, L.np, L.mg, row_bytes, kBK, kTileM,
                       CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &tb_hi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, L.dt_hi, L.np, L.mg, row_bytes, kBK, kTileN,
                       CU_TENSOR_MAP_SWIZZLE_128B));
  FKK_TRY(make_tmap_2d(ctx, &tb_lo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, L.dt_lo, L.np, L.mg, row_bytes, kBK, kTileN,
                       CU_TENSOR_MAP_SWIZZLE_128B));
  auto kern = gram_tc_kernel<kTileN, false>;
  FKK_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_smem<kTileN>()));
  GramArgs a{mb, ntiles, nkb, (int)splits, partial, ctx->d_status};
  FKK_COUNT_LAUNCH(); kern<<<dim3(ntiles, (unsigned)splits), 128, gram_smem<kTileN>(), st>>>(ta_hi, ta_lo, tb_hi, tb_lo, a);
  FKK_CUDA(ctx, cudaGetLastError());
  dim3 grid((L.m + 127) / 128, L.m);
  FKK_COUNT_LAUNCH(); gram_assemble_kernel<<<grid, 128, 0, st>>>(partial, (int)splits, ntiles, mb, L.m, L.n, L.c, L.sum_d, L.sum_d2, f,
                                                                 g);
  return cuda_check(ctx, cudaGetLastError(), "gram_assemble launch");
}

}  // namespace fkk
