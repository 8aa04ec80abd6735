// Internal launchers of the fKK-EC fit pipeline (host side).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "fkk_internal.h"

namespace fkk {

// Channel-major transformed cube: D^T_hi / D^T_lo are mg x np bf16 arrays
// (row = channel, contiguous along spectra), rows >= m and columns >= n are 0.
struct DtLayout {
  int64_t n = 0, np = 0;  // spectra, padded to a multiple of 64
  int m = 0, mg = 0;      // channels, padded to a multiple of 256
  __nv_bfloat16* dt_hi = nullptr;
  __nv_bfloat16* dt_lo = nullptr;
  float* c = nullptr;        // per-channel shift (m)
  double* sum_d = nullptr;   // sum_n d[n, j] (m)
  double* sum_i = nullptr;   // sum_n I[n, j] (m)
  double* sum_d2 = nullptr;  // sum_n d[n, j]^2 (m)
};

struct TransformArgs {
  const float* i_cars;
  int64_t n;
  int m;
  int64_t ld;
  const float* i_ref;
  float floor_;
  const float* c;
  int64_t np;
  __nv_bfloat16* dt_hi;
  __nv_bfloat16* dt_lo;
  double* part_d;
  double* part_i;
  double* part_d2;
  long long* status;
};

// raw = false: d = 1/2 ln(max(I/I_ref, floor)) - c (the fit's A before f);
// raw = true: d = I - c, the raw spectra (c the mean of the first rows).
fkk_status launch_transform(fkk_ctx* ctx, const float* i_cars, int64_t n, int m, int64_t ld,
                            const float* i_ref, float floor_, DtLayout& L, cudaStream_t st, bool raw = false);

// G = diag(f) (D^T D + s c^T + c s^T + N c c^T) diag(f), fp64, m x m (ld m).
// f == nullptr means f = 1.
fkk_status launch_gram(fkk_ctx* ctx, const DtLayout& L, const double* f, double* g, cudaStream_t st);

// f(w) = 2 <I> / sqrt(alpha <I> + sigma_g^2) from the channel sums of I.
fkk_status launch_noise_scale(fkk_ctx* ctx, const double* sum_i, int64_t n, int m, double alpha,
                              double sigma_g, double* f, cudaStream_t st);

// Top-k eigenpairs of the symmetric m x m fp64 G: lam (k, descending) and
// V (m x k, row-major), each column's largest-magnitude entry positive.
fkk_status launch_eig_topk(fkk_ctx* ctx, const double* g, int m, int k, double* lam, double* v,
                           cudaStream_t st);

// P = A W (n x k fp32, ld k) from the transformed cube, with A = (d + c) f
// folded into W: P[n,i] = sum_j d[n,j] Wf[j,i] + o_i, Wf = f W, o = c^T Wf.
// Per column of P the argmax / argmin row (ties to the lowest row) goes to
// qmax / qmin (device, k each).  Optional outputs may be null.
fkk_status launch_project(fkk_ctx* ctx, const DtLayout& L, const double* w, const double* f, int k, float* p,
                          int64_t* qmax, int64_t* qmin, cudaStream_t st);

// Same on the tensor cores (bf16 hi/lo operands, four products); cand, when
// not null, receives per 128-row tile and column (max, argmax, min, argmin).
fkk_status launch_project_tc(fkk_ctx* ctx, const DtLayout& L, const double* w, const double* f, int k, float* p,
                             float4* cand, cudaStream_t st);

// P = A W from the raw cube (for new data): A = f * 1/2 ln(max(I/I_ref, floor)).
fkk_status launch_project_raw(fkk_ctx* ctx, const float* i_cars, int64_t n, int m, int64_t ld,
                              const float* i_ref, float floor_, const double* w, const double* f, int k,
                              float* p, cudaStream_t st);

// Basis math (fKK / fPEC / fSEC on the k vectors), all fp64, on the device.
struct BasisParams {
  int m, k, L;
  int pec, sec;
  double als_lambda, als_p;
  int als_iters;
  double ridge_rel;
  int sec_mode;  // 0 Savitzky-Golay, 1 mean
  int sg_window, sg_order;
};
// v: m x k (row-major); f: m; x_rows: nq x k (P_q, fp64, row-major, device).
// Outputs (device, k x m row-major): c_amp, c_ph, and the pieces b, h_b,
// phi_pec_t, h_phi, v_sec_t when the pointers are non-null.
struct BasisOut {
  double* c_amp;
  double* c_ph;
  double* b;
  double* h_b;
  double* phi_pec_t;
  double* h_phi;
  double* v_sec_t;
};
fkk_status launch_basis_math(fkk_ctx* ctx, const BasisParams& bp, const double* v, const double* f,
                             const double* x_rows, int nq, BasisOut out, cudaStream_t st);

// q = sorted unique(qmax U qmin) (device int64, up to 2k), count to *nq_dev;
// x_rows[r, :] = (double) P[q[r], :].
fkk_status launch_gather_q(fkk_ctx* ctx, const int64_t* qmax, const int64_t* qmin, int k, const float* p,
                           int64_t n_rows, int64_t* q, int* nq_dev, double* x_rows, cudaStream_t st);

// Out = exp(P C_amp) sin(P C_ph) (and cos for re_out), P n x k fp32 (the
// tensor-core reconstruction, three bf16 products per term).
fkk_status launch_reconstruct(fkk_ctx* ctx, const float* p, int64_t n, int k, int m, const double* c_amp,
                              const double* c_ph, float* im, float* re, int64_t ld_out, cudaStream_t st);

// ML:fKK-EC apply of a trained basis in one fused launch (projection of the
// raw spectra and reconstruction) in the basis' precision.  *handled is false
// and nothing is launched when TMA cannot address the arrays (row strides not
// multiples of 4 floats, 16-byte misaligned or host arrays) or k > 62.
fkk_status launch_apply_fused(fkk_ctx* ctx, const fkk_basis* B, const float* i_cars, int64_t n, int64_t ld,
                              float* im, float* re, int64_t ld_out, cudaStream_t st, bool* handled);

// Packed operands of the fused apply, built once per basis (and again after
// fkk_basis_set_offset).
fkk_status apply_pack(fkk_ctx* ctx, const fkk_basis* B, cudaStream_t st);

// Out = P C + 1 b^T (n x m, ld_out), C k x m fp64 row-major, b m floats or
// null: the linear epilogue of the same tensor-core kernel (the SVD
// denoising's X_k = (X V_k) V_k^T, with the shift's share in b).
fkk_status launch_reconstruct_linear(fkk_ctx* ctx, const float* p, int64_t n, int k, int m, const double* c,
                                     const float* bias, float* out, int64_t ld_out, cudaStream_t st);

// Same, on the tensor cores (bf16 x3 operands, exp / sin epilogue), k <= 128.
fkk_status launch_reconstruct_tc(fkk_ctx* ctx, const float* p, int64_t n, int k, int m, const double* c_amp,
                                 const double* c_ph, float* im, float* re, int64_t ld_out, cudaStream_t st);

// Same, with the packed operands in caller-provided scratch instead of the
// context's workspace: p_hi / p_lo hold ceil(n / 128) * 128 x Kp bf16 each,
// c_hi / c_lo ceil(2m / 256) * 256 x Kp bf16 each (Kp = 64 for k <= 64,
// else 128), each 16-byte aligned.  Allocates nothing.
fkk_status launch_reconstruct_tc_scratch(fkk_ctx* ctx, const float* p, int64_t n, int k, int m,
                                         const double* c_amp, const double* c_ph, float* im, float* re,
                                         int64_t ld_out, cudaStream_t st, void* p_hi, void* p_lo, void* c_hi,
                                         void* c_lo);

// The per-spectrum KK kernel in its phase mode: phi = H{1/2 ln max(I/I_ref,
// floor)} for n spectra, written with row stride ld_phi.
// Register-FFT per-spectrum KK for pad lengths 1024 and 2048 (one warp per
// pair of spectra); *handled is false (and nothing is launched) otherwise.
fkk_status launch_kk_warp(fkk_ctx* ctx, const float* i_cars, int64_t n, int m, int64_t ld, const float* i_ref,
                          int L, float floor_, float* im, float* re, int64_t ld_out, bool phase, cudaStream_t st,
                          bool* handled);

fkk_status launch_kk_phase(fkk_ctx* ctx, const float* i_cars, int64_t n, int m, int64_t ld,
                           const float* i_ref, int L, float floor_, float* phi, int64_t ld_phi,
                           cudaStream_t st);

// Small fp64 Cholesky-QR steps (m x k row-major, k small): W = Z^T Z;
// R^-1 with W = R^T R -- a pivot below drop_tol of its column's squared norm
// is FKK_ERR_NOT_CONVERGED when strict, else that column is dropped (its
// column of Z R^-1 is 0); V = Z R^-1; the largest-magnitude component of each
// column made positive.
fkk_status launch_ztz(fkk_ctx* ctx, const double* z, int m, int k, double* w, cudaStream_t st);
fkk_status launch_chol_inv(fkk_ctx* ctx, const double* w, int k, double* rinv, cudaStream_t st, double drop_tol,
                           bool strict);
fkk_status launch_apply_rinv(fkk_ctx* ctx, const double* z, int m, int k, const double* rinv, double* v,
                             cudaStream_t st);
fkk_status launch_sign_fix(fkk_ctx* ctx, double* v, int m, int k, cudaStream_t st);
// Refinement of a kept basis of G's eigensolve (refine.cu): `steps` times
// V <- orth(G V) and the Rayleigh-Ritz pairs of G on that span; lam (k) and
// v_out (m x k, may alias v_in) receive the result.
fkk_status launch_refine(fkk_ctx* ctx, const double* g, int m, int k, const double* v_in, int steps, double* lam,
                         double* v_out, cudaStream_t st);

// Z = A^T Q (m x l fp64) for the transformed cube and Q given as Q^T in
// bf16 hi / lo ([tn][np], tn = 64 or 128 >= l, zero beyond l and n) with its
// column sums (for the shift c); f may be null (f = 1).
fkk_status launch_atq(fkk_ctx* ctx, const DtLayout& L, const __nv_bfloat16* qt_hi, const __nv_bfloat16* qt_lo,
                      int tn, int l, const double* colsum, const double* f, double* z, cudaStream_t st);

// Randomised SVD of A (the transformed cube scaled by f): randomised subspace
// iteration with l = k + oversample Philox4x64-10 Gaussian test vectors
// (counter e / 2, key (seed, 0), Box-Muller) and `power_iters` iterations;
// lam (k) = s^2 and v (m x k) of the k largest, as launch_eig_topk.
fkk_status launch_rsvd(fkk_ctx* ctx, const DtLayout& L, const double* f, int k, int oversample, int power_iters,
                       uint64_t seed, double* lam, double* v, cudaStream_t st);

// Tensor map helper (driver entry point fetched once).
fkk_status make_tmap_2d(fkk_ctx* ctx, CUtensorMap* map, CUtensorMapDataType dt, void* base, uint64_t inner,
                        uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer,
                        CUtensorMapSwizzle swz);

}  // namespace fkk
