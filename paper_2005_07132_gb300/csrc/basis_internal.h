// The trained basis object shared by the library's translation units.
#pragma once

#include <mutex>

#include "fkk_internal.h"

struct fkk_basis {
  int device = 0;
  int m = 0, k = 0, L = 0;
  fkk_fit_params params{};
  double* f = nullptr;      // m (always materialised, 1 when f = 1)
  double* lam = nullptr;    // k
  double* s = nullptr;      // k
  double* v = nullptr;      // m x k
  double* w = nullptr;      // m x k: V diag(s^2/(s^2+ml_lambda))
  double* b = nullptr;      // k x m each below
  double* h_b = nullptr;
  double* phi_pec_t = nullptr;
  double* h_phi = nullptr;
  double* v_sec_t = nullptr;
  double* c_amp = nullptr;
  double* c_ph = nullptr;
  double* a_off = nullptr;  // m: training mean of 1/2 ln max(I/I_ref, floor) (0 for imported bases)
  int64_t* q = nullptr;     // up to 2k
  int* nq = nullptr;        // device count
  double* energy = nullptr; // trace(A^T A) of the training cube (in the pad after nq)
  float* i_ref = nullptr;   // m
  void* block = nullptr;    // single allocation backing all of the above
  // Operands of the fused apply, packed on first use (not part of the saved
  // file; rebuilt after fkk_basis_set_offset): f W as bf16 hi / lo
  // (kp1 x mp), the interleaved coefficients with the offset's contribution
  // in two extra K columns as bf16 hi / lo (rows_c x 64), and per 64-channel
  // chunk 1 / I_ref and the offset as floats ([mp / 64][2][64]).
  std::mutex pack_mu;
  void* pack = nullptr;
  int pack_kp1 = 0, pack_mp = 0, pack_rows_c = 0;
  void* w_hi = nullptr;
  void* w_lo = nullptr;
  void* c_hi = nullptr;
  void* c_lo = nullptr;
  float* consts = nullptr;
};
