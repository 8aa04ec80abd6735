// Reconstruction entry used by the fit and the apply paths; the kernel is
// the tensor-core GEMM with the exp / sin epilogue in recon_tc.cu.
#include "fit.h"

namespace fkk {

fkk_status launch_reconstruct(fkk_ctx* ctx, const float* p, int64_t n, int k, int m, const double* c_amp,
                              const double* c_ph, float* im, float* re, int64_t ld_out, cudaStream_t st) {
  return launch_reconstruct_tc(ctx, p, n, k, m, c_amp, c_ph, im, re, ld_out, st);
}

}  // namespace fkk
