/*
 * fkk.h -- C ABI of the GB300 (sm_103a) fKK-EC library.
 *
 * Method: Camp, Bender & Lee, "Real-time and high-throughput Raman signal
 * extraction and processing in CARS hyperspectral imaging" (arXiv 2005.07132).
 * Section, equation and figure names below refer to that paper.
 *
 * Naming: the paper calls the number of spectra M and the number of
 * frequency channels N (Sec. 2.2).  This ABI spells both out: n_spectra
 * (rows, pixels) and n_channels (columns, frequencies).
 *
 * Conventions shared by every entry point
 *   - Arrays are row-major, one spectrum per row (Sec. 2.2 orients the data
 *     "row = spatial, column = frequency").  `ld` / `ld_out` are the row
 *     strides in elements (>= n_channels).
 *   - Unless a parameter says "host", every array pointer is a DEVICE pointer
 *     on the context's device, owned by the caller; the library never frees
 *     it and never keeps it after the call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued on it; calls return after enqueueing unless
 *     documented otherwise.  Argument errors are detected on the host before
 *     anything is enqueued and leave outputs untouched.
 *   - Every call returns an fkk_status; no exception crosses the ABI.  After
 *     FKK_ERR_CUDA, fkk_last_error() holds the CUDA message.
 *   - A context is used by one host thread at a time (the serving loop takes
 *     its own lock).
 */
#ifndef FKK_H_
#define FKK_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t fkk_status;

enum {
  FKK_OK = 0,
  FKK_ERR_INVALID_ARG = -1,  /* bad size, stride, pointer or parameter */
  FKK_ERR_BUDGET = -2,       /* the context's HBM budget would be exceeded */
  FKK_ERR_CUDA = -3,         /* a CUDA runtime/driver call failed */
  FKK_ERR_TIMEOUT = -4,      /* a bounded wait ran out (device or host) */
  FKK_ERR_NOT_CONVERGED = -5,/* the eigensolver hit its sweep limit */
  FKK_ERR_BAD_FILE = -6,     /* basis file missing, truncated or corrupt */
  FKK_ERR_SHUTDOWN = -7      /* the server stopped before the request ran */
};

/* Human-readable name of a status code (static storage). */
const char* fkk_strerror(fkk_status s);

/* Library version string, e.g. "fkk 0.1 sm_103a". */
const char* fkk_version(void);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t fkk_launch_count(void);

/* ------------------------------------------------------------------ */
/* Context                                                              */
/* ------------------------------------------------------------------ */

typedef struct fkk_ctx fkk_ctx;

/* Create a context on CUDA device `device`.  Device memory the library
 * allocates for its own workspaces (never the caller's arrays) is capped at
 * `hbm_budget_bytes` (0 = no cap); an allocation that would exceed it fails
 * with FKK_ERR_BUDGET.  *out is set only on success. */
fkk_status fkk_create(fkk_ctx** out, int32_t device, size_t hbm_budget_bytes);

/* Synchronise the device, free every workspace and the context. NULL is ok. */
fkk_status fkk_destroy(fkk_ctx* ctx);

/* Last error message recorded on this context ("" if none).  Valid until
 * the next call on the context. */
const char* fkk_last_error(const fkk_ctx* ctx);

/* Bytes of device workspace the context currently holds. */
size_t fkk_workspace_bytes(const fkk_ctx* ctx);

/* Synchronise `stream`, then read and clear the context's device status:
 * *clamped receives the number of ratios I/I_ref that were raised to the
 * ratio floor since the last read (Sec. 2.1 takes the logarithm of the
 * ratio; non-positive noisy samples are clamped), and the return value is
 * the first device-side error recorded (FKK_ERR_TIMEOUT or
 * FKK_ERR_NOT_CONVERGED), else FKK_OK.  `clamped` may be NULL. */
fkk_status fkk_sync_status(fkk_ctx* ctx, void* stream, int64_t* clamped);

/* Test of the device-side timeout path: the next eigensolve on ctx (in
 * fkk_fit_basis, fkk_eig_topk or conventional_per_spectrum's denoising)
 * waits, in the first column exchange of its tridiagonal reduction, for a
 * tag that no step publishes, with a bound of 2^14 polls instead of 2^20.
 * The wait runs out, the reduction records FKK_ERR_TIMEOUT and every CTA
 * returns; the eigenpairs of that call are undefined, fkk_sync_status
 * reports FKK_ERR_TIMEOUT, and the context stays usable.  One-shot. */
fkk_status fkk_test_stall_next_eigensolve(fkk_ctx* ctx);

/* Per-stage timing of fkk_fit_basis: 0 off; 1 on: each fit records CUDA
 * events on its stream at the boundaries of six stages: 0 transform (log
 * ratio, split, channel sums), 1 Gram, 2 eigensolve, 3 projection and
 * argmax/argmin, 4 basis math (fKK, fPEC, fSEC), 5 reconstruction; 2: as 1,
 * and the eigensolver's reduction also reads the SM clock at its phase
 * boundaries (fkk_eig_phase_cycles), which slows that kernel somewhat. */
fkk_status fkk_set_timing(fkk_ctx* ctx, int32_t on);

/* Milliseconds of the first n (<= 6) stages of the last timed fit;
 * synchronises on its last event. */
fkk_status fkk_stage_ms(fkk_ctx* ctx, float* ms, int32_t n);

/* With timing level 2, the tridiagonal reduction of the last eigensolve records
 * the SM clock cycles one CTA (the owner of the last column) spent per
 * phase, summed over the columns: 0 loading and scaling G and the first
 * reflector, 1 waiting for the exchanged p and pivot column and forming w,
 * 2 the pivot column and the next reflector, 3 the next step's p of the
 * owned columns (published), 4 the deferred update of the owned columns.
 * Copies n (<= 8) words. */
fkk_status fkk_eig_phase_cycles(fkk_ctx* ctx, int64_t* cycles, int32_t n);

/* Measured peak of the arithmetic the eigensolver's tridiagonal reduction
 * (Sec. 2.2, the SVD of A through its Gram matrix) is made of: the
 * double-word multiply-add acc * y + x (a TwoProd-based product and a
 * TwoSum-based sum on the fp32 pipe, two flops).  One kernel on every SM at
 * full occupancy runs 8 independent chains per thread for `iters` steps
 * (1 .. 2^20; about 1 ms per 1,000 steps), after a short warm-up launch,
 * timed with CUDA events on `stream` (NULL = the legacy default stream);
 * the call synchronises.
 *   flops_per_s  (host, may be NULL): 2 * chains * iters / elapsed seconds
 *   chains_out   (host, may be NULL, 8 doubles): thread 0's chain values,
 *                chain c iterating a <- a y + x_c from a = 0 with
 *                y = (1 - 2^-9) + 3 2^-33 and x_c = (0.1f + 2^-30) 2^-c
 *                exactly, for a check against exact arithmetic.
 * FKK_ERR_INVALID_ARG if both outputs are NULL or iters is out of range. */
fkk_status fkk_dw_rate(fkk_ctx* ctx, int32_t iters, double* flops_per_s, double* chains_out, void* stream);

/* ------------------------------------------------------------------ */
/* Conventional per-spectrum KK (Eq. KCARS with the surrogate, Eq. K)   */
/* ------------------------------------------------------------------ */

/* For every spectrum n:
 *   a      = 1/2 ln(max(I_CARS[n,:] / I_ref, ratio_floor))
 *   phi    = H{a}, the discrete Hilbert transform: a is edge-replicated to
 *            pad_len samples (floor((pad_len-M)/2) on the left), its DFT bin
 *            m is multiplied by -i*sgn(m) (0 at DC and Nyquist), the inverse
 *            DFT is cropped back to the M channels
 *   im_out = exp(a) sin(phi)    (Im{K}),   re_out = exp(a) cos(phi)  (Re{K})
 * i_cars: n_spectra x n_channels floats, row stride ld.
 * i_ref:  n_channels floats (the surrogate NRB spectrum).
 * pad_len: power of two with n_channels <= pad_len <= 8192; 0 selects
 *          nextpow2(2 * n_channels).
 * ratio_floor: > 0 (1e-6 is the usual choice).
 * im_out: n_spectra x n_channels floats, row stride ld_out (required).
 * re_out: same shape and stride, or NULL to skip the real part.
 * n_spectra == 0 is a no-op.  Errors: FKK_ERR_INVALID_ARG, FKK_ERR_CUDA. */
fkk_status kk_per_spectrum(fkk_ctx* ctx, const float* i_cars, int64_t n_spectra,
                           int32_t n_channels, int64_t ld, const float* i_ref,
                           int32_t pad_len, float ratio_floor, float* im_out,
                           float* re_out, int64_t ld_out, void* stream);

/* ------------------------------------------------------------------ */
/* fKK-EC fit (Fig. 1(b); Secs. 2.2-2.5) and ML apply (Sec. 2.6)        */
/* ------------------------------------------------------------------ */

enum { FKK_SEC_SAVGOL = 0, FKK_SEC_MEAN = 1 };
/* Arithmetic of ML:fKK-EC apply (fkk_apply and the serving loop; Sec. 2.6),
 * whose two GEMMs -- the projection of the raw spectra and the
 * reconstruction -- run on the tensor cores with fp32 accumulation and an
 * fp32 exp / sin epilogue, on log ratios shifted by the basis' offset
 * (fkk_basis_set_offset):
 *   FKK_PREC_BF16X3  operands split into bf16 hi + lo, three products per
 *                    GEMM (hi.hi + hi.lo + lo.hi): fp32-accurate;
 *   FKK_PREC_BF16    the reduced-precision served form: projection with one
 *                    bf16 product, reconstruction with two (P hi + lo times
 *                    bf16 coefficients) -- half the tensor work; relative L2
 *                    error of Im about 1e-3 or below.
 * The fit (Gram, eigensolve, the fit's projection and reconstruction) is
 * fp32-accurate in both.  Where the fused apply kernel cannot run (see
 * fkk_apply) the apply is fp32-accurate in both. */
enum { FKK_PREC_BF16X3 = 0, FKK_PREC_BF16 = 1 };

typedef struct {
  int32_t k;            /* kept basis vectors, 1..80; 0 = chosen by the rank rule (k_max, rank_eps) */
  int32_t pad_len;      /* Hilbert pad length: 0 = nextpow2(2M); power of two in [M, 4096] */
  int32_t pec;          /* 1 = factorised phase-error correction (Sec. 2.3) */
  int32_t sec;          /* 1 = factorised scale-error correction (Sec. 2.4) */
  double als_lambda;    /* ALS smoothness of the detrend D{}; <= 0 selects 1e4 (M/1000)^4 */
  double als_p;         /* ALS asymmetry (weight of points above the baseline), 0 < p < 1 */
  int32_t als_iters;    /* ALS reweighting iterations (>= 1) */
  double ridge_rel;     /* lambda of Eq. PEC_Ridge = ridge_rel * ||U_ss S||_F^2 / k (>= 0) */
  int32_t sec_mode;     /* FKK_SEC_SAVGOL or FKK_SEC_MEAN (trendline M{} of Eq. fSEC_VT) */
  int32_t sg_window;    /* odd Savitzky-Golay window <= M; 0 = largest odd <= M/2 */
  int32_t sg_order;     /* Savitzky-Golay polynomial order, < window, <= 7 */
  double ml_lambda;     /* ridge lambda of Eq. ML_Unew used by fkk_apply (>= 0) */
  int32_t precision;    /* FKK_PREC_BF16X3 or FKK_PREC_BF16: arithmetic of fkk_apply with the basis */
  float ratio_floor;    /* I/I_ref is clamped to >= ratio_floor before the log (> 0) */
  double noise_alpha;   /* Poisson multiplier alpha of f(w) (Sec. 2.2); used when f is NULL */
  double noise_sigma_g; /* Gaussian sigma_g of f(w); alpha = sigma_g = 0 means f = 1 */
  int32_t k_max;        /* k = 0: upper bound of the chosen k, 1..80 */
  double rank_eps;      /* k = 0: the epsilon of the rank rule (> 0); 0 = FLT_EPSILON, the input's */
  int32_t svd;          /* FKK_SVD_EXACT or FKK_SVD_RANDOMIZED (the right singular vectors' source) */
  int32_t rsvd_oversample;   /* randomised: l = k + oversample test vectors (l <= 80) */
  int32_t rsvd_power_iters;  /* randomised: subspace iterations, 0..20 */
  uint64_t rsvd_seed;        /* randomised: key of the Philox4x64-10 test matrix */
  int32_t denoise_k;    /* conventional_per_spectrum only: 0 no denoising; > 0 (<= 80) keep that many
                           singular vectors of the raw spectra; < 0 the rank rule (at most k_max) */
  int32_t refine_steps; /* FKK_SVD_EXACT: refinement steps on the kept basis after the eigensolve, 0..4
                           (see fkk_refine_basis); the randomised SVD refines through rsvd_power_iters */
} fkk_fit_params;

/* How fkk_fit_basis finds V_k and s:
 *   FKK_SVD_EXACT      the k largest eigenpairs of A^T A (tensor-core Gram,
 *                      double-word tridiagonal eigensolver);
 *   FKK_SVD_RANDOMIZED randomised subspace iteration (the randomised SVD
 *                      Sec. 5 proposes; Halko, Martinsson & Tropp 2011):
 *                      Omega (M x l) Gaussian, entry e from Philox4x64-10 at
 *                      counter (e/2, 0, 0, 0), key (rsvd_seed, 0), Box-Muller
 *                      cos/sin of u = ((w >> 11) + 1/2) 2^-53 of words 0, 1;
 *                      Y = A Omega; rsvd_power_iters times Q = orth(Y),
 *                      Z = orth(A^T Q), Y = A Z; Q = orth(Y); B = Q^T A;
 *                      V = B^T U S^-1 from B B^T = U S^2 U^T.  It reads the
 *                      cube 2 (power_iters + 1) times instead of forming
 *                      A^T A, and needs k >= 1. */
enum { FKK_SVD_EXACT = 0, FKK_SVD_RANDOMIZED = 1 };

/* Refinement of a kept basis of the eigensolve (Sec. 2.2 needs V and S of
 * the SVD of A; this makes a computed V_k more accurate): `steps` (1..4)
 * times, Q = orth(G V) = orth(A^T (A V)) by Cholesky QR, then the
 * Rayleigh-Ritz pairs of G on span(Q): Q^T G Q = U diag(mu) U^T, V = Q U,
 * lambda = mu.  g: m x m symmetric fp64, row-major (device); v: m x k fp64,
 * row-major (device); lam_out: k (device), descending; v_out: m x k
 * (device, may be v), each column's largest-magnitude component positive.
 * fp64 throughout.  Exact eigenvectors come back unchanged up to rounding;
 * the error of an approximate basis shrinks about as lambda_{k+1} /
 * lambda_k per step.  2 <= m <= 2048, 1 <= k <= min(m, 80); otherwise
 * FKK_ERR_INVALID_ARG.  Asynchronous on `stream`; device-side failures
 * (a singular Q^T Q) show in fkk_sync_status.  fkk_fit_basis runs it when
 * params.refine_steps > 0 (exact SVD). */
fkk_status fkk_refine_basis(fkk_ctx* ctx, const double* g, int32_t m, int32_t k, const double* v, int32_t steps,
                            double* lam_out, double* v_out, void* stream);

/* The randomised SVD's test-matrix entries 0..count-1 for `seed` (as
 * described above), written as doubles to the device array out.
 * Asynchronous on `stream`. */
fkk_status fkk_philox_normals(fkk_ctx* ctx, int64_t count, uint64_t seed, double* out, void* stream);

/* Defaults: k 20, pad_len 0, pec 1, sec 1, als_lambda 0 (auto), als_p 0.01,
 * als_iters 20, ridge_rel 1e-3, sec_mode SAVGOL, sg_window 0 (auto),
 * sg_order 2, ml_lambda 0, precision BF16X3, ratio_floor 1e-6, noise 0/0,
 * k_max 80, rank_eps 0 (FLT_EPSILON), svd EXACT, rsvd_oversample 10,
 * rsvd_power_iters 2, rsvd_seed 0, denoise_k 0, refine_steps 0.
 *
 * k = 0 selects the number of basis vectors by the rank rule of Sec. 4.1:
 * the count of singular values s_i > s_1 * max(N, M) * rank_eps (the NumPy /
 * MATLAB rank cutoff), computed from the k_max largest, at least 1.  The fit
 * then reads k_max eigenvalues back to the host once (a synchronisation of
 * `stream`), and the basis holds the chosen k (fkk_basis_info). */
void fkk_fit_params_default(fkk_fit_params* p);

/* Trained artefacts (Sec. 2.6: f, S, V, Phi_PEC, V_SEC) resident on the
 * context's device.  Owned by the caller; release with fkk_basis_free. */
typedef struct fkk_basis fkk_basis;

/* Fit fKK-EC on a cube and optionally reconstruct it (Eq. fKKEC).
 *   A   = f(w) * 1/2 ln(max(I_CARS/I_ref, floor))       (Sec. 2.2, scaled A)
 *   A^T A = V diag(lambda) V^T (tridiagonal eigensolve); s = sqrt(lambda_1..k);
 *   P   = A V_k = U S;   q = argmax / argmin rows of each column of P
 *   fKK: B = V^T/f, H{B};  fPEC: Eq. phi_err_USphi_b + Eq. PEC_Ridge;
 *   fSEC: Eq. fSEC_VT;  Im{K} = exp(P C_amp) sin(P C_ph).
 * i_cars: n_spectra x n_channels floats (stride ld); i_ref: n_channels floats;
 * f_or_null: n_channels floats (f(w)), or NULL to use params->noise_* (both
 * 0 means f = 1).  n_channels in [8, 2048]; 1 <= k <= min(80, n_channels);
 * n_spectra >= k.  *out_basis receives the trained basis (required).
 * im_out_or_null / re_out_or_null: n_spectra x n_channels outputs (stride
 * ld_out) or NULL to skip the reconstruction.  Enqueued on `stream`;
 * eigensolver non-convergence is reported by fkk_sync_status.
 * i_cars, i_ref, f_or_null and the outputs may be device or host memory
 * (pinned or pageable): host inputs are copied into the context's workspace
 * on `stream` before the transform and host outputs copied back after the
 * reconstruction (pinned: asynchronously on `stream`, so pinned inputs must
 * stay unchanged and pinned outputs unread until `stream` has reached the
 * end of the call; pageable: before the call returns).  im_out and re_out
 * must be of the same kind.  Fits on different streams run concurrently
 * only with one context per stream (each context owns its workspace). */
fkk_status fkk_fit_basis(fkk_ctx* ctx, const float* i_cars, int64_t n_spectra, int32_t n_channels, int64_t ld,
                         const float* i_ref, const float* f_or_null, const fkk_fit_params* params,
                         fkk_basis** out_basis, float* im_out_or_null, float* re_out_or_null, int64_t ld_out,
                         void* stream);

/* One cube of fkk_fit_many: the arguments of fkk_fit_basis for one image
 * (arrays device or host as there), with its own parameters. */
typedef struct {
  const float* i_cars;
  int64_t n_spectra;
  int32_t n_channels;
  int64_t ld;
  const float* i_ref;
  const float* f_or_null;
  float* im_out;   /* may be NULL (no reconstruction) */
  float* re_out;   /* may be NULL */
  int64_t ld_out;
  fkk_fit_params params;
} fkk_cube_job;

/* Fit many independent cubes (images of different sizes, channel counts and
 * k; Fig. 1(b) on each) in one call: out_bases[i] receives job i's basis,
 * exactly as fkk_fit_basis would produce it.  The jobs run, largest first,
 * on two worker lanes -- contexts of their own with their own streams and
 * workspaces (each capped at half of ctx's budget), kept on ctx for later
 * calls -- so the stages of different cubes overlap on the device.  The
 * lanes start after the work already on `stream`; `stream` waits for both
 * at the end, and the lanes' device status (clamp counts, eigensolver
 * failures) is added to ctx's (fkk_sync_status).  On an argument or CUDA
 * error every basis made so far is freed and out_bases is all NULL. */
fkk_status fkk_fit_many(fkk_ctx* ctx, int32_t n_jobs, const fkk_cube_job* jobs, fkk_basis** out_bases, void* stream);

/* ML:fKK-EC (Sec. 2.6): U_new S = A_new V diag(s^2/(s^2+ml_lambda)) with the
 * basis's f, I_ref and ratio floor (Eq. ML_Unew), then Eq. fKKEC with the
 * trained C_amp, C_ph.  i_cars has basis n_channels columns.  re_out may be
 * NULL.  With row strides that are multiples of 4 floats, 16-byte aligned
 * device arrays and k <= 62 this is one launch that reads I once and writes
 * Im (and Re) once, in the basis' precision; otherwise a projection kernel
 * and the reconstruction (fp32-accurate).  The first call packs the basis'
 * operands on the device (a synchronisation of `stream`).  Errors:
 * FKK_ERR_INVALID_ARG, FKK_ERR_BUDGET, FKK_ERR_CUDA. */
fkk_status fkk_apply(fkk_ctx* ctx, const fkk_basis* basis, const float* i_cars, int64_t n_spectra, int64_t ld,
                     float* im_out, float* re_out, int64_t ld_out, void* stream);

/* Residual fraction of spectra on a trained basis -- whether the basis still
 * supports new data (Sec. 1: readily testable; Sec. 5: retrain when it does
 * not):  A = f * 1/2 ln(max(I/I_ref, floor)) with the basis' f, I_ref and
 * floor, and
 *   frac = ||A - A V V^T||_F^2 / ||A||_F^2 = 1 - ||A V||_F^2 / ||A||_F^2
 * over the n spectra (V_k orthonormal).  On the training cube this equals
 * 1 - sum(lambda_1..k) / energy (FKK_ART_ENERGY); a value well above that on
 * new data means the data hold components the basis lacks.  Synchronises
 * `stream`; *frac_out is written on the host. */
fkk_status fkk_residual(fkk_ctx* ctx, const fkk_basis* basis, const float* i_cars, int64_t n_spectra, int64_t ld,
                        double* frac_out, void* stream);

/* Build a basis from HOST arrays (doubles): f (M), s (k), V (M x k), C_amp
 * and C_ph (k x M), I_ref (M).  params supplies k, pad_len, ratio_floor and
 * ml_lambda.  The arrays are copied; the call is synchronous. */
fkk_status fkk_basis_from_arrays(fkk_ctx* ctx, int32_t n_channels, const fkk_fit_params* params, const double* f,
                                 const double* s, const double* v, const double* c_amp, const double* c_ph,
                                 const double* i_ref, fkk_basis** out_basis);

/* sizeof(fkk_fit_params) as compiled into the library (ABI check). */
size_t fkk_fit_params_size(void);

/* Set the per-channel offset (n_channels doubles, HOST memory) that
 * fkk_apply subtracts from the log ratios before rounding them to bf16 and
 * adds back exactly through the reconstruction (the results are the same
 * up to rounding for any offset; the closer it is to typical spectra, the
 * smaller the rounding error of the reduced-precision form).  fkk_fit_basis
 * stores the training mean of 1/2 ln max(I/I_ref, floor); a basis built by
 * fkk_basis_from_arrays starts with 0.  Synchronises the basis' device.
 * Errors: FKK_ERR_INVALID_ARG, FKK_ERR_CUDA. */
fkk_status fkk_basis_set_offset(fkk_basis* basis, const double* offset, int32_t n_channels);

/* Set the precision (FKK_PREC_BF16X3 or FKK_PREC_BF16) that fkk_apply and
 * the serving loop use with this basis; the trained arrays are unchanged,
 * so one basis can be served in either form (Sec. 2.6 reuses it as is).
 * Not to be called while work on the basis is queued.  Errors:
 * FKK_ERR_INVALID_ARG. */
fkk_status fkk_basis_set_precision(fkk_basis* basis, int32_t precision);

/* Release a basis (NULL is ok).  Synchronises the basis's device. */
void fkk_basis_free(fkk_basis* basis);

/* Shape of a basis.  Any output pointer may be NULL.  *nq (the number of
 * sub-sampled rows of Eq. q_max/q_min) needs the fit to have completed and
 * synchronises the device. */
fkk_status fkk_basis_info(const fkk_basis* basis, int32_t* n_channels, int32_t* k, int32_t* pad_len, int32_t* nq);

/* Copy one trained artefact to HOST memory as doubles (synchronous).
 * which / element count:
 *   FKK_ART_S        k        singular values s
 *   FKK_ART_LAMBDA   k        eigenvalues of A^T A
 *   FKK_ART_V        M*k      V_k, row-major M x k
 *   FKK_ART_F        M        f(w)
 *   FKK_ART_B, FKK_ART_H_B, FKK_ART_PHI_PEC, FKK_ART_H_PHI, FKK_ART_V_SEC,
 *   FKK_ART_C_AMP, FKK_ART_C_PH      k*M each, row-major k x M
 *   FKK_ART_Q        nq       sub-sampled row indices (sorted)
 *   FKK_ART_ENERGY   1        ||A||_F^2 = trace(A^T A) of the training cube, so
 *                             that 1 - sum(lambda) / energy is the training
 *                             residual fraction (compare fkk_residual)
 * `count` must equal the element count. */
enum {
  FKK_ART_S = 0, FKK_ART_LAMBDA, FKK_ART_V, FKK_ART_F, FKK_ART_B, FKK_ART_H_B, FKK_ART_PHI_PEC,
  FKK_ART_H_PHI, FKK_ART_V_SEC, FKK_ART_C_AMP, FKK_ART_C_PH, FKK_ART_Q, FKK_ART_ENERGY
};
fkk_status fkk_basis_get(const fkk_basis* basis, int32_t which, double* host_dst, size_t count);

/* ------------------------------------------------------------------ */
/* Conventional workflow: per-spectrum KK, PEC and SEC (Sec. 2.1)       */
/* ------------------------------------------------------------------ */

/* The conventional per-spectrum workflow of Fig. 1(a), Eq. KCARS_from_K.
 * With params->denoise_k != 0 the raw spectra X (n_spectra x n_channels)
 * are first replaced by their truncated SVD (the workflow's denoising step;
 * Sec. 2.2: drop the singular vectors that carry noise):
 *   X^T X = V diag(lambda) V^T (tensor-core Gram of X - c with c the mean
 *             of the first 256 rows, exact in its shift; the double-word
 *             eigensolver of fkk_fit_basis),
 *   X_k     = (X V_k) V_k^T, k = denoise_k, or for denoise_k < 0 the rank
 *             rule of fkk_fit_basis (s_i > s_1 max(N, M) rank_eps, at most
 *             k_max) -- a synchronisation of `stream`.
 * It holds the n_spectra x n_channels denoised cube and the transformed
 * cube (4 bytes per element) in the context's workspace.  Then, for every
 * spectrum n:
 *   a       = 1/2 ln max(I_CARS[n,:] / I_ref, ratio_floor),  phi = H{a}
 *             (the discrete Hilbert transform of kk_per_spectrum)
 *   phi_err = D{phi} if params->pec, else 0: the asymmetric least squares
 *             baseline (second-difference penalty als_lambda, asymmetry
 *             als_p, als_iters reweightings, weights starting at 1) -- the
 *             same detrending operator fPEC uses
 *   K_pec   = exp(a + H{phi_err}) exp(i (phi - phi_err))
 *   K_CARS  = K_pec / M{Re K_pec} if params->sec, else K_pec; M is the
 *             Savitzky-Golay trendline (sg_window, sg_order <= 2; the
 *             polynomial of the first / last full window near the edges) or
 *             the mean over the channels (sec_mode FKK_SEC_MEAN)
 * im_out (required) and re_out (may be NULL) receive Im and Re K_CARS.
 * Uses pad_len (power of two in [M, 4096]; 0 = nextpow2(2M)), pec, sec,
 * als_*, sec_mode, sg_window, sg_order, ratio_floor, denoise_k, k_max and
 * rank_eps of *params; the other fields are ignored.  n_channels in
 * [8, 2048]; denoise_k <= min(80, n_channels, n_spectra).  Device arrays,
 * row-major, row strides ld / ld_out.  Works in chunks of spectra inside a
 * context workspace of about 32 M bytes per spectrum of a chunk (a chunk is
 * halved until it fits the context's budget).  Clamped ratios are counted
 * as by kk_per_spectrum.  Asynchronous on `stream` (but see denoise_k < 0). */
fkk_status conventional_per_spectrum(fkk_ctx* ctx, const float* i_cars, int64_t n_spectra, int32_t n_channels,
                                     int64_t ld, const float* i_ref, const fkk_fit_params* params, float* im_out,
                                     float* re_out, int64_t ld_out, void* stream);

/* ------------------------------------------------------------------ */
/* Pipeline steps, exposed for composition and step-by-step checking    */
/* ------------------------------------------------------------------ */

/* G = A^T A (fp64, n_channels x n_channels, row-major, device) with
 * A = f * 1/2 ln(max(I/I_ref, floor)); f_or_null: device doubles or NULL. */
fkk_status fkk_gram(fkk_ctx* ctx, const float* i_cars, int64_t n_spectra, int32_t n_channels, int64_t ld,
                    const float* i_ref, float ratio_floor, const double* f_or_null, double* g_out, void* stream);

/* Top-k eigenpairs of the symmetric fp64 G (device, m x m): lam_out (k,
 * descending), v_out (m x k row-major), each column's largest-magnitude
 * entry positive.  m in [2, 2048], 1 <= k <= min(80, m).  Householder
 * tridiagonalisation, Sturm multisection and twisted-factorisation
 * eigenvectors in double-word (about 48-bit) arithmetic; eigenvalues and
 * residuals accurate to about 1e-13 of the largest eigenvalue.  Errors:
 * FKK_ERR_INVALID_ARG, FKK_ERR_CUDA; a numerical breakdown (non-finite
 * input) is reported by fkk_sync_status as FKK_ERR_NOT_CONVERGED. */
fkk_status fkk_eig_topk(fkk_ctx* ctx, const double* g, int32_t m, int32_t k, double* lam_out, double* v_out,
                        void* stream);

/* P = A W (n x k fp32, row-major, device) for A as in fkk_gram and W
 * (device, m x k doubles), through the same transformed-cube path as the
 * fit; qmax/qmin (device int64, k each, or NULL) receive the argmax /
 * argmin row of each column of P (ties to the lowest row). */
fkk_status fkk_project(fkk_ctx* ctx, const float* i_cars, int64_t n_spectra, int32_t n_channels, int64_t ld,
                       const float* i_ref, float ratio_floor, const double* f_or_null, const double* w, int32_t k,
                       float* p_out, int64_t* qmax, int64_t* qmin, void* stream);

/* fKK / fPEC / fSEC on the basis (device doubles): v (m x k), f_or_null (m),
 * x_rows (nq x k, the rows P_q = U_ss S).  Outputs c_amp, c_ph (k x m). */
fkk_status fkk_basis_math(fkk_ctx* ctx, int32_t m, int32_t k, const double* v, const double* f_or_null,
                          const double* x_rows, int32_t nq, const fkk_fit_params* params, double* c_amp,
                          double* c_ph, void* stream);

/* Eq. fKKEC from P (n x k fp32) and C_amp, C_ph (k x m fp64): im_out (and
 * re_out unless NULL) n x m with stride ld_out. */
fkk_status fkk_reconstruct(fkk_ctx* ctx, const float* p, int64_t n_spectra, int32_t k, int32_t m,
                           const double* c_amp, const double* c_ph, float* im_out, float* re_out, int64_t ld_out,
                           void* stream);

/* ------------------------------------------------------------------ */
/* Trained-basis files, the noise model, and serving (Sec. 2.6)         */
/* ------------------------------------------------------------------ */

/* Write the basis (all trained arrays: f, S, V, W, B, H_B, Phi_PEC, H_Phi,
 * V_SEC, C_amp, C_ph, q, I_ref, and the fit parameters) to a file: a
 * header with format version, sizes and an FNV-1a checksum of the data.
 * Errors: FKK_ERR_INVALID_ARG, FKK_ERR_CUDA, FKK_ERR_BAD_FILE (cannot
 * write). */
fkk_status fkk_basis_save(const fkk_basis* basis, const char* path);

/* Read a file written by fkk_basis_save into a new basis on ctx's device
 * (owned by the caller, release with fkk_basis_free).  A file with another
 * magic, version or parameter layout, inconsistent sizes, truncated data or
 * a wrong checksum gives FKK_ERR_BAD_FILE and no basis. */
fkk_status fkk_basis_load(fkk_ctx* ctx, const char* path, fkk_basis** out);

/* f(w) of the noise model (Sec. 2.2): f = 2 <I> / sqrt(alpha <I> +
 * sigma_g^2) per channel, from the mean spectrum <I> (device floats,
 * n_channels) into f_out (device doubles); pass f to fkk_fit_basis as the
 * f_or_null weights (after conversion to float) when fitting with a
 * precomputed noise model.  alpha, sigma_g >= 0, not both 0. */
fkk_status fkk_noise_scale(fkk_ctx* ctx, const float* mean_spectrum, int32_t n_channels, double alpha,
                           double sigma_g, double* f_out, void* stream);

/* Serving of a trained basis (Sec. 2.6, Eq. ML_Unew then Eq. fKKEC) with
 * continuous batching.  A server has its own context on the basis' device
 * (same HBM budget as ctx, workspace separate from ctx's), a dispatcher
 * thread and three batch slots; each slot owns a CUDA stream and device
 * staging for `cap` spectra in and out.  cap is the tune cache's max_batch
 * (or 65,536), reduced to what the HBM budget leaves for the three slots.
 * Submitted requests queue in order; the dispatcher moves them into the
 * first free slot -- consecutive host tiles gathered into one batch while
 * their spectra fit the slot (one fused apply for all of them), a device
 * tile alone, in place -- and enqueues the batch (copies in, apply, copies
 * out) on the slot's stream without waiting, so up to three batches are in
 * flight and the copies of one overlap the kernel of another.  The apply of
 * a gathered batch is replayed from a CUDA graph of its slot and
 * 1,024-spectrum bucket; fkk_serve_start captures all of them (slots x
 * staging / 1,024 graphs) before it returns, so no request pays for a
 * capture.  A request waits in the queue while every slot is
 * busy (admission deferred until staging frees up).  The basis must outlive
 * the server and keep its precision while the server runs. */
typedef struct fkk_server fkk_server;
typedef uint64_t fkk_req;

/* tune_cache_or_null: a text file with the lines "max_batch=<spectra>" and
 * "stages=<0..4>" (ring depth of the fused apply, 0 = the deepest that
 * fits).  When the path is given but lacks either entry, an autotuner times
 * the apply at each ring depth and at batch sizes 2,048, 4,096, ..., cap,
 * keeps the fastest depth and the smallest batch within 10 % of the best
 * throughput, and writes both.  Errors: FKK_ERR_INVALID_ARG, FKK_ERR_CUDA,
 * FKK_ERR_BUDGET (the budget leaves no room for 128 spectra per slot). */
fkk_status fkk_serve_start(fkk_ctx* ctx, const fkk_basis* basis, const char* tune_cache_or_null, fkk_server** out);

/* Queue a tile of n_spectra spectra (n_channels of the basis each, rows
 * contiguous) and return its id at once.  tile_on_host = 0: tile and
 * im_out are device pointers; 1: both are pinned host memory.  The buffers
 * belong to the caller and must stay valid until the request is waited.
 * Errors: FKK_ERR_INVALID_ARG, FKK_ERR_SHUTDOWN (server stopping),
 * FKK_ERR_BUDGET (a host tile of more spectra than a slot's staging holds:
 * it can never be admitted; split it). */
fkk_status fkk_serve_submit(fkk_server* server, const float* tile, int64_t n_spectra, int32_t tile_on_host,
                            float* im_out, fkk_req* out_id);

/* Wait for a request: its status (FKK_OK, a CUDA error, or
 * FKK_ERR_SHUTDOWN if the server stopped before it ran), after which the id
 * is released; FKK_ERR_TIMEOUT if it has not completed within timeout_ms
 * (< 0: no limit), the id stays valid; FKK_ERR_INVALID_ARG for an unknown
 * or already released id.  Each request is waited by one thread. */
fkk_status fkk_serve_wait(fkk_server* server, fkk_req id, int32_t timeout_ms);

/* p50 / p99 of submit-to-completion latency over the last 16,384 requests
 * and the throughput (spectra completed per second since the first
 * submit).  Any pointer may be NULL. */
fkk_status fkk_serve_stats(fkk_server* server, double* p50_ms, double* p99_ms, double* spectra_per_s);

/* The last (up to 1,024) completed batches, oldest first, 5 doubles each:
 * start and end in milliseconds (CUDA events recorded on the slot's stream
 * before its first copy and after its last, relative to the server's start),
 * slot index, number of requests, number of spectra.  Writes at most
 * max_rows rows to out (host) and their count to *n_rows. */
fkk_status fkk_serve_batch_log(fkk_server* server, double* out, int32_t max_rows, int32_t* n_rows);

/* Stop: queued requests complete with FKK_ERR_SHUTDOWN, batches already
 * issued finish, threads blocked in fkk_serve_wait return, and the server
 * (its streams, graphs, context and staging) is freed. */
fkk_status fkk_serve_stop(fkk_server* server);

/* Largest problem fkk_reconstruct_noalloc accepts in one call. */
#define FKK_NOALLOC_MAX_SPECTRA 16384
#define FKK_NOALLOC_MAX_CHANNELS 2048

/* fkk_reconstruct_noalloc: the same reconstruction as fkk_reconstruct
 * (Eq. fKKEC; same kernels, same arguments and layout, identical results),
 * but it allocates no device memory.  The paper has no counterpart: this is
 * an interface of this library for callers that cannot allocate, e.g. a
 * serving loop that has fixed its HBM footprint at start-up, or code that
 * must not hit the implicit device synchronisation of cudaMalloc/cudaFree.
 * fkk_reconstruct keeps its packed operands in the context's grow-only
 * workspace, which is (re)allocated the first time a larger batch arrives;
 * this entry point packs them instead into four fixed arrays compiled into
 * the library (bf16 hi and lo parts of P for up to FKK_NOALLOC_MAX_SPECTRA
 * rows at K = 128, and of the interleaved coefficients for up to
 * FKK_NOALLOC_MAX_CHANNELS channels; 10 MiB of static device memory per
 * device).
 *
 * Limits: 0 <= n_spectra <= FKK_NOALLOC_MAX_SPECTRA, 1 <= k <= 80,
 * 1 <= m <= FKK_NOALLOC_MAX_CHANNELS, ld_out >= m; anything larger returns
 * FKK_ERR_INVALID_ARG with a message in fkk_last_error() and launches
 * nothing (split larger batches into calls of at most the maximum).
 * Setup: the first call on a device looks up the addresses of the static
 * arrays (cudaGetSymbolAddress, which may load the library's device code on
 * that device); make that first call before any stream capture.  A call
 * with n_spectra == 0 does only this setup and accepts NULL data pointers.
 * Nothing in the arrays needs to start at zero: every call rewrites the
 * whole region its kernels read (zero padding included).
 * Concurrency: the arrays are shared by every context of the process on
 * that device, so calls whose work overlaps on the device (other streams,
 * other threads or contexts) race on them and give wrong results; order
 * such calls on one stream or with events.  Device-side errors are reported
 * through fkk_sync_status() of ctx as for the other calls.
 * Errors: FKK_ERR_INVALID_ARG, FKK_ERR_CUDA. */
fkk_status fkk_reconstruct_noalloc(fkk_ctx* ctx, const float* p, int64_t n_spectra, int32_t k, int32_t m,
                                   const double* c_amp, const double* c_ph, float* im_out, float* re_out,
                                   int64_t ld_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FKK_H_ */
