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

#ifdef __cplusplus
}
#endif

#endif /* FKK_H_ */
