/*
 * shearlet.h - C ABI of libshearlet, the GB300 (sm_103a) digital shearlet
 * transform after tfShearlab (arXiv 2006.04591).
 *
 * The library exposes the paper's three operations (Sec. 3.4): build the
 * filter bank (``getshearletsystem2D``), decompose (``tfsheardec2D``) and
 * reconstruct (``tfshearrec2D``), plus the adjoint of each transform.  All
 * transform work runs in hand-written CUDA kernels; nothing here falls back to
 * the CPU.
 *
 * Conventions shared by every call
 * --------------------------------
 * Return value: shl_status.  SHL_OK (0) on success; otherwise nothing was
 * launched, or (for SHL_ECUDA) the launch failed, and shl_last_error_detail()
 * gives a thread-local message.  No call aborts, traps or throws.  Kernel
 * faults are asynchronous and surface at the next CUDA call or at
 * shl_sync().
 *
 * Streams: ``stream`` is a cudaStream_t passed as void* (NULL = legacy
 * default stream).  Every launch goes on that stream; no call synchronises.
 *
 * Images: ``rows`` x ``cols`` real float32, row-major, batch-major:
 * x[b][y][x].  rows and cols are in [1, 4096].  Powers of two in
 * [16, 2048] with real spectra run on the half-spectrum kernels; every other
 * size, and every bank with complex spectra, runs on the general kernels
 * (row-major half-spectrum planes, mixed-radix or Bluestein line DFTs; the
 * same results to float32 rounding, at a lower throughput).  Image
 * arguments (x, x_out, f_masked, f_est, mask) may be device memory of the
 * bank's device, managed memory, or pinned host memory mapped into the
 * device's address space (cudaHostAlloc / cudaHostRegister): the first or
 * last kernel of the call then reads or writes the images over the CPU-GPU
 * link, with no separate copy.  Other pointers must be device memory.  A
 * pointer the device cannot dereference gives SHL_EINVAL before any launch.
 *
 * Coefficients: c[b][i][y][x] (batch, filter, row, column), float32 or
 * bfloat16 (round-to-nearest-even on store).  This is the paper's
 * [1, N, M, nShearlets] tensor with the filter axis moved before the image
 * axes (paper coeffs[0, y, x, i] == c[0][i][y][x]), so each subband is one
 * contiguous image.
 *
 * Filters: K spectra G_i in natural DFT order (index 0 = zero frequency),
 * i.e. ifftshift of the conjugated centred ``shearletFilters[i]`` of the
 * paper.  Decomposition multiplies the image spectrum by G_i, reconstruction
 * by conj(G_i) / W with W = sum_i |G_i|^2 (Sec. 3.4).  Real spectra must be
 * even, complex ones Hermitian, G(-k) = conj(G(k)), so that real images have
 * real coefficients.  The shift pairs of the paper cancel at every size:
 * a circular translation commutes with the filtering.
 *
 * Ownership: the library owns a bank (device spectra, 1/W, RMS, indices).
 * The caller owns all image, coefficient, threshold and workspace buffers,
 * which must be device pointers on the bank's device, 16-byte aligned, and
 * must not alias each other.  The hot calls allocate nothing.
 *
 * Concurrency: a bank is immutable after creation; calls with distinct
 * workspaces may run concurrently on different streams.
 */
#ifndef SHEARLET_H
#define SHEARLET_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SHL_ABI_VERSION 1
/* Version of the filter-bank construction (host builder bank_build.cpp and
 * GPU builder bank_gpu.cu, which produce the same spectra).  Raised whenever
 * either changes its output; saved banks keyed on an older value are not
 * reused. */
#define SHL_BANK_BUILDER_VERSION 1

typedef enum {
  SHL_OK = 0,
  SHL_EINVAL = 1,        /* bad argument (null pointer, size, alignment)   */
  SHL_ENOMEM = 2,        /* device or host allocation failed (bank create) */
  SHL_ECUDA = 3,         /* a CUDA runtime call or launch failed           */
  SHL_EUNSUPPORTED = 4,  /* size or option this build does not support     */
  SHL_ETIMEOUT = 5,      /* a bounded device wait gave up                  */
  SHL_EDEVICE = 6        /* a kernel reported an error through its flag    */
} shl_status;

typedef enum { SHL_F32 = 0, SHL_BF16 = 1 } shl_dtype;

/* shl_decompose flags */
#define SHL_DUAL_WEIGHTED 1  /* multiply by G_i / W: adjoint of reconstruct */

/* shl_workspace_size ops */
typedef enum {
  SHL_OP_DECOMPOSE = 0,
  SHL_OP_RECONSTRUCT = 1, /* also shl_adjoint */
  SHL_OP_SHRINK = 2,      /* shl_shrink */
} shl_op;

typedef struct shl_bank shl_bank;

int shl_abi_version(void);
const char* shl_status_str(shl_status s);
/* Thread-local text for the last non-OK status returned on this thread. */
const char* shl_last_error_detail(void);

/*
 * shl_bank_create - build the digital shearlet system (Sec. 2.1, Sec. 3.4
 * ``getshearletsystem2D(rows, cols, nScales, ...)``) in float64 on the host
 * and upload it to ``device``.
 *   n_scales      J >= 1.
 *   shear_levels  J ints (scale 0 = coarsest) or NULL for ceil((j+1)/2).
 *                 Levels must be in [0, 4].
 *   full          0: cone 2 omits the two diagonal shears +-2^l (17/33/49
 *                 filters for 2/3/4 scales, Eq. 3.2); 1: keeps them.
 *   out           receives the bank; release with shl_bank_destroy.
 * Filters: 1D maximally flat low-pass h (9 taps, 3 dB at pi/2) and its
 * mirror g, iterated filters h_j / g_j, McClellan fan filter P, digital
 * shear of Eqs. 2.4-2.5.  Order: 0 = low-pass, then per scale (coarse to
 * fine) cone 1 with shear k ascending, then cone 2 with k ascending.
 * rows, cols in [1, 4096] (the float64 line DFTs of the construction use
 * Bluestein's algorithm at lengths that are not powers of two).
 * device < 0 builds a host-only bank: shl_bank_query / shl_bank_copy_info
 * work (no GPU needed), transform calls return SHL_EINVAL.
 * Errors: SHL_EUNSUPPORTED for sizes outside [1, 4096], SHL_EINVAL for bad
 * levels, SHL_ENOMEM, SHL_ECUDA.
 */
shl_status shl_bank_create(int rows, int cols, int n_scales, const int* shear_levels,
                           int full, int device, shl_bank** out);

/*
 * shl_bank_create_gpu - shl_bank_create with the construction on `device`
 * (float64 throughout: one CTA per filter column builds the column spectrum,
 * its inverse DFT along w2, the digital-shear multiplier of Eqs. 2.4-2.5 and
 * the forward DFT; then the even part, W, RMS and the float32 tables).  The
 * result is the bank shl_bank_create builds, to float64 rounding (the host
 * copies read by shl_bank_copy_info are downloaded).  The paper times this
 * construction as its first experiment (filters on the GPU vs the CPU).
 * rows and cols powers of two in [16, 2048] (else SHL_EUNSUPPORTED; build
 * other sizes with shl_bank_create); device >= 0; errors as shl_bank_create.
 */
shl_status shl_bank_create_gpu(int rows, int cols, int n_scales, const int* shear_levels,
                               int full, int device, shl_bank** out);

/*
 * shl_bank_create_from_spectra - use caller-supplied spectra (Sec. 3.4: any
 * filter tensor ``tfshearlets`` of shape [1, N, M, K]).
 *   spectra  host float64 [K][rows][cols], natural order, real.  Each must
 *            be even, G(-k) == G(k), to 1e-9 of its max |G|, and the dual
 *            weights W = sum_i G_i^2 must be > 0 everywhere, else SHL_EINVAL.
 *   idx      host int [K][3] (cone, scale, shear) copied for reference, or
 *            NULL (all zeros).
 * rows, cols in [1, 4096] (SHL_EUNSUPPORTED otherwise).
 * RMS_i = sqrt(sum G_i^2 / (rows cols)) is computed in float64.
 * device < 0 builds a host-only bank as for shl_bank_create.
 */
shl_status shl_bank_create_from_spectra(int rows, int cols, int K, const double* spectra,
                                        const int* idx, int device, shl_bank** out);

/*
 * shl_bank_create_general - a bank that always runs on the general kernels,
 * with real or complex spectra (Sec. 3.4 allows complex filter tensors; the
 * paper's listings keep complex64 spectra).
 *   spectra_re, spectra_im  host float64 [K][rows][cols], natural order;
 *            spectra_im NULL for real spectra.  Complex spectra must be
 *            Hermitian, G(-k) == conj(G(k)), real ones even, to 1e-9 of the
 *            largest |G|; W = sum_i |G_i|^2 > 0 everywhere; else SHL_EINVAL.
 *   idx      as for shl_bank_create_from_spectra.
 * rows, cols in [1, 4096].  The decomposition computes
 * c_i = IDFT2(G_i DFT2 x) (real by Hermitian symmetry), the reconstruction
 * IDFT2(sum_i conj(G_i) DFT2 c_i / W), the adjoints as for real banks.
 * device < 0 builds a host-only bank.
 */
shl_status shl_bank_create_general(int rows, int cols, int K, const double* spectra_re,
                                   const double* spectra_im, const int* idx, int device,
                                   shl_bank** out);

shl_status shl_bank_destroy(shl_bank* bank);

/* Number of filters and image size of a bank. Any out pointer may be NULL. */
shl_status shl_bank_query(const shl_bank* bank, int* K, int* rows, int* cols);

/*
 * shl_bank_copy_info - copy host-side float64 data of a bank (Sec. 3.4: the
 * system's filters, its RMS array and its index array; and the dual frame
 * weights ``tfdualFrameWeights``).  Any out pointer may be NULL.
 *   idx [K][3], rms [K], spectra [K][rows][cols] natural order (the real
 *   parts for a complex bank), dual_w [rows][cols] natural order
 *   (W = sum_i |G_i|^2).
 */
shl_status shl_bank_copy_info(const shl_bank* bank, int* idx, double* rms, double* spectra,
                              double* dual_w);

/* Imaginary parts [K][rows][cols] of the spectra (zeros for a real bank). */
shl_status shl_bank_copy_spectra_imag(const shl_bank* bank, double* imag);

/* *general = 1 when the bank runs on the general kernels, 0 on the
 * power-of-two half-spectrum kernels. */
shl_status shl_bank_path(const shl_bank* bank, int* general);

/*
 * shl_workspace_size - bytes of device workspace ``op`` needs for ``batch``
 * images.  The workspace holds the image spectra (decompose) or the
 * per-image accumulators (reconstruct / adjoint) plus a staging area for
 * per-subband intermediates: up to 1 GiB of staging (e.g. all 784
 * subbands of 16 images at 512 x 512 with 49 filters).  A plane is
 * rows * (cols/2 + 1) complex float32 on both paths.  With the environment
 * variable SHL_PIPE=1 the power-of-two decomposition at rows = 512, cols in
 * {512, 1024} runs pipelined and stages 24 planes plus a few counters per 8
 * subbands instead.  Its contents on entry are ignored.
 */
shl_status shl_workspace_size(const shl_bank* bank, shl_op op, int batch, size_t* bytes);

/*
 * shl_decompose - shearlet decomposition (Sec. 3.4, Alg. "Shearlet
 * Decomposition" and the ``tfsheardec2D`` listing):
 *   c[b][i] = IFFT2( G_i * FFT2(x[b]) )         flags = 0
 *   c[b][i] = IFFT2( G_i / W * FFT2(x[b]) )     flags = SHL_DUAL_WEIGHTED
 * (the second is the adjoint of shl_reconstruct).  IFFT2 includes 1/(rows
 * cols).  The Fourier shifts of the paper cancel for even sizes and are not
 * performed.  Coefficients are real.
 *   x       device float32 [batch][rows][cols].
 *   coeffs  device [batch][K][rows][cols] of dtype (SHL_F32 / SHL_BF16).
 *   ws      device workspace of >= shl_workspace_size(DECOMPOSE) bytes.
 * batch == 0 is a no-op.
 */
shl_status shl_decompose(const shl_bank* bank, const float* x, int batch, void* coeffs,
                         shl_dtype dtype, int flags, void* ws, size_t ws_bytes, void* stream);

/*
 * shl_decompose_noalloc - shl_decompose without a caller-provided workspace
 * (the paper has no counterpart; this is a deployment convenience).
 * For callers that cannot allocate device memory when they call: a host
 * framework that owns all device memory and offers plug-ins no allocator, a
 * latency-critical loop that cannot afford cudaMalloc's implicit device
 * synchronisation, or a service at its memory budget that must not fail
 * with out-of-memory at call time.
 *   Scratch: a fixed array of SHL_NOALLOC_SCRATCH_BYTES compiled into the
 *   library, which every GPU that loads the library holds until the process
 *   exits.  The call allocates nothing (no cudaMalloc or cudaFree).
 *   Limit: the image spectra of the batch plus one subband plane must fit,
 *   (batch + 1) * rows * (cols/2 + 1) * 8 bytes <= SHL_NOALLOC_SCRATCH_BYTES
 *   (e.g. batch <= 30 at 512 x 512); larger batches return SHL_EINVAL with a
 *   message - use shl_decompose with your own workspace instead.
 *   Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before capturing any stream work that uses this entry point.
 *   Sharing: all calls on a device share the one array, and it keeps whatever
 *   the last call left there (nothing needs to start at zero).  Calls whose
 *   kernels overlap on the GPU - on different streams, or from different
 *   threads without ordering - race on it and give wrong results; order them
 *   on one stream.
 * Other arguments and the result are exactly those of shl_decompose.
 */
#define SHL_NOALLOC_SCRATCH_BYTES (32u << 20)
shl_status shl_decompose_noalloc(const shl_bank* bank, const float* x, int batch, void* coeffs,
                                 shl_dtype dtype, int flags, void* stream);

/*
 * shl_decompose_masked - decomposition of u = mask * (f_masked - f_est) +
 * f_est, the input of one step of the inpainting iteration (Sec. 4.3, Alg.
 * "Shearlet inpainting by iterative hard thresholding"), with u formed while
 * the images are loaded.
 *   f_masked, f_est  device float32 [batch][rows][cols];
 *   mask             device uint8 [batch][rows][cols], nonzero = observed.
 * Other arguments as shl_decompose (flags must be 0).
 */
shl_status shl_decompose_masked(const shl_bank* bank, const float* f_masked,
                                const unsigned char* mask, const float* f_est, int batch,
                                void* coeffs, shl_dtype dtype, void* ws, size_t ws_bytes,
                                void* stream);

/*
 * shl_reconstruct - shearlet reconstruction (Sec. 3.4, Alg. "Shearlet
 * reconstruction" and the ``tfshearrec2D`` listing; Eq. 2.7):
 *   x[b] = IFFT2( (1/W) * sum_{i=0..K-1} G_i * FFT2(T(c[b][i])) )
 * summed in float32 in a fixed order (the same bits on every run).  T is the hard
 * threshold of Sec. 4.2 applied while the coefficients are read: an entry
 * with |c| < thresh[b][i] becomes 0 (ties are kept).
 *   coeffs  device [batch][K][rows][cols] of dtype.
 *   thresh  device float32 [batch][K], or NULL for no thresholding.
 *   x_out   device float32 [batch][rows][cols].
 *   ws      device workspace of >= shl_workspace_size(RECONSTRUCT) bytes.
 */
shl_status shl_reconstruct(const shl_bank* bank, const void* coeffs, shl_dtype dtype, int batch,
                           const float* thresh, float* x_out, void* ws, size_t ws_bytes,
                           void* stream);

/*
 * shl_adjoint - adjoint of shl_decompose: shl_reconstruct without 1/W,
 *   x[b] = IFFT2( sum_i G_i * FFT2(T(c[b][i])) ).
 * Arguments as shl_reconstruct.
 */
shl_status shl_adjoint(const shl_bank* bank, const void* coeffs, shl_dtype dtype, int batch,
                       const float* thresh, float* x_out, void* ws, size_t ws_bytes,
                       void* stream);

/*
 * shl_shrink - one hard-threshold step of denoising (Sec. 4.2) or of the
 * inpainting iteration (Sec. 4.3, Alg. "Shearlet inpainting by iterative
 * hard thresholding") without storing coefficients:
 *   x_out[b] = IFFT2( (1/W) sum_i G_i FFT2( T_b,i( IFFT2( G_i FFT2(u[b]) ) ) ) )
 *   u = x                                 (mask == NULL; f_est ignored)
 *   u = mask * (x - f_est) + f_est        (mask != NULL: x = f_masked)
 * T_b,i zeroes coefficients with |c| < thresh[b][i] (ties kept).  The
 * coefficients live only in registers: each staged half-spectrum row tile
 * is inverse-transformed, thresholded and transformed back in place, so
 * the result equals shl_decompose (float32) followed by
 * shl_reconstruct(thresh) while moving ~2/3 of their DRAM bytes.
 *   x, f_est  device float32 [batch][rows][cols]; mask device uint8 or NULL.
 *   thresh    device float32 [batch][K].
 *   x_out     device float32 [batch][rows][cols]; may alias x or f_est.
 *   ws        device workspace of >= shl_workspace_size(SHRINK) bytes.
 */
shl_status shl_shrink(const shl_bank* bank, const float* x, const unsigned char* mask,
                      const float* f_est, int batch, const float* thresh, float* x_out, void* ws,
                      size_t ws_bytes, void* stream);

/*
 * shl_subband_absmax - out[b][i] = max_{y,x} |c[b][i][y][x]| / scale_i with
 * scale_i = RMS_i when by_rms != 0, else 1.  Used for the inpainting
 * threshold start value delta_init = max_{i,n} |c_i(n)| / RMS_i (Sec. 4.3).
 *   out  device float32 [batch][K].
 */
shl_status shl_subband_absmax(const shl_bank* bank, const void* coeffs, shl_dtype dtype,
                              int batch, int by_rms, float* out, void* stream);

/*
 * shl_iht_thresholds - the threshold schedule of the inpainting iteration
 * (Sec. 4.3, Alg. "Shearlet inpainting by iterative hard thresholding"), on
 * the device so that no host read sits between the start value and the loop:
 *   delta_0[b] = max_i absmax_by_rms[b][i]          (shl_subband_absmax, by_rms)
 *   out[t][b][i] = delta_0[b] * lambda_b^t * RMS_i,  t = 0 .. iterations-1,
 *   lambda_b = (delta_min / delta_0[b])^(1 / (iterations - 1))  (1 for one
 *   iteration or delta_0 = 0), computed in float64 and rounded to float32.
 * The printed decay delta_min^(1/(T-1)) reaches delta_min only for
 * delta_0 = 1; the ratio above is that rule for any start value.
 *   absmax_by_rms  device float32 [batch][K];  out  device float32
 *   [iterations][batch][K].  delta_min > 0, else SHL_EINVAL.
 */
shl_status shl_iht_thresholds(const shl_bank* bank, const float* absmax_by_rms, int batch,
                              int iterations, double delta_min, float* out, void* stream);

/*
 * Launch accounting (no counterpart in the paper; instrumentation for
 * measurement).  shl_launch_count returns the number of kernels this
 * process's library calls have launched.  While shl_profile_enable(1) is in
 * effect every launch is bracketed by CUDA events recorded on its stream;
 * shl_profile_read waits for them and writes a JSON object
 * {"kernel": {"launches": n, "ms": total}, ...} into buf (len bytes) and
 * clears the records.  SHL_EINVAL if buf is too small (output truncated).
 */
long long shl_launch_count(void);
shl_status shl_profile_enable(int on);
shl_status shl_profile_read(char* buf, size_t len);

/* Wait for all work on ``stream``; returns SHL_ECUDA with the CUDA error text
 * if a kernel faulted, and SHL_ETIMEOUT if a bounded device wait ran out
 * since the last shl_sync on this device: inside the pipelined
 * decomposition (between its column and row passes, Sec. 3.4), or a row
 * pass waiting for the bulk copy of an input tile; the results of that
 * call are then incomplete.  The flag is per device (the stream's device),
 * is cleared only here, and while it is set every later pipelined
 * decomposition on that device stops at once and leaves its coefficients
 * incomplete: call shl_sync after such a call before the next one. */
shl_status shl_sync(void* stream);

/*
 * Checked build (a build step, not the paper's method): libshearlet_checked.so
 * is the same library compiled with -DSHL_CHECKED, in which every global
 * access of the power-of-two transform kernels first compares its index with
 * the extent of its buffer as the launch's sizes give it.  An index outside
 * sets a bit of a per-device guard word and the access is skipped, so an
 * indexing error shows up here instead of as a fault.
 *   shl_checked_build  1 in the checked library, 0 in libshearlet.so.
 *   shl_check_status   synchronises `device`, then reads and clears its
 *                      guard word into *word (always 0 in libshearlet.so).
 */
int shl_checked_build(void);
shl_status shl_check_status(int device, unsigned* word);

#ifdef __cplusplus
}
#endif

#endif /* SHEARLET_H */
