/*
 * osar.h -- C ABI of libosar: Online FISTA for sparse SAR on one GB300 (sm_103a).
 *
 * Method: Flynn, Ivanov, Yazici, "Online Sparse Synthetic Aperture Radar
 * Imaging" (arXiv 2603.08582).  Per slow-time pulse n the library
 *   1. synthesises the pulse's forward block G_n = F_n H on the device, with
 *      F_n[m, p] = exp(-i 2 k_m |gamma(s_n) - x_p|), k_m = 2 pi f_m / c
 *      (Eqs. 2-4 and 6; the dictionary H is the identity, a host matrix or a
 *      seeded complex Gaussian);
 *   2. updates the sufficient statistics A_n = A_{n-1} + G_n^H G_n and
 *      b_n = b_{n-1} + G_n^H d_n (Eqs. 12-13, white noise R_n = I);
 *   3. refreshes lambda_n and the Lipschitz constant L_n (Eq. 11) by a
 *      warm-started power iteration;
 * and osar_iterate runs the inner loop of Algorithm 1 (gradient step,
 * complex soft-thresholding, momentum update).
 *
 * Naming: the paper writes the accumulated Gram as A_n and the per-pulse
 * operator as G_n; this header calls the accumulated Gram "gram" and the
 * per-pulse operator "block", and the coefficients c (length M, complex).
 *
 * Conventions for every call:
 *  - Complex numbers cross the boundary as interleaved (re, im) float64
 *    pairs ("c128").  Host pointers are plain CPU memory; "_dev" variants
 *    take device pointers of the stated type.
 *  - Calls on one context are ordered on the context's CUDA stream and are
 *    asynchronous unless they return data to host memory (those synchronise
 *    the stream before returning).
 *  - Every call returns an osar_status.  A CUDA error makes the context
 *    sticky-failed: later calls return OSAR_E_CUDA until osar_destroy.
 *    osar_last_error gives a one-line message for the last failure.
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - The library owns every device buffer it allocates; inputs are copied
 *    (or consumed on the stream) before the call's work completes, so the
 *    caller may reuse host buffers once a call returns.
 */
#ifndef OSAR_H
#define OSAR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct osar_ctx osar_ctx;

typedef enum {
  OSAR_OK = 0,
  OSAR_E_INVALID = 1,  /* bad argument or unsupported size */
  OSAR_E_OOM = 2,      /* device or host allocation failed */
  OSAR_E_CUDA = 3,     /* a CUDA call failed; the context is sticky-failed */
  OSAR_E_STATE = 4,    /* call not valid in the context's current state */
  OSAR_E_TIMEOUT = 5,  /* a bounded device-side wait gave up */
  OSAR_E_NUMERIC = 6,  /* non-finite value detected in a scalar */
  OSAR_E_IO = 7        /* checkpoint file could not be read or written */
} osar_status;

/* Arithmetic of the Gram update and of the FISTA matvec. */
typedef enum {
  OSAR_FP64 = 0,        /* plain path: FP64 everywhere (FP64 FMA pipes) */
  OSAR_FP32 = 1,        /* FP32 SIMT Gram and matvec */
  OSAR_SPLIT_BF16 = 2   /* tcgen05 split-BF16 (hi*hi + hi*lo + lo*hi) Gram
                           with FP32 accumulation; FP32 matvec; FP64 phases,
                           lambda and L */
} osar_precision;

typedef enum {
  OSAR_DICT_IDENTITY = 0,  /* H = I, M = N (pixel basis) */
  OSAR_DICT_HOST = 1,      /* H given as an N x M complex matrix */
  OSAR_DICT_GAUSSIAN = 2,  /* H = unit-norm complex Gaussian columns drawn by
                              Philox4x32-10 (see osar_config.dict_seed) */
  OSAR_DICT_EDGELET = 3    /* H = binary edgelets (Sec. III-A): see
                              osar_config.edgelet_lengths / _angles_deg */
} osar_dict_kind;

typedef struct {
  /* Pixel grid (Sec. II): nx x ny pixels of pixel_m metres, centred at the
     origin on flat ground; pixel p = i*nx + j sits at
     ((j - (nx-1)/2) pixel_m, (i - (ny-1)/2) pixel_m, 0). */
  int32_t nx, ny;
  double pixel_m;
  /* Frequencies f_m = linspace(f_lo_hz, f_hi_hz, n_freq), both ends kept. */
  int32_t n_freq;
  double f_lo_hz, f_hi_hz;
  /* Dictionary H (Sec. III-A). */
  int32_t dict_kind;          /* osar_dict_kind */
  int32_t n_atoms;            /* M; ignored (M = N) for the identity */
  const double* dict_c128;    /* OSAR_DICT_HOST: N x M column-major c128,
                                 copied during osar_create */
  uint64_t dict_seed;         /* OSAR_DICT_GAUSSIAN: entry (p, j) uses Philox
                                 counter (p, j, 0x5A5D1C7, 0), key = seed;
                                 z = sqrt(-2 ln u1) exp(2 pi i u2) with
                                 u = (k + 1/2) 2^-53 from 64-bit word pairs;
                                 columns scaled to unit 2-norm */
  int32_t precision;          /* osar_precision */
  /* lambda: lambda_relative != 0 => lambda_n = lambda * ||b_n||_inf, else
     lambda_n = lambda. */
  double lambda;
  int32_t lambda_relative;
  /* Power iteration for Eq. 11: power_iters_first steps at the first pulse
     (from v = 1/sqrt(M)), power_iters warm-started steps afterwards;
     L_n = max(L_{n-1}, (1 + lipschitz_margin) mu_n). */
  int32_t power_iters_first, power_iters;
  double lipschitz_margin;
  /* 0: Algorithm 1 as printed (t carried across pulses); 1: t = 1 per pulse */
  int32_t restart_momentum;
  /* SPLIT_BF16 only: 1 keeps a second FP32 word per Gram entry and adds each
     pulse with error-free (TwoSum) compensation; 0 plain FP32 accumulation */
  int32_t compensated;
  /* cudaStream_t for all work; NULL => a library-owned non-blocking stream */
  void* cuda_stream;
  /* Dictionary models only.  1: the phase synthesis and dictionary product
     of a pushed pulse run on a second, library-owned stream, on at most
     synth_ctas SMs, beside the FISTA burst of the previous pulse that is
     still streaming the Gram on cuda_stream; the pulse's data update waits
     for them.  Results are bitwise identical to 0, which runs every step of
     a push on cuda_stream.  Ignored while cuda_stream is being captured. */
  int32_t overlap_synthesis;
  /* SMs given to the overlapped dictionary product; 0 = chosen per pulse
     from the problem shape and the last burst's length, so that the product
     ends about when the burst does */
  int32_t synth_ctas;
  /* SPLIT_BF16: tensor-core products on pairs of SMs (one M = 256 tcgen05
     MMA per two 128 x 128 blocks that share their B rows, each SM loading
     half of B) instead of one SM per block.  Bit 0: the dictionary product;
     bit 1: the Gram update (whose read-modify-write of the Gram then goes
     through shared memory by bulk copies, in the room the smaller operand
     ring leaves).  Bitwise the same results either way.  Default 3. */
  int32_t tc_pairs;
  /* 1: the last power step of a push also applies the Gram to the next
     burst's first iterate z = c_hat (both vectors in one pass over the
     Gram), and that burst's first FISTA step uses the result; one Gram
     pass fewer per pulse, bitwise the same results.  0: separate passes.
     (FP32 and split-BF16 matvecs; the FP64 path and the pixel-space Gram
     form always use separate passes.) */
  int32_t fuse_first_step;
  /* lambda path: 1..8 solutions of the same pulses that differ only in
     lambda.  n_lambdas > 1 takes lambda_list[l] (relative or absolute per
     lambda_relative) for solution l and ignores `lambda`; the Gram, b, L_n
     and the power iteration are shared, and each Gram pass applies the Gram
     to two solutions' iterates at once.  Solution l is bitwise the one a
     context with lambda = lambda_list[l] computes.  osar_get_coeffs and
     osar_get_state report solution 0; osar_get_lambda_state any.  The list
     is copied at create. */
  int32_t n_lambdas;
  const double* lambda_list;
  /* SPLIT_BF16 with a dictionary, overlap_synthesis = 1, one lambda and
     n_freq <= 2048.  1 takes the Gram update off the critical path: the
     power steps and FISTA steps of pulse n apply G_n x as
     G_{n-1} x + A_n^H (A_n x) (two reads of the K x M block A_n besides the
     pass over G_{n-1}) while the side stream forms G_n = G_{n-1} + A_n^H A_n
     into a second Gram buffer; forward blocks alternate between two block
     buffers, and the next push swaps the Gram buffers.  The Gram is bitwise
     the one of 0; the iterates agree with 0 to rounding.  Needs a second
     Gram and block in device memory.  osar_get_gram*, osar_save,
     osar_gram_apply* and osar_unroll_grad first wait for the pending update
     (the rest of that pulse's burst then reads G_n).  A push while
     cuda_stream is being captured returns OSAR_E_STATE.  0: the update runs
     on cuda_stream before the power steps. */
  int32_t defer_gram;
  /* Guard regions (a memory-checking aid): 0 off; > 0 (a multiple of 256, at
     most 1 MiB) puts that many bytes, filled with 0xA5, behind every device
     buffer the context (or a batch created with this config first) owns;
     osar_check_guards reports buffers whose guard a kernel overwrote. */
  int32_t guard_bytes;
  /* OSAR_DICT_EDGELET (Sec. III-A, Dictionary Model): one binary atom per
     (length l, rotation psi, centre pixel), M = n_lengths x n_angles x N
     (n_atoms must be 0 or that number).  The edgelet steps by
     (round(cos psi), round(sin psi)) pixels, psi a multiple of 45 degrees in
     [0, 360), and covers the centre plus j - (l - 1) / 2 (integer division)
     steps for j = 0 .. l - 1; pixels off the grid are dropped.  Atom
     m = (length index x n_angles + angle index) x N + y x nx + x.  Lengths
     in [1, 64], at most 16 of each list; the lists are copied at create.
     The forward block A_s = F_s H is then a sum of l phase rows per atom
     (no GEMM, no dictionary in device memory). */
  int32_t n_edgelet_lengths;
  const int32_t* edgelet_lengths;
  int32_t n_edgelet_angles;
  const double* edgelet_angles_deg;
  /* SPLIT_BF16 with the Gram update on SM pairs (tc_pairs bit 1), defer_gram
     = 0.  1: the Gram update's epilogue, which holds each updated 128 x 128
     block of G_n, also applies it to the power vector v (Eq. 11: the first
     power step of the pulse), so that step reads no Gram: one Gram pass fewer
     per pulse.  The partial sums are combined in a fixed order (results do
     not depend on the grid) but in another order than a separate pass, so
     mu_n, L_n and the iterates agree with 0 to rounding, not bitwise.  0:
     every power step is a separate pass.  Ignored on the other paths.
     Default 1. */
  int32_t fuse_power_gram;
  /* OSAR_DICT_EDGELET only, one lambda, defer_gram = 0.  1: the pixel-space
     Gram form.  Since A_s = F_s H, G_n = H^H P_n H and b_n = H^H b_pix with
     P_n = sum_s F_s^H F_s (N x N) and b_pix = sum_s F_s^H d_s; the context
     accumulates P_n and b_pix with its pixel-basis kernels and applies G_n
     to a coefficient vector x as H^H (P_n (H x)) (sums over H's pixel and
     atom lists around one pass over the packed P_n), in Algorithm 1 and in
     the power iteration.  P_n has N^2 entries where G_n has M^2, and no
     forward block A_s is formed.  Coefficients, b (osar_get_b returns
     H^H b_pix), lambda_n, L_n and t are those of the stored-Gram form to
     rounding.  In this form osar_get_gram, osar_get_gram_entries and
     osar_gram_apply work on P_n (N x N, pixel vectors); osar_save,
     osar_load, osar_unroll_grad and osar_get_lambda_state return
     OSAR_E_STATE.  Default 0. */
  int32_t pixel_gram;
  /* Order of the Gram update's tiles: the upper blocks in super-blocks of
     gram_superblock x gram_superblock blocks, so that the tiles running at
     the same time share operand rows in L2; 0 = 32 (16 with gram_ahead).
     Any order gives the same results (each output block is one tile's).
     In [0, 64]. */
  int32_t gram_superblock;
  /* SPLIT_BF16, overlap_synthesis = 1, defer_gram = 0 and pixel_gram = 0
     (any dictionary, the pixel basis included, lambda paths too).  The Gram
     update of Eqs. 12-13 run ahead: a push queues the pulse's forward block
     A_n and G_n = G_{n-1} + A_n^H A_n on the side stream, into a second
     Gram buffer, so that both run beside the previous pulse's burst (which
     still reads G_{n-1}); cuda_stream then waits for G_n, the buffers swap,
     and the data update, power steps and burst follow as usual.  The update's
     tensor work then overlaps the bandwidth-bound Gram passes instead of
     running between bursts.  1: a model of the last bursts' length against
     the tensor work decides per push between this and the in-order
     schedule (the forward block beside the burst, the update after it on
     cuda_stream), so short bursts keep the in-order one, and so does a
     push queued while cuda_stream is idle (after an osar_iterate that
     returned its step count, say: nothing runs for the update to hide
     beside); 2: always ahead.
     Every result is bitwise that of 0.  Needs a second Gram in device
     memory.  A push while cuda_stream is being captured returns
     OSAR_E_STATE; bursts and osar_unroll_grad may still be captured (the
     Gram passes read the current buffer's address from device memory,
     which each swap rewrites in stream order).  0 (default): in order. */
  int32_t gram_ahead;
} osar_config;

/* Fill *cfg with defaults: 32 x 32 grid, 1 m pixels, 128 frequencies over
   9.9-10.1 GHz, identity dictionary, FP64, lambda = 0.05 relative,
   30 / 4 power steps, margin 0.01, carried momentum, compensated = 1,
   overlap_synthesis = 1, synth_ctas = 0 (automatic), tc_pairs = 3
   (both tensor-core products on SM pairs), fuse_first_step = 1,
   n_lambdas = 1, defer_gram = 0, guard_bytes = 0, fuse_power_gram = 1,
   pixel_gram = 0, gram_superblock = 0 (32), gram_ahead = 0. */
void osar_config_default(osar_config* cfg);

/* Create a context for the problem of Sec. III-C: the online reconstruction
   starts from A_0 = 0, b_0 = 0 and c_hat_0 = 0 (Algorithm 1's input), over
   the grid, frequencies and dictionary of Sec. II and III-A that cfg gives.
   Validates cfg, allocates the Gram (packed upper 128 x 128 blocks), data
   vector, coefficient state and per-pulse work buffers, and builds the
   dictionary on the device.  *out is NULL on failure.
   Errors: OSAR_E_INVALID (sizes <= 0, unknown enums, M or N too large),
   OSAR_E_OOM, OSAR_E_CUDA. */
osar_status osar_create(const osar_config* cfg, osar_ctx** out);

/* Release every device and host resource of ctx (NULL is accepted). */
osar_status osar_destroy(osar_ctx* ctx);

/* One pulse (Eqs. 12-13 and the lambda / L refresh).  gamma_xyz: platform
   position gamma(s_n) in metres (3 doubles, host).  d_c128: the pulse's
   n_freq complex samples (host).  Asynchronous; the inputs are staged before
   return.  Errors: OSAR_E_INVALID for NULL pointers or non-finite gamma. */
osar_status osar_push_pulse(osar_ctx* ctx, const double gamma_xyz[3],
                            const double* d_c128);

/* Same, with d already on the device (n_freq complex128, 16-byte aligned).
   The buffer must stay valid until the stream reaches the call's work. */
osar_status osar_push_pulse_dev(osar_ctx* ctx, const double gamma_xyz[3],
                                const void* d_dev_c128);

/* A pulse with non-white noise (Eq. 12 with R_n = diag(noise_var)):
   noise_var holds the K (n_freq) noise variances of this pulse's
   frequencies, finite and > 0 (host, copied).  Its update is
   G_n^H R_n^{-1} G_n and G_n^H R_n^{-1} d_n: the library scales the data and
   the rows of the pulse's phase block by 1 / sqrt(noise_var[k]), so the
   dictionary products, Gram update and data update run unchanged.
   noise_var = NULL is osar_push_pulse (R_n = I).  Otherwise as
   osar_push_pulse. */
osar_status osar_push_pulse_var(osar_ctx* ctx, const double gamma_xyz[3],
                                const double* d_c128, const double* noise_var);

/* Run up to max_iters steps of Algorithm 1's inner loop.  The first call
   after a pulse starts the burst (c^(0) = c_hat_{n-1}, z^(1) = c^(0),
   t_1 = t_{n-1}, or 1 at the first pulse); later calls continue it, so
   iterate(a) then iterate(b) equals iterate(a + b).  tol > 0 stops the burst
   once ||c^(k) - z^(k)||_2 <= tol ||c^(k)||_2 (decided on the device; the
   remaining launches return at once).  iters_done (nullable) receives the
   number of steps taken in this call, which synchronises the stream.
   With iters_done = NULL a call only queues kernels on cuda_stream, so a
   continuing call (not the first after a pulse) can be captured into a
   CUDA graph and replayed, in order on that stream, for later pulses.
   Errors: OSAR_E_STATE before the first pulse, OSAR_E_INVALID for
   max_iters < 0. */
osar_status osar_iterate(osar_ctx* ctx, int32_t max_iters, double tol,
                         int32_t* iters_done);

/* Copy c_hat_n (M complex), the estimate Algorithm 1 returns after the
   pulses pushed so far (Sec. III-C), to host memory; synchronises. */
osar_status osar_get_coeffs(osar_ctx* ctx, double* out_c128);

/* Copy c_hat (M complex128) into device memory out_dev; asynchronous. */
osar_status osar_get_coeffs_dev(osar_ctx* ctx, void* out_dev_c128);

/* Queue a copy of c_hat (M complex, interleaved doubles) into host memory
   on the context's stream and return at once; the copy has landed when
   osar_wait_coeffs(ctx, slot) returns.  slot in [0, OSAR_COPY_SLOTS) names
   the copy, so that the image of pulse s can be read while pulse s + 1 is
   already queued.  out_c128 should be pinned (page-locked) memory: CUDA
   copies into pageable memory before returning.  The buffer belongs to the
   caller and must stay valid until the wait.  No paper counterpart.
   Errors: OSAR_E_INVALID (NULL buffer, slot out of range). */
#define OSAR_COPY_SLOTS 4
osar_status osar_get_coeffs_async(osar_ctx* ctx, double* out_c128,
                                  int32_t slot);

/* Wait for the last copy queued on `slot` by osar_get_coeffs_async (returns
   at once when none was queued).  Errors: OSAR_E_INVALID (slot out of
   range), OSAR_E_TIMEOUT (a bounded device wait gave up). */
osar_status osar_wait_coeffs(osar_ctx* ctx, int32_t slot);

/* Solution l of a lambda path (0 <= l < n_lambdas): c_hat (M complex, may
   be NULL), lambda_n, momentum t and the FISTA steps of the last
   osar_iterate call (may be NULL); synchronises.  No paper counterpart:
   the path shares one Gram (Eqs. 12-13) between several lambdas.
   Errors: OSAR_E_INVALID (l out of range). */
osar_status osar_get_lambda_state(osar_ctx* ctx, int32_t l, double* out_c128,
                                  double* lambda, double* t, int32_t* iters);

/* Pulse count n, L_n, lambda_n, momentum t; synchronises.  Any pointer may
   be NULL. */
osar_status osar_get_state(osar_ctx* ctx, int32_t* n, double* lipschitz,
                           double* lambda, double* t);

/* M and N of the context. */
osar_status osar_get_dims(const osar_ctx* ctx, int32_t* m_atoms,
                          int32_t* n_pixels, int32_t* n_freq);

/* The accumulated Gram A_n as a dense M x M row-major c128 host matrix
   (the stored upper half is mirrored; the compensation word is added when
   present).  Synchronises. */
osar_status osar_get_gram(osar_ctx* ctx, double* out_c128);

/* Gram entries at (rows[q], cols[q]) for q < count, as c128; synchronises. */
osar_status osar_get_gram_entries(osar_ctx* ctx, const int32_t* rows,
                                  const int32_t* cols, int32_t count,
                                  double* out_c128);

/* The data vector b_n (M complex) as c128 host memory; synchronises. */
osar_status osar_get_b(osar_ctx* ctx, double* out_c128);

/* y = A_n x with the stored Gram, in the context's matvec arithmetic
   (x, y: M complex, host c128); synchronises.  Does not touch the FISTA
   state. */
osar_status osar_gram_apply(osar_ctx* ctx, const double* x_c128,
                            double* y_c128);

/* y = A_n x like osar_gram_apply, but without any allocation: x and y are
   caller device buffers, the call is asynchronous on the context's stream,
   and the matvec's scratch comes from a 4 MiB static device array inside the
   library instead of cudaMalloc.  No counterpart in the paper: it exists for
   callers that may not allocate device memory after start-up (fixed-budget
   embedded or flight pipelines, hosts with their own memory pool).
   Vectors: M complex128 each (interleaved doubles), device or managed memory
   of the current device, 16-byte aligned; in the pixel-space Gram form the
   apply works on P_n and the vectors have N (pixel) entries.
   Limit: the Gram's dimension (M atoms, or N pixels in the pixel-space form)
   at most 4096 always fits; larger ones return OSAR_E_INVALID, as do NULL,
   host, other-device or unaligned vectors (checked before any launch).
   The array is shared by all calls on a device and keeps the last call's
   contents; calls that overlap on the GPU race on it and must be ordered by
   the caller.  osar_create looks up the array's address on its device (under
   CUDA's lazy module loading this is also when the array is placed in device
   memory), so the apply itself allocates nothing; if that lookup failed the
   first call repeats it (make that call before any stream capture). */
osar_status osar_gram_apply_static(osar_ctx* ctx, const void* x_dev_c128,
                                   void* y_dev_c128);

/* Reconstruction quality of c_hat_n (Sec. IV-B).  The experiments count
   the "large" coefficients, |c_m| > 2e-2, against slow time, and report the
   SNR of Eq. 18, 20 log10(mu_signal / mu_noise).  This call reads mu as an
   RMS amplitude in the coefficient domain: over a reference support (the
   scene's true atoms, which only the caller knows) and over its complement.
   Deterministic (one CTA reduces the vector in a fixed order), in FP64;
   synchronises.  A lambda path reports solution 0; the pixel-space Gram form
   its atom coefficients. */
typedef struct {
  int32_t n_large;                /* m with |c_m| > threshold */
  int32_t n_nonzero;              /* m with c_m != 0 */
  int32_t n_support;              /* distinct indices of the support given */
  int32_t large_outside_support;  /* large coefficients off the support (all
                                     of them without a support) */
  double l1;                      /* sum_m |c_m| */
  double max_abs;                 /* max_m |c_m| */
  double rms_signal;              /* RMS of |c_m| on the support (0 without) */
  double rms_noise;               /* RMS of |c_m| off the support */
  double snr_db;                  /* 20 log10(rms_signal / rms_noise); NaN
                                     without a support, +inf when rms_noise
                                     is 0 and rms_signal is not */
} osar_metrics;

/* threshold >= 0 (finite); support: n_support atom indices in [0, M) (host,
   duplicates allowed), or NULL with n_support = 0.  The first call allocates
   a scratch of M + 256 bytes, kept until destroy.  Errors: OSAR_E_INVALID
   (NULL out, bad threshold, index out of range), OSAR_E_OOM, OSAR_E_CUDA. */
osar_status osar_get_metrics(osar_ctx* ctx, double threshold,
                             const int32_t* support, int32_t n_support,
                             osar_metrics* out);

/* Noise-free pulse data d = G_n c for a platform at gamma_xyz (Eqs. 5-6),
   computed on the device in FP64: c (M complex, host) in, d (n_freq
   complex, host) out.  Does not touch the statistics; synchronises. */
osar_status osar_simulate_pulse(osar_ctx* ctx, const double gamma_xyz[3],
                                const double* coeffs_c128, double* d_c128);

/* Differentiation form.  The paper leaves online parameter tuning to future
   work (Sec. I, Sec. V); this call provides the gradients it would need.  It
   runs `steps` (T) steps of Algorithm 1's inner loop on the context's current
   Gram A_n and data vector b_n, from c^(0) = z^(1) = c0 with t_1 = t0, using
   the given step tau and threshold lambda * tau (not the context's own), then
   evaluates L = ||c_T - c_true||_2^2 and back-propagates through all T steps
   with hand-written adjoint kernels.  Memory: (z_k, c_{k-1}) is stored every
   ckpt_every steps (sqrt(T) is the usual choice) and each segment is
   recomputed during the reverse sweep, so a step costs three Gram passes.
   Outputs (host memory, each nullable): loss, dL/dlambda, dL/dtau, dL/db
   (M complex, convention dL/dRe + i dL/dIm), c_T (M complex).  Since
   b_n = sum_s G_s^H d_s, the gradient with respect to pulse s's data is
   dL/dd_s = G_s dL/db, which osar_simulate_pulse computes when given dL/db
   as its coefficients.  Arithmetic: FP64 on the FP64 path; on the FP32 and
   split-BF16 paths the Gram passes run in FP32 and everything else in FP64.
   The first call allocates the scratch (kept until destroy).  Synchronises.
   Errors: OSAR_E_STATE before the first pulse; OSAR_E_INVALID for steps < 1,
   ckpt_every < 1, tau <= 0, lambda < 0, t0 < 1 or NULL c0 / c_true. */
osar_status osar_unroll_grad(osar_ctx* ctx, int32_t steps, int32_t ckpt_every,
                             double lambda, double tau, double t0,
                             const double* c0_c128, const double* c_true_c128,
                             double* loss, double* d_lambda, double* d_tau,
                             double* d_b_c128, double* c_T_c128);

/* Change the lambda setting of solution l (0 <= l < n_lambdas; 0 without a
   lambda path): a factor rho (lambda_n = rho ||b_n||_inf) when the context
   is relative, else the absolute lambda, finite and >= 0.  It takes effect
   at the next pulse's lambda_n refresh (the current burst keeps its
   lambda_n).  The paper leaves online parameter tuning to future work
   (Sec. I, Sec. V); this call and osar_unroll_grad let a caller tune lambda
   while the pulses arrive.  Errors: OSAR_E_INVALID. */
osar_status osar_set_lambda(osar_ctx* ctx, int32_t l, double lambda);

/* The gram_ahead schedule (see osar_config) from the next push on: 0 in
   order, 1 decided per push by the model, 2 ahead.  Results do not depend
   on it.  OSAR_E_STATE when the context was created with gram_ahead = 0
   (no second Gram buffer), OSAR_E_INVALID for another mode. */
osar_status osar_set_gram_ahead(osar_ctx* ctx, int32_t mode);

/* Wait for all work queued on the context's stream (and on its side
   stream, see overlap_synthesis). */
osar_status osar_synchronize(osar_ctx* ctx);

/* Failure-detection check.  Every wait inside the library's kernels (TMA
   copies, tensor-core commits, peer CTAs) polls its barrier against the GPU
   clock and gives up after a limit: it records a timeout in the context's
   device error word, stops its CTA's other roles, drains what it issued and
   returns, so the GPU stays usable and the next state read returns
   OSAR_E_TIMEOUT.  This call exercises that path on purpose: one CTA waits,
   through the same bounded wait, on a shared-memory barrier nothing arrives
   on, with limit_ns in [1e6, 1e10] nanoseconds.  It synchronises and returns
   OSAR_E_TIMEOUT when the wait gave up as designed (OSAR_E_CUDA if the
   launch failed).  Nothing else is touched, but the context keeps the
   recorded timeout: its state reads return OSAR_E_TIMEOUT from then on. */
osar_status osar_probe_bounded_wait(osar_ctx* ctx, int64_t limit_ns);

/* Guard check (config guard_bytes > 0): synchronises, then sets *corrupted
   to the number of device buffers whose guard region no longer holds its
   fill; osar_last_error then names the first one.  With guards off,
   *corrupted = 0. */
osar_status osar_check_guards(osar_ctx* ctx, int32_t* corrupted);

/* Test aid for the guard check: overwrites one byte of guard region `index`
   (allocation order) from the host.  OSAR_E_INVALID when guards are off or
   index is out of range. */
osar_status osar_poke_guard(osar_ctx* ctx, int32_t index);

/* Per-kernel device timing.  When enabled, CUDA events bracket every
   launch of the listed kernel classes on the context's stream; reading the
   counters synchronises.  kernel: 0 phase, 1 dictionary GEMM, 2 Gram GEMM,
   3 data-vector update, 4 matvec (FISTA and power steps), 5 FISTA finalize,
   6 power finalize, 7 deferred update's block term, 8 the dense
   dictionary products of the pixel-space Gram form (u = D x and D^H w, the
   latter with its step).
   launches / total_ms may be NULL.
   Phase and dictionary launches of an overlapped push are bracketed on the
   side stream, so their time includes sharing the GPU with the burst. */
osar_status osar_profile_enable(osar_ctx* ctx, int32_t on);
/* Restricts the bracketed launches to the classes whose bits are set in
   mask (bit k = class k above; the default is every class).  Each bracket
   adds two event records to the stream between launches, which lengthens
   a sequence of short launches measurably, so a timing run can bracket
   only the classes it needs.  OSAR_E_INVALID for bits past the last
   class. */
osar_status osar_profile_select(osar_ctx* ctx, uint32_t mask);
/* Brackets one launch in `every` of class `kernel` (the next one first,
   and again after each osar_profile_reset; the default is 1, every
   launch): the counters then hold that sample.  OSAR_E_INVALID for an
   unknown class or every < 1. */
osar_status osar_profile_sample(osar_ctx* ctx, int32_t kernel, int32_t every);
osar_status osar_profile_read(osar_ctx* ctx, int32_t kernel,
                              int64_t* launches, double* total_ms);
/* Clears the timing counters, the launch count and the pass count. */
osar_status osar_profile_reset(osar_ctx* ctx);

/* Gram passes that did work since the last osar_profile_reset: one per
   power step and one per FISTA step that ran (steps skipped after the stop
   rule held launch a matvec that returns at once and are not counted).
   Synchronises.  No paper counterpart: instrumentation for the roofline. */
osar_status osar_profile_passes(osar_ctx* ctx, int64_t* passes);

/* Pushes since the last osar_profile_reset whose Gram update ran ahead on
   the side stream (gram_ahead); the others ran in order.  *last_grid
   (nullable) gets the side stream's SM count of the last such push.
   Host-side, no synchronisation. */
osar_status osar_profile_ahead(const osar_ctx* ctx, int64_t* pushes,
                               int32_t* last_grid);

/* Total library kernel launches issued on this context since creation
   (or since the last reset); no synchronisation. */
osar_status osar_launch_count(const osar_ctx* ctx, int64_t* launches);

/* Bytes of device memory the context holds. */
osar_status osar_device_bytes(const osar_ctx* ctx, int64_t* bytes);

/* Checkpoint: the sufficient statistics (Gram, b), c_hat, t, L, lambda, the
   power-iteration vector and the pulse count are exactly what Table I says
   Online FISTA must keep; osar_save writes them with the config, osar_load
   rebuilds a context (with cfg's stream, dictionary and precision, which
   must match the file) that continues bit-for-bit.  Errors: OSAR_E_IO,
   OSAR_E_INVALID on a mismatched config. */
osar_status osar_save(osar_ctx* ctx, const char* path);
osar_status osar_load(const char* path, const osar_config* cfg,
                      osar_ctx** out);

/* ------------------------------------------------------------------------
 * Batching form: many independent online reconstructions of uneven size
 * (several platforms or image patches) in one context.  Each scene keeps its
 * own Gram, data vector, warm start, lambda, L and momentum, exactly as a
 * separate osar_ctx would; the per-pulse work of all scenes runs as single
 * launches (one persistent tensor-core launch covers every scene's Gram
 * blocks) and FISTA bursts are replayed from CUDA graphs captured per step
 * count.  Scenes use the pixel basis and one precision; frequencies, grids,
 * lambda settings and power-iteration counts may differ per scene.
 * ------------------------------------------------------------------------ */
typedef struct osar_batch osar_batch;

/* Create a batch from n_scenes configs (copied).  cuda_stream as in
   osar_config.  Errors: OSAR_E_INVALID (non-identity dictionary, mixed
   precision, bad sizes), OSAR_E_OOM, OSAR_E_CUDA. */
osar_status osar_batch_create(const osar_config* cfgs, int32_t n_scenes,
                              void* cuda_stream, osar_batch** out);
osar_status osar_batch_destroy(osar_batch* batch);

/* One pulse for every scene with active[s] != 0 (Eqs. 12-13, lambda and L
   per scene); scenes with active[s] == 0 keep their state and skip the next
   bursts.  gammas_xyz: n_scenes x 3 positions; d_c128: n_scenes rows of
   d_stride complex samples, row s holding scene s's n_freq samples (host).
   Asynchronous; inputs are staged before return. */
osar_status osar_batch_push(osar_batch* batch, const int32_t* active,
                            const double* gammas_xyz, const double* d_c128,
                            int32_t d_stride);

/* Up to max_iters steps of Algorithm 1 for every scene active in the last
   push (same semantics per scene as osar_iterate, including tol).  iters
   (nullable, n_scenes) receives each scene's steps in this call and
   synchronises. */
osar_status osar_batch_iterate(osar_batch* batch, int32_t max_iters, double tol,
                               int32_t* iters);

/* c_hat of one scene (M complex, host); synchronises. */
osar_status osar_batch_get_coeffs(osar_batch* batch, int32_t scene,
                                  double* out_c128);

/* Pulse count, L, lambda and t of one scene; synchronises. */
osar_status osar_batch_get_state(osar_batch* batch, int32_t scene, int32_t* n,
                                 double* lipschitz, double* lambda, double* t);

/* Autotuner of the batching form, timing candidates on the device:
    1. the Gram update's tile order: each scene's upper blocks in
       super-blocks of 4, 8, 16 or 32 x 32 blocks (the tiles running together
       share operand rows in L2), the scenes in index order or the largest
       first.  Timed only when no pulse has been pushed yet (the statistics
       and operands are then zero, so the timed updates change nothing);
       after the first push the current order is kept.  Every output block is
       one tile's, so results are bitwise the same in any order;
    2. the matvec's work-item size: 1, 2, 4, 8 or 16 blocks per segment.
   The choices are cached in the text file named by the environment variable
   OSAR_TUNE_CACHE (when set) and reused by later batches of the same shape
   (also at create).  chosen (nullable) receives the segment size.  No paper
   counterpart. */
osar_status osar_batch_autotune(osar_batch* batch, int32_t* chosen);

/* The tuning in force: blocks per matvec segment, the Gram tile order's
   super-block size and scene order (1: largest first), and the Gram update's
   time in the default order (8, index order) and in the chosen one, as the
   last autotune measured them (0 when it did not time them).  Any pointer
   may be NULL. */
osar_status osar_batch_get_tuning(const osar_batch* batch, int32_t* segment_blocks,
                                  int32_t* gram_superblock,
                                  int32_t* gram_largest_first,
                                  double* gram_ms_default, double* gram_ms_chosen);

/* Scene count, device bytes, kernel launches so far, segment size. */
osar_status osar_batch_info(const osar_batch* batch, int32_t* n_scenes,
                            int64_t* device_bytes, int64_t* launches,
                            int32_t* segment_blocks);
osar_status osar_batch_synchronize(osar_batch* batch);
/* Guard check of a batch (guard_bytes of the first scene's config). */
osar_status osar_batch_check_guards(osar_batch* batch, int32_t* corrupted);
const char* osar_batch_last_error(const osar_batch* batch);

/* One-line description of the last error on ctx (or of the last failed
   osar_create when ctx is NULL).  Never NULL. */
const char* osar_last_error(const osar_ctx* ctx);

/* Library version string. */
const char* osar_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OSAR_H */
