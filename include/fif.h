/*
 * fif.h -- C ABI of the GB300 (sm_103a) FFT-based Iterative Filtering library
 * (libfif.so).
 *
 * The method is the "FIF" direct form of Iterative Filtering from Cicone &
 * Zhou, "Numerical Analysis for Iterative Filtering with New Efficient
 * Implementations Based on FFT":
 *
 *   - outer loop (Algorithm 2, Sec. 3): while the remainder r has at least two
 *     extrema, pick the window half-support L from the extrema count k
 *     (eq. Unif_Mask_length, L = mask_scale * floor(nu*n/k)), extract one IMF,
 *     subtract it; the final remainder is appended (Algorithm 1/2);
 *   - inner loop, replaced by one spectral multiplier (Theorem 5,
 *     eq. IMF1_direct, eq. One step_algo of Sec. 4):
 *         IMF_hat_k = (1 - w_hat_k)^m * r_hat_k,
 *     with w_hat the eigenvalues of the circulant window matrix (eq. Lambdas)
 *     and m the number of inner iterations picked by the relative stopping
 *     rule eq. SD, ||u_m - u_{m-1}|| / ||u_{m-1}|| < delta, evaluated in the
 *     frequency domain through Parseval (proof of Theorem 2), capped by
 *     max_inner (Sec. 3, after eq. SD).
 *
 * Signals are real, periodic (Sec. 4 requires a periodic extension), sampled
 * on x_j = j/n.  The window is the triangle of eq. triangular, sampled at
 * integer offsets (taps (L-|d|)/L^2, |d| < L): the autocorrelation of a
 * length-L box, so 0 <= w_hat <= 1 (Corollary 2).
 *
 * Conventions for every entry point:
 *   - All work is asynchronous on the plan's CUDA stream unless stated.
 *   - Data pointers are DEVICE pointers unless the name or comment says host.
 *     The library never allocates or frees caller memory; the plan owns its
 *     own device tables and scratch and frees them in fif_plan_destroy.
 *   - The return value reports argument and launch errors only.  Per-signal
 *     outcomes are written to sig_status (stop reason | flags, see below).
 *   - Integer outputs are int32; sample data is float32, row-major.
 *   - A plan is not thread-safe: calls on one plan must not overlap.
 */
#ifndef FIF_H
#define FIF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fif_plan_s* fif_plan_t;

typedef enum {
  FIF_OK = 0,
  FIF_EINVAL = 1,        /* invalid argument (NULL pointer, bad size, bad descriptor) */
  FIF_ENOMEM = 2,        /* the plan could not allocate its device tables or scratch */
  FIF_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
  FIF_ETIMEOUT = 4,      /* a bounded device wait gave up */
  FIF_EUNSUPPORTED = 5   /* valid request the library does not implement (e.g. n not 2^a 3^b) */
} fif_status;

typedef enum {
  FIF_WIN_TRIANGLE = 0,  /* eq. triangular, sampled; w_hat = [sin(pi k L/n) / (L sin(pi k/n))]^2 */
  FIF_WIN_SHAPE = 1      /* generated by a shape g (Theorem 4's double convolution, eq. W_m): the
                            filter h_i = g((i + 1/2)/L), i < L, g the piecewise-linear
                            interpolant of fif_plan_desc.window_shape on [0, 1] (one sample = a
                            constant); the window is the autocorrelation h * h divided by its
                            sum, half-support L like the triangle's, and
                            w_hat_k = |DFT(h)_k|^2 / (sum h)^2 in [0, 1].  A constant shape is
                            the triangle.  Fused and staged lengths: tabulated for every L
                            when the plan first meets a length n (Lmax * P * 16 bytes of
                            device memory, Lmax = (n+1)/2, P = n/2+1).  Multi-pass lengths:
                            each IMF's row is computed for its L (a float-float transform of
                            h per IMF, P * 8 more bytes per signal).  FIF_APRIORI_N0 and
                            fif_decompose_noalloc return FIF_EUNSUPPORTED with it. */
} fif_window;

typedef enum {
  FIF_PREC_FP32 = 0,      /* FP32 FFTs and multiplier; m chosen with an FP32 screen + FP64 tie-break */
  FIF_PREC_SPLIT_BF16 = 1 /* as FIF_PREC_FP32, but the radix-16 passes of the fused path's inverse
                             FFT (powers of two 32 <= n <= fif_fused_max_n(), which take an
                             E = 16 schedule) run on the tensor cores: each 16-point DFT as a
                             real 32 x 32 matrix product (warp-level mma, BF16 operands, FP32
                             accumulation; no reference in the paper, which uses plain FFTs,
                             Sec. 4) with both the DFT
                             matrix and the data split into BF16 hi + lo and three products
                             (hi*hi + hi*lo + lo*hi), good to a few times 2^-18 relative per pass
                             instead of FP32's 2^-24.  The forward transform, m selection, window
                             spectrum and epilogue are those of FIF_PREC_FP32.  Other lengths
                             (a factor 3, or n < 32), the staged path
                             (fif_decompose), the multi-pass path (n above fif_fused_max_n) and
                             fif_decompose_noalloc run FP32.  fif_plan_tune keeps the schedule. */
} fif_precision;

/* ---- per-signal status word (sig_status): low byte = stop reason ---- */
#define FIF_STOP_EXTREMA    1   /* remainder has < 2 extrema (Algorithm 1/2 outer test) */
#define FIF_STOP_MASK       2   /* 2L-1 > n: the window would wrap the period (Sec. 3.1, l <= (n-1)/2) */
#define FIF_STOP_MAX_IMFS   3   /* max_imfs IMFs extracted */
#define FIF_STOP_FORCED_END 4   /* FIF_FORCE_L schedule ended (mask_len[K] <= 0) */
#define FIF_STOP_NONFINITE  5   /* NaN or Inf in the input: no IMF, the input is copied as remainder */
/* flags, OR-ed into sig_status (any IMF) and into fif_imf_diag.flags (that IMF) */
#define FIF_FLAG_NEAR_DELTA_TIE  (1 << 8)  /* |SD_m - delta| or |SD_{m-1} - delta| <= 1e-6 delta */
#define FIF_FLAG_EXTREMA_TIE     (1 << 9)  /* the extrema count could change under a perturbation of
                                              r of 2^-18 max|s|: a first difference within
                                              2^-17 max|s| of zero whose flip changes the
                                              count (see fif_imf_diag) */
#define FIF_FLAG_MAX_INNER_HIT   (1 << 10) /* SD_j >= delta for every j <= max_inner; m = max_inner */
#define FIF_FLAG_FP64_TIEBREAK   (1 << 11) /* an m decision fell inside the FP32 screen's error band
                                              and was re-evaluated in FP64 */
#define FIF_FLAG_L_CLAMPED       (1 << 12) /* the mask rule gave L < 2; L = 2 used */

/* ---- plan flags ---- */
#define FIF_FORCE_L 1  /* mask_len[] is an INPUT: L for IMF K is mask_len[K]; a value <= 0 ends the
                          decomposition (FIF_STOP_FORCED_END).  The extrema test is skipped.  For
                          tests of linearity and worked examples. */
#define FIF_FORCE_MULTIPASS 2  /* run every signal through the multi-pass path that long signals
                                  take (FFT passes through global memory), whatever its length;
                                  for tests that compare the two paths */
#define FIF_APRIORI_N0 4  /* m = the a-priori bound of Theorem 5 (eq. N0_discrete) instead of the
                             search of eq. SD: the least natural N0 with
                             N0^N0 / (N0+1)^(N0+1) < delta / (||U^T r||_inf sqrt(n-1-k)),
                             U^T the unitary DFT, r the current remainder, k = gcd(n, L) - 1
                             zero eigenvalues of W; capped at max_inner (MAX_INNER_HIT).  delta
                             is then the absolute threshold of eq. Discrete_Abs_StopCond.
                             NEAR_DELTA_TIE marks a bound within 1e-6 of the threshold. */
#define FIF_PEAK_MASK 8  /* mask length from the spectrum (end of Sec. 2): L = mask_scale *
                            floor(nu n / (2 k*)), k* the largest |r_hat_k| over 1 <= k <= n/2
                            (smallest k among equal magnitudes) of the current remainder; the
                            extrema count still decides the stop.  EXTREMA_TIE also marks a
                            second bin within 1e-5 (relative) of the peak. */

typedef struct {
  fif_window window;        /* FIF_WIN_TRIANGLE or FIF_WIN_SHAPE */
  double nu;                /* eq. Unif_Mask_length tuning parameter (1.6) */
  int32_t mask_scale;       /* leading factor of the mask rule: 1 (half-support L = floor(nu n/k))
                               or 2 (the paper's l = 2 floor(nu N/k)) */
  double delta;             /* stopping threshold of eq. SD, > 0 */
  int32_t max_inner;        /* cap on m (number of inner iterations), 1 .. 1<<20 */
  int32_t max_imfs;         /* cap on the number of IMFs (remainder not counted), 0 .. 64 */
  fif_precision precision;  /* FIF_PREC_FP32 or FIF_PREC_SPLIT_BF16 */
  int64_t max_n;            /* largest signal length this plan accepts */
  int32_t flags;            /* 0 or FIF_FORCE_L | FIF_FORCE_MULTIPASS | FIF_APRIORI_N0 |
                               FIF_PEAK_MASK */
  double gamma;             /* 0, or 0 < gamma < 1: thresholded IMF (eq. I_gamma,
                               eq. IMF_cont_stop_threshold): with m chosen as usual, every bin
                               with (1 - w_hat_k)^m >= 1 - gamma passes whole into the IMF
                               (w_hat_k taken as 0) and leaves the remainder */
  const double* window_shape;  /* FIF_WIN_SHAPE: HOST array of the shape's samples g_0..g_{len-1}
                                  at x = j/(len-1) (copied by fif_plan_create): finite, >= 0,
                                  and the interpolant > 0 inside (0, 1) (every interior sample
                                  > 0; len 1: g_0 > 0; len 2: g_0 + g_1 > 0), else FIF_EINVAL.
                                  Ignored for FIF_WIN_TRIANGLE. */
  int32_t window_shape_len;    /* 1 .. 65536 */
} fif_plan_desc;

/* Optional per-IMF diagnostics, one record per outer step: record K < n_imfs
 * describes IMF K; record n_imfs describes the final remainder. */
typedef struct {
  int32_t k_extrema;       /* extrema count of the remainder at the outer test before IMF K
                              (for record n_imfs: of the final remainder) */
  int32_t zero_crossings;  /* zero crossings of that remainder (IMF definition, Sec. 1) */
  int32_t flags;           /* FIF_FLAG_* raised while extracting IMF K */
  float inf_norm;          /* ||IMF_K||_inf (significance, Sec. 2.3); record n_imfs: ||r||_inf */
} fif_imf_diag;

/* Create a plan.  desc is copied.  cuda_stream is a cudaStream_t (NULL = the
 * legacy default stream).  Allocates the plan's device scratch for signals up
 * to desc->max_n.  Window tables for a length n are built on the first call
 * that sees n (fif_plan_prepare builds them ahead of time); building them
 * allocates, so that first call must not be inside a stream capture.
 * Errors: FIF_EINVAL (NULL out/desc, out-of-range field), FIF_ENOMEM,
 * FIF_ECUDA. */
fif_status fif_plan_create(fif_plan_t* out, const fif_plan_desc* desc, void* cuda_stream);

/* Free the plan and everything it owns.  Synchronizes the plan's stream.
 * NULL is accepted. */
fif_status fif_plan_destroy(fif_plan_t plan);

/* Change the stream later calls run on. */
fif_status fif_plan_set_stream(fif_plan_t plan, void* cuda_stream);

/* Build (if not yet built) the tables for every length in lengths[0..count)
 * (HOST array).  Blocking.  Errors: FIF_EINVAL, FIF_EUNSUPPORTED (length not
 * of the form 2^a 3^b, or above max_n), FIF_ENOMEM, FIF_ECUDA. */
fif_status fif_plan_prepare(fif_plan_t plan, const int64_t* lengths, int64_t count);

/* Decompose ONE signal of length n (2^a 3^b, 4 <= n <= max_n) with the plain
 * staged path: one kernel launch per step of the method per outer iteration
 * (R2C; m selection; multiplier and spectral remainder update; C2R with the
 * remainder update and the extrema count), the remainder spectrum and work
 * arrays staged through the plan's device scratch.  Lengths whose transform
 * does not fit one CTA's shared memory (or every length under
 * FIF_FORCE_MULTIPASS) take the multi-pass path instead: FFTs as two passes
 * through global memory, the m search spread over the whole GPU.
 *   signal    [n]                      input samples
 *   imfs      [(max_imfs+1) * n]       row K = IMF K, row n_imfs = final remainder;
 *                                      rows after n_imfs are not written
 *   m         [max_imfs]               inner iteration count per IMF
 *   mask_len  [max_imfs]               L per IMF (input under FIF_FORCE_L)
 *   n_imfs    [1]                      number of IMFs
 *   sig_status[1]                      stop reason | flags
 *   diag      [max_imfs+1] or NULL     optional fif_imf_diag records
 * Errors: FIF_EINVAL, FIF_EUNSUPPORTED, FIF_ENOMEM, FIF_ECUDA. */
fif_status fif_decompose(fif_plan_t plan, const float* signal, int64_t n, float* imfs, int32_t* m,
                         int32_t* mask_len, int32_t* n_imfs, int32_t* sig_status, fif_imf_diag* diag);

/* Decompose a batch of independent signals of any lengths.  Signals are
 * grouped by length into classes: lengths up to fif_fused_max_n() run in one
 * fused launch per class (each CTA keeps a whole signal's spectrum, work
 * array and remainder in shared memory and runs every outer iteration on
 * chip); longer ones run the multi-pass path, one sequence of grid-wide
 * kernels per class.  The first call with a new layout (offsets, pointers,
 * stream) captures every class's launches into one CUDA graph, the classes on
 * parallel branches; later calls with the same layout replay it.  Inside a
 * stream capture of the caller's, the launches are only enqueued.
 *   signals     packed samples; signal i is signals[offsets[i] .. offsets[i+1])
 *   offsets     HOST int64[batch+1], offsets[0] = 0, non-decreasing
 *   imfs        packed outputs; signal i's (max_imfs+1) x n_i block starts at out_offsets[i]
 *   out_offsets HOST int64[batch]
 *   m, mask_len [batch * max_imfs]   (row i = signal i)
 *   n_imfs, sig_status [batch]
 *   diag        [batch * (max_imfs+1)] or NULL
 * Lengths must be 2^a 3^b with 4 <= n_i <= max_n.
 * Errors: FIF_EINVAL, FIF_EUNSUPPORTED, FIF_ENOMEM, FIF_ECUDA. */
fif_status fif_decompose_batch(fif_plan_t plan, const float* signals, const int64_t* offsets,
                               int64_t batch, float* imfs, const int64_t* out_offsets, int32_t* m,
                               int32_t* mask_len, int32_t* n_imfs, int32_t* sig_status,
                               fif_imf_diag* diag);

/* Same as fif_decompose_batch, but every data pointer (signals, imfs, m,
 * mask_len, n_imfs, sig_status, diag) is a HOST pointer; returns after the
 * results are in host memory (blocking).  A buffer in page-locked memory that
 * is mapped into the device's address space (cudaMallocHost, cudaHostAlloc,
 * or cudaHostRegister with mapping) is read or written in place by the
 * kernels, so its transfer over the host link overlaps the computation.  Any
 * other buffer is staged: copied to the plan's device buffers before the
 * batch, or from them after it.  Rows after n_imfs of an in-place imfs buffer
 * are left untouched (as on the device path). */
fif_status fif_decompose_batch_host(fif_plan_t plan, const float* signals, const int64_t* offsets,
                                    int64_t batch, float* imfs, const int64_t* out_offsets,
                                    int32_t* m, int32_t* mask_len, int32_t* n_imfs,
                                    int32_t* sig_status, fif_imf_diag* diag);

/* ---- schedule autotuning per length class ---------------------------------
 * The fused kernel's FFT schedule (elements per thread E, hence E-point
 * register butterflies and Nc/E threads per CTA) has one to four valid
 * choices per length; the multi-pass path's two FP32 inverse levels (the
 * transform of Nc = R1 R2 points as R2 sub-FFTs of R1 points, then R1 of R2)
 * each have a sub-FFT schedule E and a count TJ of sub-FFTs per CTA.  The
 * library picks them by fixed rules unless the plan has been tuned.
 *
 * fif_plan_tune runs the batch (same arguments and outputs as
 * fif_decompose_batch) once per candidate schedule of every fused length
 * class in it, times each class's launch with CUDA events after a warm-up,
 * and keeps the fastest schedule per length in the plan; then, for every
 * multi-pass length class, it times whole runs of the class with each
 * candidate (E in {8, 16, 4, 12, 6, 24, 9, 18}, TJ in {4, 3, 2, 1}, as fits) for the first
 * inverse level, keeps the fastest, then does the same for the second.
 * Later calls use the choices.  Results of the last run are left in the
 * outputs (a valid decomposition).  Under FIF_PREC_SPLIT_BF16 the fused
 * schedules stay at E = 16 and nothing is tuned.  Blocking; not allowed
 * during stream capture (FIF_EINVAL).
 * Errors: as fif_decompose_batch. */
fif_status fif_plan_tune(fif_plan_t plan, const float* signals, const int64_t* offsets,
                         int64_t batch, float* imfs, const int64_t* out_offsets, int32_t* m,
                         int32_t* mask_len, int32_t* n_imfs, int32_t* sig_status);

/* The fused schedule the plan uses for length n: *E elements per thread,
 * *threads per CTA, *tuned = 1 if set by tuning or loading, 0 if by the fixed
 * rule.  FIF_EUNSUPPORTED if n does not take the fused path. */
fif_status fif_plan_get_schedule(fif_plan_t plan, int64_t n, int32_t* E, int32_t* threads,
                                 int32_t* tuned);

/* The multi-pass schedule the plan uses for length n: Nc = *R1 * *R2 (n/2
 * complex points for even n, n for odd n), the first FP32 inverse level's
 * sub-FFT elements per thread *E1 and sub-FFTs per CTA *TJ1, the second's *E2
 * and *TJ2; *tuned = 1 if set by tuning or loading.  Builds the length's
 * multi-pass tables if needed (not during stream capture).
 * FIF_EUNSUPPORTED if n takes the fused path (and the plan does not force
 * the multi-pass path) or is not a valid length.  Errors: FIF_EINVAL (NULL). */
fif_status fif_plan_get_multipass_schedule(fif_plan_t plan, int64_t n, int32_t* R1, int32_t* R2,
                                           int32_t* E1, int32_t* TJ1, int32_t* E2, int32_t* TJ2,
                                           int32_t* tuned);

/* Save the plan's tuned schedules to a text file (HOST path; one line
 * "n E" per tuned fused length, "n E1 TJ1 E2 TJ2" per tuned multi-pass
 * length), or load them from one (lines for lengths or schedules the device
 * cannot use are skipped).  Errors: FIF_EINVAL (NULL or unreadable /
 * unwritable path, malformed line). */
fif_status fif_plan_save_tuning(fif_plan_t plan, const char* path);
fif_status fif_plan_load_tuning(fif_plan_t plan, const char* path);

/* Kernel launches one fif_decompose_batch (or fif_decompose_batch_host) call
 * enqueues for the batch layout the plan last prepared: one fused kernel per
 * length class of the fused path, and the multi-pass kernels of every longer
 * class (their number depends on max_imfs, max_inner, the class size and the
 * peak mode).  0 before the first batch call.  Host-side only (no CUDA call).
 * Errors: FIF_EINVAL (NULL argument). */
fif_status fif_plan_batch_launches(fif_plan_t plan, int64_t* launches);

/* ---- allocation-free single-signal entry point ----------------------------
 * The paper has no counterpart to this; it exists for callers of this
 * library that cannot allocate device memory at the moment they decompose:
 * latency-critical code (cudaMalloc synchronises the device and can take
 * milliseconds), hosts that hand all device memory to their own pool at
 * start-up, and plug-in integrations that may only allocate during setup.
 *
 * Same method, parameters and outputs as fif_decompose, but no plan: desc is
 * read on every call (desc->max_n is ignored) and every array besides the
 * caller's inputs and outputs lives in one fixed file-scope device array of
 * the library (FIF_NOALLOC_SCRATCH_BYTES = 656,640 bytes, sized for
 * FIF_NOALLOC_MAX_N), which each GPU that loads the library keeps until the
 * process exits.  The call allocates and frees nothing.  It runs the staged
 * path's schedule for n, so its integers (m, L, IMF count) equal
 * fif_decompose's.
 *   - n must be 2^a 3^b with 4 <= n <= FIF_NOALLOC_MAX_N; larger n returns
 *     FIF_EUNSUPPORTED, smaller FIF_EINVAL.
 *   - The first call on each device looks up the device address of the array
 *     (with that device current) and keeps it for later calls; make that
 *     first call before any stream capture.  The address stays valid for the
 *     life of the device's primary context: after cudaDeviceReset the library
 *     must not be called again in that process.
 *   - On entry the call reads and clears a pending (non-sticky) CUDA error of
 *     the calling thread, so that an earlier, unrelated failure is not
 *     reported as this call's.
 *   - All calls share the array.  Each call rewrites everything it reads from
 *     it, but calls whose GPU work overlaps (several streams, several host
 *     threads) race on it and must be serialised by the caller.
 * Pointers: signal, imfs, m, mask_len, n_imfs, sig_status, diag as in
 * fif_decompose (device memory); cuda_stream is a cudaStream_t or NULL.
 * Errors: FIF_EINVAL, FIF_EUNSUPPORTED, FIF_ECUDA. */
#define FIF_NOALLOC_MAX_N 16384
#define FIF_NOALLOC_SCRATCH_BYTES 656640
fif_status fif_decompose_noalloc(const fif_plan_desc* desc, const float* signal, int64_t n,
                                 float* imfs, int32_t* m, int32_t* mask_len, int32_t* n_imfs,
                                 int32_t* sig_status, fif_imf_diag* diag, void* cuda_stream);

/* Largest n the fused (shared-memory resident) batch path supports on the
 * current device (0 if the device query fails). */
int64_t fif_fused_max_n(void);

/* Static string for a status code. */
const char* fif_status_string(fif_status status);

#ifdef __cplusplus
}
#endif
#endif /* FIF_H */
