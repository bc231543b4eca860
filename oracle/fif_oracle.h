/*
 * FP64 CPU oracle for Iterative Filtering / Fast Iterative Filtering
 * (Cicone & Zhou, "Numerical Analysis for Iterative Filtering with New
 * Efficient Implementations Based on FFT").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this code; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * constant with the CUDA library: its status codes below are written out
 * here independently and are compared by value in the tests.
 *
 * Two tiers, same outer loop (Algorithm 2, Section 3):
 *   tier A  fifo_iterative(): the discrete IF of Algorithm 2 literally --
 *           repeated periodic convolution with the sampled window (the
 *           triangle, or the taps of a shape-generated window; eq. s_m+1,
 *           eq. MatrixForm, eq. W_m), stopping rule eq. SD.
 *   tier B  fifo_direct(): the FIF direct method of Section 4
 *           (eq. One step_algo): DFT, multiply the spectrum by (1-w_hat)^m,
 *           inverse DFT, with m chosen by evaluating eq. SD for
 *           successively larger m through Parseval (Theorem 2 proof,
 *           Theorem 5); the remainder spectrum is updated by the factor
 *           1 - (1-w_hat)^m.
 * Both run entirely in double precision.  They agree (Theorem 5) except
 * where a window eigenvalue is exactly 0 and the same L is used again: exact
 * arithmetic leaves that bin of the remainder empty, tier B keeps it empty,
 * tier A carries binary64 round-off in it, and at large j that round-off can
 * decide m.  Tier B is the reference for such cases (it is pinned against
 * Algorithm 2 run in 60-digit arithmetic).
 */
#ifndef FIF_ORACLE_H
#define FIF_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

/* stop reasons (low byte of the status word) */
#define FIFO_STOP_EXTREMA     1  /* fewer than 2 extrema (Algorithm 1/2 outer test) */
#define FIFO_STOP_MASK        2  /* 2L-1 > n: the window would wrap the period (Sec. 3.1, l <= (n-1)/2) */
#define FIFO_STOP_MAX_IMFS    3  /* max_imfs IMFs produced */
#define FIFO_STOP_FORCED_END  4  /* forced schedule ran out (L_in[K] <= 0) */
#define FIFO_STOP_NONFINITE   5  /* NaN or Inf in the input */
/* flags (OR-ed above the low byte) */
#define FIFO_FLAG_NEAR_DELTA_TIE (1 << 8)  /* |SD_m - delta| or |SD_{m-1} - delta| <= 1e-6 delta */
#define FIFO_FLAG_MASK_TIE       (1 << 9)  /* peak mask rule: another bin within 1e-5 of the peak */
#define FIFO_FLAG_MAX_INNER_HIT  (1 << 10) /* no j <= max_inner had SD_j < delta */
#define FIFO_FLAG_L_CLAMPED      (1 << 12) /* mask length rule gave L < 2; clamped to 2 */

typedef struct {
  double nu;          /* eq. Unif_Mask_length tuning parameter, ~1.6 */
  int mask_scale;     /* L = mask_scale * floor(nu*n/k); 1 or 2 (eq. Unif_Mask_length has 2) */
  double delta;       /* stopping threshold of eq. SD */
  int max_inner;      /* cap on the number of inner iterations (Sec. 3, after eq. SD) */
  int max_imfs;       /* cap on the number of IMFs (remainder not counted) */
  const int* L_in;    /* if non-NULL: forced half-support per IMF, <= 0 ends the loop */
  int absolute;       /* 0: relative SD (eq. SD); 1: absolute ||u_j-u_{j-1}||_2 (eq. Discrete_Abs_StopCond) */
  int apriori;        /* 1: m = the a-priori N0 of Theorem 5 (eq. N0_discrete), no SD loop */
  double gamma;       /* 0, or the threshold of eq. I_gamma (0 < gamma < 1): bins with
                         (1 - w_hat)^m >= 1 - gamma pass whole into the IMF
                         (eq. IMF_cont_stop_threshold; direct method only) */
  int peak_mask;      /* 1: L from the largest spectral peak k* of r (end of Sec. 2):
                         the mask rule with k = 2 k*; the extrema count still stops */
  const double* shape; /* NULL: the triangle.  Else the generating filter's shape g on [0, 1],
                          shape_len >= 1 equispaced samples (linear interpolation; one sample
                          = a constant): the window of half-support L is the autocorrelation
                          h * h of h_i = g((i + 1/2)/L), i < L (Theorem 4 setting, eq. W_m),
                          divided by its sum.  g >= 0 with g > 0 inside (0, 1).  Not with
                          apriori (its zero-eigenvalue count is the triangle's closed form). */
  int shape_len;
} fifo_params;

/* Per-call outputs.  imfs: (max_imfs+1)*n doubles, row K = IMF K, row n_imfs
 * = final remainder.  m, L: [max_imfs].  kext: [max_imfs+1] extrema count of
 * the remainder at each outer test.  sd_m, sd_prev: [max_imfs] SD_m and
 * SD_{m-1} (SD_0 reported as +inf).  sd_trace (optional, may be NULL):
 * [max_imfs*max_inner], SD_j for j = 1..m of each IMF (rest untouched). */
typedef struct {
  double* imfs;
  int* m;
  int* L;
  int* kext;
  int* n_imfs;
  int* status;
  double* sd_m;
  double* sd_prev;
  double* sd_trace;
  int* imf_flags;     /* NULL, or [max_imfs + 1]: the FIFO_FLAG_* raised at each outer step
                         (entry K: the step that extracted IMF K, or the final stop test) */
} fifo_outputs;

int fifo_iterative(const double* s, long n, const fifo_params* p, const fifo_outputs* o);
int fifo_direct(const double* s, long n, const fifo_params* p, const fifo_outputs* o);

/* building blocks, exported for the pins */
void fifo_dft_bruteforce(const double* re, const double* im, long n, int sign, double* ore, double* oim);
int fifo_fft(double* re, double* im, long n, int sign); /* in place, any n >= 1 */
/* Theorem 5, eq. N0_discrete: the smallest natural N >= 1 with
 * N^N / (N+1)^(N+1) < delta / (snorm sqrt(n-1-kzero)), snorm = ||U^T r||_inf
 * (U^T the unitary DFT), kzero the number of zero eigenvalues of W; returns
 * max_inner+1 if no N <= max_inner qualifies.  *near_tie is set if the left
 * side at the returned N or at N-1 lies within 1e-6 (relative) of the right. */
int fifo_apriori_n0(double snorm, long n, long kzero, double delta, int max_inner, int* near_tie);
/* The largest bin k* of |X_k| over 1 <= k <= n/2 (smallest k among equal
 * magnitudes); *tie is set if another bin in that range is within 1e-5
 * (relative) of it.  0 if every such bin is zero. */
long fifo_spectral_peak(const double* re, const double* im, long n, int* tie);
void fifo_triangle_taps(long n, int L, double* c);   /* c[d mod n], normalized by the sum */
void fifo_window_spectrum(long n, int L, double* w); /* closed form, k = 0..n-1 */
/* Shape-generated window (see fifo_params.shape): the generating filter
 * h_0..h_{L-1}, its autocorrelation taps c[d mod n] (normalized by the sum)
 * and their DFT w_hat_k, k = 0..n-1, by the definition (clamped to [0, 1]).
 * Each returns -1 for an invalid shape or L < 1, -2 if out of memory. */
int fifo_shape_filter(const double* g, int glen, int L, double* h);
int fifo_shape_taps(long n, int L, const double* g, int glen, double* c);
int fifo_shape_spectrum(long n, int L, const double* g, int glen, double* w);
long fifo_count_extrema(const double* r, long n);
long fifo_count_zero_crossings(const double* r, long n);
int fifo_mask_length(long n, long k, double nu, int mask_scale);

#ifdef __cplusplus
}
#endif
#endif
