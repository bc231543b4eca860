/*
 * FP64 CPU oracle for (Fast) Iterative Filtering -- TEST INFRASTRUCTURE ONLY.
 * See fif_oracle.h for the contract.  Every routine here is deliberately the
 * plain, slow form of its definition: no blocking, no fusion, no reordering
 * beyond what the cited passage states.
 *
 * Readings of the paper that this file implements (the paper is silent or
 * ambiguous on these points):
 *  - periodic sampling x_j = j/n for any n (Sec. 3 uses j/(n-1), n odd);
 *  - the discrete triangle is the continuous triangle of eq. triangular with
 *    half-support L sampled at integer offsets: c_d = (L-|d|)/L^2, |d| < L,
 *    then normalised by its sum as Sec. 3 says the implemented code does;
 *  - an extremum of the periodic sequence r is an index i with
 *    d_{i-1} d_i < 0, d_i = r[(i+1) mod n] - r[i]; flat steps count none;
 *  - L = mask_scale * floor(nu*n/k) evaluated in binary64 as ((nu*n)/k),
 *    clamped to 2; the loop stops when 2L-1 > n (window wider than the
 *    period, Sec. 3.1 asks l <= (n-1)/2);
 *  - m counts applications of (I-W); SD_j compares iterates j and j-1;
 *    m = first j in [1, max_inner] with SD_j < delta, else max_inner;
 *  - 0^0 = 1 (the DC bin keeps weight 1 at j = 1);
 *  - a shape window takes the double-convolution construction of Theorem 4
 *    discretely: the filter h samples the shape at the cell midpoints
 *    (i + 1/2)/L, i < L, and the window is h * h divided by its sum, so its
 *    half-support is L like the triangle's, and a constant shape gives back
 *    the triangle (box * box) exactly.
 */
#include "fif_oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ DFT */

/* Definition of the DFT, O(n^2): X_k = sum_j x_j exp(sign*2*pi*i*j*k/n).
 * The product j*k is reduced mod n in integers before the angle is formed. */
void fifo_dft_bruteforce(const double* re, const double* im, long n, int sign, double* ore,
                         double* oim) {
  for (long k = 0; k < n; k++) {
    double sr = 0.0, si = 0.0;
    for (long j = 0; j < n; j++) {
      long q = (long)(((long long)j * (long long)k) % (long long)n);
      double a = (double)sign * 2.0 * M_PI * (double)q / (double)n;
      double c = cos(a), s = sin(a);
      double xr = re[j], xi = im ? im[j] : 0.0;
      sr += xr * c - xi * s;
      si += xr * s + xi * c;
    }
    ore[k] = sr;
    oim[k] = si;
  }
}

static long smallest_prime_factor(long n) {
  for (long p = 2; p * p <= n; p++)
    if (n % p == 0) return p;
  return n;
}

/* Recursive decimation in time on the smallest prime factor p of n:
 * with j = p*t + r,  X_k = sum_r w_n^{r k} Y_r[k mod m],  m = n/p,
 * Y_r = DFT_m of the subsequence x[r], x[r+p], ...  (Cooley-Tukey). */
static void fft_rec(const double complex* in, long stride, long n, int sign, double complex* out,
                    double complex* tmp) {
  if (n == 1) {
    out[0] = in[0];
    return;
  }
  long p = smallest_prime_factor(n), m = n / p;
  for (long r = 0; r < p; r++) fft_rec(in + r * stride, stride * p, m, sign, out + r * m, tmp);
  for (long k = 0; k < n; k++) {
    double complex acc = 0.0;
    for (long r = 0; r < p; r++) {
      long q = (long)(((long long)r * (long long)k) % (long long)n);
      double a = (double)sign * 2.0 * M_PI * (double)q / (double)n;
      acc += (cos(a) + I * sin(a)) * out[r * m + (k % m)];
    }
    tmp[k] = acc;
  }
  memcpy(out, tmp, (size_t)n * sizeof(double complex));
}

int fifo_fft(double* re, double* im, long n, int sign) {
  if (n < 1) return -1;
  double complex* x = malloc((size_t)n * sizeof(double complex));
  double complex* y = malloc((size_t)n * sizeof(double complex));
  double complex* t = malloc((size_t)n * sizeof(double complex));
  if (!x || !y || !t) {
    free(x), free(y), free(t);
    return -2;
  }
  for (long j = 0; j < n; j++) x[j] = re[j] + I * (im ? im[j] : 0.0);
  fft_rec(x, 1, n, sign, y, t);
  for (long j = 0; j < n; j++) {
    re[j] = creal(y[j]);
    if (im) im[j] = cimag(y[j]);
  }
  free(x), free(y), free(t);
  return 0;
}

/* ------------------------------------------------------ window and mask */

/* Triangle of eq. triangular with half-support L, sampled at the integer
 * offsets d (|d| < L), stored circularly at index d mod n, then divided by
 * its sum so that W is row stochastic (Sec. 3, rectangle-rule remark). */
void fifo_triangle_taps(long n, int L, double* c) {
  for (long i = 0; i < n; i++) c[i] = 0.0;
  double sum = 0.0;
  for (long d = -(L - 1); d <= L - 1; d++) {
    double v = ((double)L - fabs((double)d)) / ((double)L * (double)L);
    long idx = ((d % n) + n) % n;
    c[idx] += v;
    sum += v;
  }
  for (long i = 0; i < n; i++) c[i] /= sum;
}

/* |sin(pi*q/n)| for an integer q, with the argument reduced exactly. */
static double abs_sinpi_ratio(long long q, long n) {
  long long t = q % (long long)n;
  if (t < 0) t += n;
  if (t > n - t) t = n - t; /* |sin| is symmetric about n/2 */
  return sin(M_PI * (double)t / (double)n);
}

/* Eigenvalues of the circulant W built from the triangle taps (eq. Lambdas,
 * eq. eig2).  The taps are the autocorrelation of a length-L box, so
 * lambda_k = |DFT(box)_k|^2 = [sin(pi k L/n) / (L sin(pi k/n))]^2, lambda_0
 * = 1 (the discrete counterpart of eq. triangular_fourier).  Clamped to
 * [0, 1] (Corollary 2). */
void fifo_window_spectrum(long n, int L, double* w) {
  for (long k = 0; k < n; k++) {
    double v;
    if (k == 0) {
      v = 1.0;
    } else {
      double num = abs_sinpi_ratio((long long)k * (long long)L, n);
      double den = (double)L * abs_sinpi_ratio(k, n);
      v = (num / den) * (num / den);
    }
    if (v > 1.0) v = 1.0;
    if (v < 0.0) v = 0.0;
    w[k] = v;
  }
}

/* A shape g is usable when its samples are finite and >= 0 and its linear
 * interpolant is > 0 on the open interval (0, 1): every h_i is then > 0 and
 * the window has a positive sum. */
static int shape_valid(const double* g, int glen) {
  if (!g || glen < 1) return 0;
  for (int j = 0; j < glen; j++)
    if (!isfinite(g[j]) || g[j] < 0.0) return 0;
  if (glen == 1) return g[0] > 0.0;
  if (glen == 2) return g[0] + g[1] > 0.0;
  for (int j = 1; j < glen - 1; j++)
    if (!(g[j] > 0.0)) return 0;
  return 1;
}

/* Generating filter of half-support L: h_i = g((i + 1/2)/L), i = 0..L-1,
 * with g the piecewise-linear interpolant of glen equispaced samples on
 * [0, 1] (a constant when glen = 1).  The window of eq. W_m is then the
 * autocorrelation of h (the double-convolution construction of Theorem 4),
 * so its spectrum is |DFT(h)|^2 / (sum h)^2, inside [0, 1]. */
int fifo_shape_filter(const double* g, int glen, int L, double* h) {
  if (!shape_valid(g, glen) || L < 1 || !h) return -1;
  for (int i = 0; i < L; i++) {
    if (glen == 1) {
      h[i] = g[0];
      continue;
    }
    const double t = ((double)i + 0.5) / (double)L * (double)(glen - 1);
    int j = (int)floor(t);
    if (j > glen - 2) j = glen - 2;
    const double f = t - (double)j;
    h[i] = (1.0 - f) * g[j] + f * g[j + 1];
  }
  return 0;
}

/* a[d] = sum_i h_i h_{i+d}, d = 0..L-1 (the autocorrelation of h, even in d). */
static int shape_autocorrelation(const double* g, int glen, int L, double* a) {
  double* h = malloc((size_t)L * sizeof(double));
  if (!h) return -2;
  const int rc = fifo_shape_filter(g, glen, L, h);
  if (rc == 0)
    for (int d = 0; d < L; d++) {
      double v = 0.0;
      for (int i = 0; i + d < L; i++) v += h[i] * h[i + d];
      a[d] = v;
    }
  free(h);
  return rc;
}

/* Taps of the shape window at the offsets |d| < L, stored circularly at
 * index d mod n and divided by their sum (row-stochastic W, as for the
 * triangle). */
int fifo_shape_taps(long n, int L, const double* g, int glen, double* c) {
  if (L < 1 || n < 1 || !c) return -1;
  double* a = malloc((size_t)L * sizeof(double));
  if (!a) return -2;
  const int rc = shape_autocorrelation(g, glen, L, a);
  if (rc == 0) {
    for (long i = 0; i < n; i++) c[i] = 0.0;
    double sum = 0.0;
    for (long d = -(L - 1); d <= L - 1; d++) {
      const double v = a[d < 0 ? -d : d];
      c[((d % n) + n) % n] += v;
      sum += v;
    }
    for (long i = 0; i < n; i++) c[i] /= sum;
  }
  free(a);
  return rc;
}

/* cos(2 pi q / n) for an integer q, with the argument reduced exactly. */
static double cos2pi_ratio(long long q, long n) {
  long long t = q % (long long)n;
  if (t < 0) t += n;
  return cos(2.0 * M_PI * (double)t / (double)n);
}

/* Eigenvalues of the circulant W of the shape window (eq. Lambdas): the DFT
 * of its even taps, w_hat_k = (a_0 + 2 sum_{d>=1} a_d cos(2 pi k d/n)) /
 * (a_0 + 2 sum_{d>=1} a_d), by the definition; clamped to [0, 1]. */
int fifo_shape_spectrum(long n, int L, const double* g, int glen, double* w) {
  if (L < 1 || n < 1 || !w) return -1;
  double* a = malloc((size_t)L * sizeof(double));
  if (!a) return -2;
  const int rc = shape_autocorrelation(g, glen, L, a);
  if (rc == 0) {
    double sum = a[0];
    for (int d = 1; d < L; d++) sum += 2.0 * a[d];
    for (long k = 0; k < n; k++) {
      double v = a[0];
      for (int d = 1; d < L; d++) v += 2.0 * a[d] * cos2pi_ratio((long long)k * d, n);
      v /= sum;
      if (v > 1.0) v = 1.0;
      if (v < 0.0) v = 0.0;
      w[k] = v;
    }
    w[0] = 1.0;
  }
  free(a);
  return rc;
}

/* The window the parameters select: taps (tier A) and spectrum (tier B). */
static int window_taps(long n, int L, const fifo_params* p, double* c) {
  if (p->shape) return fifo_shape_taps(n, L, p->shape, p->shape_len, c);
  fifo_triangle_taps(n, L, c);
  return 0;
}

static int window_spectrum(long n, int L, const fifo_params* p, double* w) {
  if (p->shape) return fifo_shape_spectrum(n, L, p->shape, p->shape_len, w);
  fifo_window_spectrum(n, L, w);
  return 0;
}

long fifo_count_extrema(const double* r, long n) {
  long count = 0;
  for (long i = 0; i < n; i++) {
    double dprev = r[i] - r[(i - 1 + n) % n];
    double dnext = r[(i + 1) % n] - r[i];
    if ((dprev > 0.0 && dnext < 0.0) || (dprev < 0.0 && dnext > 0.0)) count++;
  }
  return count;
}

long fifo_count_zero_crossings(const double* r, long n) {
  long count = 0;
  for (long i = 0; i < n; i++) {
    double a = r[i], b = r[(i + 1) % n];
    if ((a > 0.0 && b < 0.0) || (a < 0.0 && b > 0.0)) count++;
  }
  return count;
}

/* eq. Unif_Mask_length, l = 2 floor(nu N / k); mask_scale selects the
 * leading factor (1 = half-support L = floor(nu n/k)). */
int fifo_mask_length(long n, long k, double nu, int mask_scale) {
  double t = nu * (double)n;
  t = t / (double)k;
  return mask_scale * (int)floor(t);
}

/* ------------------------------------------------------------ outer loop */

static int check_args(const double* s, long n, const fifo_params* p, const fifo_outputs* o) {
  if (!s || n < 1 || !p || !o || !o->imfs || !o->m || !o->L || !o->kext || !o->n_imfs ||
      !o->status || !o->sd_m || !o->sd_prev)
    return -1;
  if (!(p->delta > 0.0) || p->max_inner < 1 || p->max_imfs < 0) return -1;
  if (!p->L_in && (!(p->nu > 0.0) || p->mask_scale < 1)) return -1;
  if (p->shape && (!shape_valid(p->shape, p->shape_len) || p->apriori)) return -1;
  return 0;
}

/* Outer-loop test shared by both tiers (Algorithm 2 "while #extrema >= 2",
 * the max_imfs cap, the window-length limit).  Returns 0 to continue with
 * *L set, else the stop reason. */
long fifo_spectral_peak(const double* re, const double* im, long n, int* tie) {
  long best = 0;
  double bv = 0.0;
  for (long k = 1; k <= n / 2; k++) {
    const double v = re[k] * re[k] + im[k] * im[k];
    if (v > bv) bv = v, best = k;
  }
  *tie = 0;
  for (long k = 1; k <= n / 2 && best; k++)
    if (k != best && re[k] * re[k] + im[k] * im[k] >= bv * (1.0 - 1e-5)) *tie = 1;
  return best;
}

/* peak: the spectral peak k* of r when p->peak_mask (from the caller's spectrum). */
static int outer_test(const double* r, long n, int K, const fifo_params* p, int* kext, int* L,
                      int* flags, long peak, int peak_tie) {
  long k = fifo_count_extrema(r, n);
  kext[K] = (int)k;
  if (p->L_in) {
    if (K == p->max_imfs) return FIFO_STOP_MAX_IMFS;
    *L = p->L_in[K];
    if (*L <= 0) return FIFO_STOP_FORCED_END;
    if (2L * (long)(*L) - 1 > n) return FIFO_STOP_MASK;
    return 0;
  }
  if (k < 2) return FIFO_STOP_EXTREMA;
  if (p->peak_mask) {
    /* a tone of k* cycles has 2 k* extrema: the same rule at that count */
    *L = fifo_mask_length(n, 2 * (peak > 0 ? peak : 1), p->nu, p->mask_scale);
    if (peak_tie) *flags |= FIFO_FLAG_MASK_TIE;
  } else {
    *L = fifo_mask_length(n, k, p->nu, p->mask_scale);
  }
  if (*L < 2) {
    *L = 2;
    *flags |= FIFO_FLAG_L_CLAMPED;
  }
  if (2L * (long)(*L) - 1 > n) return FIFO_STOP_MASK;
  if (K == p->max_imfs) return FIFO_STOP_MAX_IMFS;
  return 0;
}

static int near_tie(double sd, double delta) { return fabs(sd - delta) <= 1e-6 * delta; }

static void finish(const double* r, long n, int K, int reason, int flags, const fifo_outputs* o) {
  memcpy(o->imfs + (size_t)K * (size_t)n, r, (size_t)n * sizeof(double));
  *o->n_imfs = K;
  *o->status = reason | flags;
}

static int all_finite(const double* s, long n) {
  for (long i = 0; i < n; i++)
    if (!isfinite(s[i])) return 0;
  return 1;
}

int fifo_apriori_n0(double snorm, long n, long kzero, double delta, int max_inner, int* near_tie) {
  const long dof = n - 1 - kzero;
  *near_tie = 0;
  if (!(snorm > 0.0) || dof <= 0) return 1; /* the right side is +inf */
  /* both sides in logs: log(N^N / (N+1)^(N+1)) = N log N - (N+1) log(N+1) */
  const double rhs = log(delta) - log(snorm) - 0.5 * log((double)dof);
  double prev = 0.0; /* N = 0: 0^0 / 1 = 1 */
  for (int N = 1; N <= max_inner; N++) {
    const double lhs = (double)N * log((double)N) - (double)(N + 1) * log((double)(N + 1));
    if (lhs < rhs) {
      if (fabs(lhs - rhs) <= 1e-6 || (N > 1 && fabs(prev - rhs) <= 1e-6)) *near_tie = 1;
      return N;
    }
    prev = lhs;
  }
  if (max_inner >= 1 && fabs(prev - rhs) <= 1e-6) *near_tie = 1;
  return max_inner + 1;
}

/* ||U^T r||_inf of the unitary DFT: max_k |DFT(r)_k| / sqrt(n). */
static double unitary_inf_norm(const double* Rre, const double* Rim, long n) {
  double mx = 0.0;
  for (long k = 0; k < n; k++) {
    const double a = sqrt(Rre[k] * Rre[k] + Rim[k] * Rim[k]);
    if (a > mx) mx = a;
  }
  return mx / sqrt((double)n);
}

/* m in the a-priori mode for the remainder spectrum R and window spectrum w. */
static int apriori_m(const double* Rre, const double* Rim, const double* w, long n,
                     const fifo_params* p, int* flags) {
  long kzero = 0;
  for (long k = 1; k < n; k++) kzero += w[k] == 0.0;
  int tie = 0;
  const int N0 = fifo_apriori_n0(unitary_inf_norm(Rre, Rim, n), n, kzero, p->delta, p->max_inner,
                                 &tie);
  if (tie) *flags |= FIFO_FLAG_NEAR_DELTA_TIE;
  if (N0 > p->max_inner) {
    *flags |= FIFO_FLAG_MAX_INNER_HIT;
    return p->max_inner;
  }
  return N0;
}

/* Tier A: Algorithm 2 with a fixed mask length per inner loop (eq.
 * First_IMF_fixed_length), u_j = u_{j-1} - W u_{j-1} by direct periodic
 * convolution with the circulant W of eq. W_m (first column = the taps),
 * stopping rule eq. SD. */
int fifo_iterative(const double* s, long n, const fifo_params* p, const fifo_outputs* o) {
  if (check_args(s, n, p, o)) return -1;
  if (p->gamma != 0.0) return -1; /* thresholding is a spectral operation (direct method) */
  double* r = malloc((size_t)n * sizeof(double));
  double* u = malloc((size_t)n * sizeof(double));
  double* v = malloc((size_t)n * sizeof(double));
  double* c = malloc((size_t)n * sizeof(double));
  if (!r || !u || !v || !c) {
    free(r), free(u), free(v), free(c);
    return -2;
  }
  memcpy(r, s, (size_t)n * sizeof(double));
  int K = 0, flags = 0, reason = 0;
  if (!all_finite(s, n)) {
    finish(r, n, 0, FIFO_STOP_NONFINITE, 0, o);
    free(r), free(u), free(v), free(c);
    return 0;
  }
  for (;;) {
    int L = 0;
    long peak = 0;
    int ptie = 0;
    if (p->peak_mask) {
      double* Xre = malloc((size_t)n * sizeof(double));
      double* Xim = malloc((size_t)n * sizeof(double));
      if (!Xre || !Xim) {
        free(Xre), free(Xim);
        free(r), free(u), free(v), free(c);
        return -2;
      }
      memcpy(Xre, r, (size_t)n * sizeof(double));
      for (long i = 0; i < n; i++) Xim[i] = 0.0;
      fifo_fft(Xre, Xim, n, -1);
      peak = fifo_spectral_peak(Xre, Xim, n, &ptie);
      free(Xre), free(Xim);
    }
    int iflags = 0; /* flags raised at this outer step (recorded per step) */
    reason = outer_test(r, n, K, p, o->kext, &L, &iflags, peak, ptie);
    if (reason) {
      flags |= iflags;
      if (o->imf_flags) o->imf_flags[K] = iflags;
      break;
    }
    if (window_taps(n, L, p, c)) { /* the shape was checked: out of memory */
      free(r), free(u), free(v), free(c);
      return -2;
    }
    memcpy(u, r, (size_t)n * sizeof(double));
    double sd = INFINITY, sd_prev = INFINITY;
    int n0 = 0; /* a-priori mode: exactly n0 applications of (I - W) */
    if (p->apriori) {
      double* Xre = malloc((size_t)n * sizeof(double));
      double* Xim = malloc((size_t)n * sizeof(double));
      double* wk = malloc((size_t)n * sizeof(double));
      if (!Xre || !Xim || !wk) {
        free(Xre), free(Xim), free(wk);
        free(r), free(u), free(v), free(c);
        return -2;
      }
      memcpy(Xre, r, (size_t)n * sizeof(double));
      for (long i = 0; i < n; i++) Xim[i] = 0.0;
      fifo_fft(Xre, Xim, n, -1);
      fifo_window_spectrum(n, L, wk);
      n0 = apriori_m(Xre, Xim, wk, n, p, &iflags);
      free(Xre), free(Xim), free(wk);
    }
    int j;
    for (j = 1; j <= p->max_inner; j++) {
      /* v = W u, (W u)_i = sum_d c[d mod n] u[(i-d) mod n] */
      for (long i = 0; i < n; i++) {
        double acc = 0.0;
        for (long d = -(L - 1); d <= L - 1; d++) {
          long cd = ((d % n) + n) % n;
          long ui = (((i - d) % n) + n) % n;
          acc += c[cd] * u[ui];
        }
        v[i] = acc;
      }
      double num = 0.0, den = 0.0;
      for (long i = 0; i < n; i++) {
        num += v[i] * v[i]; /* ||u_j - u_{j-1}||^2 */
        den += u[i] * u[i]; /* ||u_{j-1}||^2 */
      }
      for (long i = 0; i < n; i++) u[i] -= v[i];
      sd_prev = sd;
      if (p->absolute)
        sd = sqrt(num);
      else
        sd = den > 0.0 ? sqrt(num / den) : 0.0;
      if (o->sd_trace) o->sd_trace[(size_t)K * (size_t)p->max_inner + (size_t)(j - 1)] = sd;
      if (p->apriori ? j == n0 : sd < p->delta) break;
    }
    int m = j > p->max_inner ? p->max_inner : j;
    if (!p->apriori) {
      if (j > p->max_inner) iflags |= FIFO_FLAG_MAX_INNER_HIT;
      if (near_tie(sd, p->delta) || (m > 1 && near_tie(sd_prev, p->delta)))
        iflags |= FIFO_FLAG_NEAR_DELTA_TIE;
    }
    flags |= iflags;
    if (o->imf_flags) o->imf_flags[K] = iflags;
    o->m[K] = m;
    o->L[K] = L;
    o->sd_m[K] = sd;
    o->sd_prev[K] = sd_prev;
    memcpy(o->imfs + (size_t)K * (size_t)n, u, (size_t)n * sizeof(double));
    for (long i = 0; i < n; i++) r[i] -= u[i];
    K++;
  }
  finish(r, n, K, reason, flags, o);
  free(r), free(u), free(v), free(c);
  return 0;
}

/* Tier B: the FIF direct method.  IMF = IDFT((1 - w_hat)^m DFT(r))
 * (eq. One step_algo), m found by evaluating eq. SD for successively larger
 * m through Parseval: ||u_j - u_{j-1}||^2 = (1/n) sum_k |R_k|^2
 * (1-w_k)^{2(j-1)} w_k^2 and ||u_{j-1}||^2 = (1/n) sum_k |R_k|^2
 * (1-w_k)^{2(j-1)} (proof of Theorem 2, Theorem 5).
 * The remainder r - IMF (Algorithm 2) is kept in the spectral domain as
 * well: R <- (1 - (1-w)^m) R, the DFT of r - IMF by linearity, with
 * 1 - (1-w)^m = -expm1(m log1p(-w)).  Where w_k = 0 exactly this empties bin
 * k exactly, as exact arithmetic does; a time-domain subtraction would leave
 * round-off there, and at large j that round-off (weight 1, w = 0) would
 * decide SD_j. */
int fifo_direct(const double* s, long n, const fifo_params* p, const fifo_outputs* o) {
  if (check_args(s, n, p, o)) return -1;
  double* r = malloc((size_t)n * sizeof(double));
  double* Rre = malloc((size_t)n * sizeof(double));
  double* Rim = malloc((size_t)n * sizeof(double));
  double* Ire = malloc((size_t)n * sizeof(double));
  double* Iim = malloc((size_t)n * sizeof(double));
  double* w = malloc((size_t)n * sizeof(double));
  double* E = malloc((size_t)n * sizeof(double));
  if (!r || !Rre || !Rim || !Ire || !Iim || !w || !E) {
    free(r), free(Rre), free(Rim), free(Ire), free(Iim), free(w), free(E);
    return -2;
  }
  memcpy(r, s, (size_t)n * sizeof(double));
  int K = 0, flags = 0, reason = 0;
  if (!all_finite(s, n)) {
    finish(r, n, 0, FIFO_STOP_NONFINITE, 0, o);
    free(r), free(Rre), free(Rim), free(Ire), free(Iim), free(w), free(E);
    return 0;
  }
  for (long i = 0; i < n; i++) {
    Rre[i] = s[i];
    Rim[i] = 0.0;
  }
  fifo_fft(Rre, Rim, n, -1);
  for (;;) {
    int L = 0;
    int ptie = 0;
    const long peak = p->peak_mask ? fifo_spectral_peak(Rre, Rim, n, &ptie) : 0;
    int iflags = 0; /* flags raised at this outer step (recorded per step) */
    reason = outer_test(r, n, K, p, o->kext, &L, &iflags, peak, ptie);
    if (reason) {
      flags |= iflags;
      if (o->imf_flags) o->imf_flags[K] = iflags;
      break;
    }
    if (window_spectrum(n, L, p, w)) { /* the shape was checked: out of memory */
      free(r), free(Rre), free(Rim), free(Ire), free(Iim), free(w), free(E);
      return -2;
    }
    for (long k = 0; k < n; k++) E[k] = Rre[k] * Rre[k] + Rim[k] * Rim[k];
    double sd = INFINITY, sd_prev = INFINITY;
    int j;
    const int n0 = p->apriori ? apriori_m(Rre, Rim, w, n, p, &iflags) : 0;
    for (j = p->apriori ? p->max_inner + 1 : 1; j <= p->max_inner; j++) {
      double num = 0.0, den = 0.0;
      for (long k = 0; k < n; k++) {
        num += E[k] * w[k] * w[k];
        den += E[k];
      }
      sd_prev = sd;
      if (p->absolute)
        sd = sqrt(num / (double)n);
      else
        sd = den > 0.0 ? sqrt(num / den) : 0.0;
      if (o->sd_trace) o->sd_trace[(size_t)K * (size_t)p->max_inner + (size_t)(j - 1)] = sd;
      if (sd < p->delta) break;
      for (long k = 0; k < n; k++) E[k] *= (1.0 - w[k]) * (1.0 - w[k]);
    }
    int m = j > p->max_inner ? p->max_inner : j;
    if (p->apriori) {
      m = n0;
    } else {
      if (j > p->max_inner) iflags |= FIFO_FLAG_MAX_INNER_HIT;
      if (near_tie(sd, p->delta) || (m > 1 && near_tie(sd_prev, p->delta)))
        iflags |= FIFO_FLAG_NEAR_DELTA_TIE;
    }
    flags |= iflags;
    if (o->imf_flags) o->imf_flags[K] = iflags;
    for (long k = 0; k < n; k++) {
      double g = pow(1.0 - w[k], (double)m);
      double keep = -expm1((double)m * log1p(-w[k]));
      if (p->gamma > 0.0 && g >= 1.0 - p->gamma) {
        /* k in I_{w,gamma,m}: w_hat_k taken as 0, the bin passes whole */
        g = 1.0;
        keep = 0.0;
      }
      Ire[k] = g * Rre[k];
      Iim[k] = g * Rim[k];
      Rre[k] *= keep;
      Rim[k] *= keep;
    }
    fifo_fft(Ire, Iim, n, +1);
    double* imf = o->imfs + (size_t)K * (size_t)n;
    for (long i = 0; i < n; i++) imf[i] = Ire[i] / (double)n;
    for (long i = 0; i < n; i++) r[i] -= imf[i];
    o->m[K] = m;
    o->L[K] = L;
    o->sd_m[K] = sd;
    o->sd_prev[K] = sd_prev;
    K++;
  }
  finish(r, n, K, reason, flags, o);
  free(r), free(Rre), free(Rim), free(Ire), free(Iim), free(w), free(E);
  return 0;
}
