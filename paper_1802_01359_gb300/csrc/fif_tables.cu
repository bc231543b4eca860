// Plan-time tables for one signal length n, computed in binary64 on the GPU
// and rounded once:
//   tw[t]     = exp(-2 pi i t/n), t = 0..n-1             (FFT twiddles, float2)
//   tw_lo[t]  = exp(-2 pi i t/n) - tw[t], rounded          (float-float twiddles)
//   sin64[t]  = sin(pi t/n), t = 0..n/2                  (binary64 tie-break path)
//   wtab[(L-1) P + k] = { log2(1 - w_hat_k(L)), w_hat_k(L) },  L = 1..Lmax, k = 0..P-1
// with w_hat_k(L) = [sin(pi k L/n) / (L sin(pi k/n))]^2, w_hat_0 = 1: the
// eigenvalues of the circulant built from the sampled triangle (eq. Lambdas,
// eq. eig2; the taps are the autocorrelation of a length-L box).  The paper
// suggests storing the window's eigenvalues for every support length ahead of
// time (end of Sec. 3 and Sec. 4); this is that table.
#include "fif_internal.h"

namespace fif {

__global__ void twiddle_kernel(float2* tw, float2* tw_lo, double* sin64, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    double s, c;
    sincospi(2.0 * (double)t / (double)n, &s, &c);
    const float ch = (float)c, sh = (float)(-s);
    tw[t] = make_float2(ch, sh);
    tw_lo[t] = make_float2((float)(c - (double)ch), (float)(-s - (double)sh));
  }
  if (t <= n / 2) sin64[t] = sinpi((double)t / (double)n);
}

__global__ void window_kernel(float2* wtab, int n, int P, int Lmax) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)Lmax * P;
  if (idx >= total) return;
  const int L = (int)(idx / P) + 1;
  const int k = (int)(idx % P);
  double w;
  if (k == 0) {
    w = 1.0;
  } else {
    long long t = ((long long)k * (long long)L) % n;
    if (t > n - t) t = n - t;
    const double num = sinpi((double)t / (double)n);
    const double den = (double)L * sinpi((double)k / (double)n);
    w = (num / den) * (num / den);
    w = w > 1.0 ? 1.0 : (w < 0.0 ? 0.0 : w);
  }
  const double hl = log1p(-w) * 1.4426950408889634;  // log2(1 - w); -inf at w = 1
  wtab[idx] = make_float2((float)hl, (float)w);
}

cudaError_t build_tables(int n, int P, int Lmax, float2* tw, float2* tw_lo, float2* wtab,
                         double* sin64, cudaStream_t st) {
  twiddle_kernel<<<(n + 255) / 256, 256, 0, st>>>(tw, tw_lo, sin64, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long total = (long long)Lmax * P;
  const long long blocks = (total + 255) / 256;
  window_kernel<<<(unsigned)blocks, 256, 0, st>>>(wtab, n, P, Lmax);
  return cudaGetLastError();
}

}  // namespace fif

namespace fif {

// Twiddles and the binary64 sine table only (no window table), into caller
// memory.
cudaError_t build_twiddles(int n, float2* tw, float2* tw_lo, double* sin64, cudaStream_t st) {
  twiddle_kernel<<<(n + 255) / 256, 256, 0, st>>>(tw, tw_lo, sin64, n);
  return cudaGetLastError();
}

}  // namespace fif

namespace fif {

// Per-pass twiddles of an FFT schedule (the inverse direction), gathered from
// the binary64-rounded table tw[t] = exp(-2 pi i t/n): for the pass with
// radix R over sub-transforms of Ns points (Ns = product of the earlier
// radices), entry (Ns - 1) + (r - 1) Ns + k, 1 <= r < R, 0 <= k < Ns, holds
// exp(+2 pi i r k / (Ns R)) = conj tw[r k n / (Ns R)].  The passes' blocks tile
// [0, Nc - 1) (sum over passes of Ns (R - 1) = Nc - 1), each r-major so that a
// warp's consecutive k read consecutive entries.
__global__ void pass_twiddle_kernel(float2* ptw, const float2* __restrict__ tw, int n, int Nc,
                                    int npass, PassRadix pr) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Nc - 1) return;
  int Ns = 1;
  for (int p = 0; p < npass; p++) {
    const int R = pr.r[p];
    const int base = Ns - 1, span = Ns * (R - 1);
    if (idx >= base && idx < base + span) {
      const int o = idx - base, r = o / Ns + 1, k = o % Ns;
      const long long t = (long long)r * k * (n / (Ns * R));
      const float2 w = tw[t];
      ptw[idx] = make_float2(w.x, -w.y);
      return;
    }
    Ns *= R;
  }
}

cudaError_t build_pass_twiddles(const FftSched& s, float2* ptw, cudaStream_t st) {
  PassRadix pr;
  for (int p = 0; p < kMaxPass; p++) pr.r[p] = p < s.npass ? s.radix[p] : 1;
  if (s.Nc < 2) return cudaSuccess;
  pass_twiddle_kernel<<<(s.Nc + 254) / 256, 256, 0, st>>>(ptw, s.tw, s.n, s.Nc, s.npass, pr);
  return cudaGetLastError();
}

}  // namespace fif

namespace fif {

// Multipliers of the usual m = max_inner for every (L, k):
//   gtab[(L-1) P + k] = { (1 - w_hat_k)^m, 1 - (1 - w_hat_k)^m },
// in binary64 ((1-w)^m = pow(1-w, m), the complement -expm1(m log1p(-w)),
// without cancellation), rounded once.  With gamma > 0 a bin with
// (1-w)^m >= 1 - gamma passes whole (eq. I_gamma): {1, 0}.  w_hat from the
// triangle's closed form (om64 == nullptr) or the shape window's binary64
// rows of 1 - w_hat (om64[(L-1) P + k]).
__global__ void mult_table_kernel(float2* gtab, const double* __restrict__ om64, int n, int P,
                                  int Lmax, int m, double gamma) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)Lmax * P;
  if (idx >= total) return;
  const int L = (int)(idx / P) + 1;
  const int k = (int)(idx % P);
  double om;
  if (om64) {
    om = om64[idx];
  } else if (k == 0) {
    om = 0.0;
  } else {
    long long t = ((long long)k * (long long)L) % n;
    if (t > n - t) t = n - t;
    const double num = sinpi((double)t / (double)n);
    const double den = (double)L * sinpi((double)k / (double)n);
    double w = (num / den) * (num / den);
    w = w > 1.0 ? 1.0 : (w < 0.0 ? 0.0 : w);
    om = 1.0 - w;
  }
  double g = pow(om, (double)m);
  double keep = -expm1((double)m * log(om));  // log(0) = -inf: keep = 1
  if (gamma > 0.0 && g >= 1.0 - gamma) {
    g = 1.0;
    keep = 0.0;
  }
  gtab[idx] = make_float2((float)g, (float)keep);
}

cudaError_t build_mult_table(int n, int P, int Lmax, int m, double gamma, const double* om64,
                             float2* gtab, cudaStream_t st) {
  const long long total = (long long)Lmax * P;
  mult_table_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(gtab, om64, n, P, Lmax, m,
                                                                     gamma);
  return cudaGetLastError();
}

}  // namespace fif
