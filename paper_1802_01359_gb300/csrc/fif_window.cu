// Window table of a shape-generated window (the double-convolution
// construction of Theorem 4, discretised as in eq. W_m): for half-support L
// the filter is h_i = g((i + 1/2)/L), i < L, g the piecewise-linear
// interpolant of the shape's samples on [0, 1], and the window is the
// autocorrelation h * h divided by its sum, so that
//   w_hat_k = |H_k|^2 / H_0^2,   H_k = sum_i h_i exp(-2 pi i k i / n).
// One CTA per L writes row L-1 of
//   om64[(L-1) P + k] = 1 - w_hat_k                       (binary64)
//   wtab[(L-1) P + k] = { log2(1 - w_hat_k), w_hat_k }    (rounded to FP32)
// H comes from a float-float R2C FFT of h / sum(h) (about 1e-13 absolute per
// bin).  Where 1 - w_hat_k < 2^-12 (the bins next to DC) that difference of
// squares has lost its leading digits, and the bin is redone in binary64
// from a sum of non-negative terms, the phase centred on the centroid c of h:
//   H_0^2 - |H_k|^2 = (H_0 - C)(H_0 + C) - S^2,
//   H_0 - C = 2 sum_i h_i sin^2(pi k (i - c)/n),  S = sum_i h_i sin(2 pi k (i - c)/n),
// where S is third order in k (i - c)/n and nothing cancels.  Both routes
// leave log2(1 - w_hat_k) good to well under 4 FP32 ulps, the accuracy the
// m screen assumes of the table.
#include "fif_device.cuh"

namespace fif {

__device__ __forceinline__ void put_row(float2* wtab, double* om64, size_t idx, double w, double om,
                                        double hl) {
  om64[idx] = om;
  wtab[idx] = make_float2((float)hl, (float)w);
}

template <int E>
__global__ void __launch_bounds__(512, 1) shape_window_kernel(FftSched S, const double* __restrict__ g,
                                                           int glen, float2* __restrict__ wtab,
                                                           double* __restrict__ om64) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RedScratch red;
  __shared__ ffc nyq;
  ffc* zf = reinterpret_cast<ffc*>(smem);
  const int tid = threadIdx.x, nt = blockDim.x, n = S.n, P = S.P, Nc = S.Nc;
  const int L = blockIdx.x + 1;
  const size_t row = (size_t)(L - 1) * (size_t)P;

  // sum and centroid of h
  double s0 = 0.0, s1 = 0.0;
  for (int i = tid; i < L; i += nt) {
    const double h = shape_tap(g, glen, L, i);
    s0 += h;
    s1 += h * (double)i;
  }
  block_reduce2(s0, s1, OpAdd(), 0.0, &red);
  const double inv = 1.0 / s0, c = s1 / s0;

  // h / sum(h) in float-float, two real samples per complex point (even n)
  if (!S.odd) {
    for (int t = tid; t < Nc; t += nt) {
      const double a = 2 * t < L ? shape_tap(g, glen, L, 2 * t) * inv : 0.0;
      const double b = 2 * t + 1 < L ? shape_tap(g, glen, L, 2 * t + 1) * inv : 0.0;
      zf[t] = ffc{ff_from_double(a), ff_from_double(b)};
    }
  } else {
    for (int t = tid; t < n; t += nt)
      zf[t] = ffc{ff_from_double(t < L ? shape_tap(g, glen, L, t) * inv : 0.0), ff{0.f, 0.f}};
  }
  __syncthreads();
  fft_inplace<ffc, false, E>(zf, S, S);
  if (!S.odd) {
    // unpack the half-length transform: X_k = E_k + W^k O_k, X_{Nc-k} =
    // conj(E_k - W^k O_k), E = (Z_k + conj Z_{Nc-k})/2, O = -i (Z_k - conj Z_{Nc-k})/2
    for (int k = tid; k <= Nc / 2; k += nt) {
      const ffc zk = zf[k];
      const ffc zc = cconj(zf[k == 0 ? 0 : Nc - k]);
      const ffc e = chalf(cadd(zk, zc));
      const ffc o = rot_i<false>(chalf(csub(zk, zc)));
      const ffc wo = cmul(load_tw<ffc, false>(S, k), o);
      zf[k] = cadd(e, wo);
      if (k == 0)
        nyq = cconj(csub(e, wo));
      else
        zf[Nc - k] = cconj(csub(e, wo));
    }
    __syncthreads();
  }

  // every bin from the FFT; note the last bin that needs the direct sum
  const ffc x0 = zf[0];
  const double h0 = ff_to_double(x0.re), h0i = ff_to_double(x0.im);
  const double p0 = h0 * h0 + h0i * h0i;
  int kdc = 0;
  for (int k = tid; k < P; k += nt) {
    if (k == 0) {
      put_row(wtab, om64, row, 1.0, 0.0, -INFINITY);
      continue;
    }
    const ffc x = (!S.odd && k == Nc) ? nyq : zf[k];
    const double re = ff_to_double(x.re), im = ff_to_double(x.im);
    double w = (re * re + im * im) / p0;
    w = w > 1.0 ? 1.0 : w;
    const double om = 1.0 - w;
    put_row(wtab, om64, row + k, w, om, log1p(-w) * 1.4426950408889634);
    if (om < kShapeDirectBelow) kdc = k;
  }
  int dummy = 0;
  block_reduce2(kdc, dummy, OpMax(), 0, &red);

  // bins 1..kdc again, one warp per bin: the centred sums in binary64
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  for (int k = 1 + warp; k <= kdc; k += nwarps) {
    const double om = shape_om_direct(g, glen, L, n, k, c, inv);
    if (lane == 0) put_row(wtab, om64, row + k, 1.0 - om, om, log2(om));
  }
}

#define FIF_E_LIST(X) X(2) X(3) X(4) X(6) X(8) X(9) X(12) X(16) X(18) X(24) X(27)

template <int E>
static cudaError_t launch_shape_e(const FftSched& s, const double* g, int glen, float2* wtab,
                                  double* om64, cudaStream_t st) {
  const size_t ff_bytes = (size_t)s.Nc * sizeof(ffc);
  cudaError_t e = cudaFuncSetAttribute(shape_window_kernel<E>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ff_bytes);
  if (e != cudaSuccess) return e;
  shape_window_kernel<E><<<s.Lmax, sched_threads(s), ff_bytes, st>>>(s, g, glen, wtab, om64);
  return cudaGetLastError();
}

cudaError_t build_shape_window(const FftSched& s, const double* g, int glen, float2* wtab,
                               double* om64, cudaStream_t st) {
  switch (s.E) {
#define FIF_CASE(e) \
  case e:           \
    return launch_shape_e<e>(s, g, glen, wtab, om64, st);
    FIF_E_LIST(FIF_CASE)
#undef FIF_CASE
  }
  return cudaErrorInvalidValue;
}

}  // namespace fif
