// Plain staged path for one signal: each step of one outer iteration is its
// own kernel launch, with the remainder spectrum, the complex work array, the
// time-domain remainder and the loop state in the plan's global scratch:
//   forward   R2C of the input, first extrema count            (1 CTA)
//   select    outer-loop test, window row, m by eq. SD            (1 CTA)
//   multiply  IMF_hat = (1-w_hat)^m r_hat, r_hat -= IMF_hat       (grid over bins)
//   inverse   C2R of IMF_hat, IMF row, r -= IMF, extrema count   (1 CTA)
// The host enqueues forward, then max_imfs+1 rounds of select/multiply/
// inverse; once a stop rule has fired, the remaining launches return at once.
#include "fif_device.cuh"

namespace fif {

// loop state words in scratch.state
enum {
  ST_K = 0, ST_K_EXT, ST_ZC, ST_TIE, ST_FLAGS, ST_DONE, ST_L, ST_M, ST_IFLAGS, ST_SMAX, ST_RMAX,
  ST_WORDS = 16
};

template <int E>
__global__ void __launch_bounds__(512, 1) staged_forward(FftSched S, const float* __restrict__ x,
                                                      StagedScratch scr, Outputs out,
                                                      MethodParams mp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RedScratch red;
  ffc* zf = reinterpret_cast<ffc*>(smem);
  int* st = scr.state;
  const float smax = forward_real<E>(x, scr.rem, zf, scr.spec, S, &red);
  if (smax < 0.f) {
    for (int i = threadIdx.x; i < S.n; i += blockDim.x) out.imfs[i] = x[i];
    if (threadIdx.x == 0) {
      out.n_imfs[0] = 0;
      out.sig_status[0] = FIF_STOP_NONFINITE;
      if (out.diag) out.diag[0] = fif_imf_diag{0, 0, 0, 0.f};
      st[ST_DONE] = 1;
    }
    return;
  }
  const ExtremaInfo e = count_extrema(scr.rem, S.n, tie_tau(smax), &red);
  if (threadIdx.x == 0) {
    st[ST_K] = 0;
    st[ST_K_EXT] = e.k;
    st[ST_ZC] = e.zc;
    st[ST_TIE] = 0;
    st[ST_FLAGS] = 0;
    st[ST_DONE] = 0;
    st[ST_SMAX] = __float_as_int(smax);
    st[ST_RMAX] = __float_as_int(e.rmax);
  }
}

__global__ void __launch_bounds__(512, 1) staged_select(FftSched S, StagedScratch scr, Outputs out,
                                                     MethodParams mp) {
  __shared__ RedScratch red;
  int* st = scr.state;
  if (st[ST_DONE]) return;
  const int K = st[ST_K], k = st[ST_K_EXT], tie = st[ST_TIE];
  int L = 0, iflags = tie ? FIF_FLAG_EXTREMA_TIE : 0;
  SpecPeak pk{0, 0};
  if (mp.peak_mask) pk = spectral_peak(scr.spec, S, &red);
  if (pk.tie) iflags |= FIF_FLAG_EXTREMA_TIE;
  const int reason = outer_test(k, K, S.n, mp, out.mask_len, L, iflags, pk.k);
  if (out.diag && threadIdx.x == 0) {
    out.diag[K].k_extrema = k;
    out.diag[K].zero_crossings = st[ST_ZC];
  }
  if (reason) {
    float* rrow = out.imfs + (size_t)K * S.n;
    for (int i = threadIdx.x; i < S.n; i += blockDim.x) rrow[i] = scr.rem[i];
    if (threadIdx.x == 0) {
      const int flags = st[ST_FLAGS] | (iflags & FIF_FLAG_EXTREMA_TIE);
      out.n_imfs[0] = K;
      out.sig_status[0] = reason | flags;
      if (out.diag) {
        out.diag[K].flags = iflags & FIF_FLAG_EXTREMA_TIE;
        out.diag[K].inf_norm = __int_as_float(st[ST_RMAX]);
      }
      st[ST_DONE] = 1;
    }
    return;
  }
  const float sc = spectrum_scale(S.n, __int_as_float(st[ST_SMAX]));
  const int m = select_m(scr.spec, S, L, mp, sc, iflags, &red);
  if (threadIdx.x == 0) {
    st[ST_L] = L;
    st[ST_M] = m;
    st[ST_IFLAGS] = iflags;
  }
}

__global__ void staged_multiply(FftSched S, StagedScratch scr, MethodParams mp) {
  const int* st = scr.state;
  if (st[ST_DONE]) return;
  const int L = st[ST_L], m = st[ST_M];
  const float2* row = wrow(S, L);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < S.P) {
    const float2 z = scr.spec[k];
    float g, omg;
    multiplier_th(m, __ldg(&row[k]).x, S, L, k, mp, g, omg);
    scr.work[k] = make_float2(g * z.x, g * z.y);
    scr.spec[k] = make_float2(omg * z.x, omg * z.y);
  }
}

template <int E>
__global__ void __launch_bounds__(512, 1) staged_inverse(FftSched S, StagedScratch scr, Outputs out,
                                                      MethodParams mp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RedScratch red;
  int* st = scr.state;
  if (st[ST_DONE]) return;
  float2* work = reinterpret_cast<float2*>(smem);
  float2* smtw = work + ((work_points(S) + 1) & ~(size_t)1);
  for (int k = threadIdx.x; k < S.P; k += blockDim.x) work[k] = scr.work[k];
  for (int u = threadIdx.x; u < S.tw_entries; u += blockDim.x) {
    const float2 w = __ldg(&S.tw[u]);
    smtw[tw_slot(u)] = make_float2(w.x, -w.y);
  }
  __syncthreads();
  const TwSrc ts{smtw, S.tw, S.n, S.tw_fold};
  inverse_real<E>(work, S, ts);
  const int K = st[ST_K];
  const float tau = tie_tau(__int_as_float(st[ST_SMAX]));
  float imax;
  ExtremaInfo e;
  if (!S.odd) {
    const EpiOut eo = epilogue_extrema_even(work, scr.rem, out.imfs + (size_t)K * S.n, S, tau, &red);
    imax = eo.imax;
    e = ExtremaInfo{eo.k, eo.zc, eo.tie, eo.rmax};
  } else {
    imax = store_imf_update_rem(work, scr.rem, out.imfs + (size_t)K * S.n, S, &red);
    e = count_extrema(scr.rem, S.n, tau, &red);
  }
  if (threadIdx.x == 0) {
    const int iflags = st[ST_IFLAGS];
    out.m[K] = st[ST_M];
    if (!mp.force_L) out.mask_len[K] = st[ST_L];
    if (out.diag) {
      out.diag[K].flags = iflags;
      out.diag[K].inf_norm = imax;
    }
    st[ST_FLAGS] |= iflags;
    st[ST_K] = K + 1;
    st[ST_K_EXT] = e.k;
    st[ST_ZC] = e.zc;
    st[ST_TIE] = e.tie;
    st[ST_RMAX] = __float_as_int(e.rmax);
  }
}

#define FIF_E_LIST(X) X(2) X(3) X(4) X(6) X(8) X(9) X(12) X(16) X(18) X(24) X(27)

template <int E>
static cudaError_t launch_staged_e(const FftSched& s, const MethodParams& mp, const float* signal,
                                   const Outputs& out, const StagedScratch& scr, cudaStream_t st) {
  int dev = 0, maxsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int dyn_max = maxsm - (int)sizeof(RedScratch);
  cudaFuncSetAttribute(staged_forward<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
  cudaFuncSetAttribute(staged_inverse<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
  const int threads = sched_threads(s);
  const size_t work_bytes = ((work_points(s) + 1) & ~(size_t)1) * sizeof(float2) +
                            tw_slots(s) * sizeof(float2);
  const size_t ff_bytes = (size_t)s.Nc * sizeof(ffc);
  staged_forward<E><<<1, threads, ff_bytes, st>>>(s, signal, scr, out, mp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int mblocks = (s.P + 255) / 256;
  for (int it = 0; it <= mp.max_imfs; it++) {
    staged_select<<<1, threads, 0, st>>>(s, scr, out, mp);
    staged_multiply<<<mblocks, 256, 0, st>>>(s, scr, mp);
    staged_inverse<E><<<1, threads, work_bytes, st>>>(s, scr, out, mp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_staged(const FftSched& s, const FftSched* /*d_sched*/, const MethodParams& mp,
                          const float* signal, const Outputs& out, const StagedScratch& scr,
                          cudaStream_t st) {
  switch (s.E) {
#define FIF_CASE(e) \
  case e:           \
    return launch_staged_e<e>(s, mp, signal, out, scr, st);
    FIF_E_LIST(FIF_CASE)
#undef FIF_CASE
  }
  return cudaErrorInvalidValue;
}

}  // namespace fif
